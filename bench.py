#!/usr/bin/env python
"""GLS solves per second (SNPs/s) at n = 10^4, p = 4 on one or more B300s.

One step = the whole hot path over 8 blocks of bs = 4096 SNPs (32,768 SNPs)
of the paper-scale workload (n = 10,000 samples, p = 4, int8 dosages;
Sec. 1.4 of the paper): per block, the blocked triangular solve
X~ = L^-1 X_b, the per-SNP reductions and the p x p solves with standard
errors.  The study set-up (M, Cholesky,
diagonal-block inverses, the X_L / y precompute) is done once before timing,
as in the paper's measurements (Sec. 4).

  value   device-resident throughput: the step's 8 int8 blocks already in
          HBM (328 MB, larger than the 126 MB L2; every block also streams
          the n x n operator), results written to HBM;
  e2e     the same metric through gwas_solve_stream with HOST buffers: each
          step is one call over the 8 blocks eight times over, their int8
          columns host->device from pinned memory and b / se / status back,
          overlapped by the library's block ring; W untimed calls first.

Paths: "fp64" (all-FP64 solve, DFMA), "sliced64" (the FP64 bar from exact
integer products of a sliced M^-1 on the tensor cores) and the split-precision
tensor-core paths.  The headline `value` is the fastest split path when one is
built, else fp64; every path's numbers are in "paths", the two paths held to
the FP64 bar side by side in "fp64_class".

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU: launched by torchrun, one rank per GPU; SNP blocks are sharded
across ranks with no collective on the data path ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GLS solves/sec (SNPs/s) at n=10k,p=4: split-prec vs FP64 path, % roofline"
UNIT = "SNPs/s"
WORKLOAD = "n10k_p4_m1M_int8"
SPLIT_PATHS = ("bf16x3", "tf32x3", "f16x2")
SLICED_SLABS = 4  # the sliced path's 11-bit slices of M^-1's triangle
E2E_REPEATS = 8  # the end-to-end step streams the resident blocks this many times over (64 blocks a call)
STRIP_GROUP = 0  # tile order of the split paths: strips per group (0 = all)
N_RESIDENT_BLOCKS = 8


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--paths", default="auto", help="comma list of fp64,bf16x3,tf32x3,f16x2 (auto: all built)")
    ap.add_argument("--n", type=int, default=None, help="override n (smaller smoke runs only)")
    ap.add_argument("--bs", type=int, default=None, help="override bs (smaller smoke runs only)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the batch / disk / adjoint / REML measurements")
    ap.add_argument("--strip-group", type=int, default=None,
                    help="split paths: column strips per tile-order group (0 = all; default: the measured best)")
    ap.add_argument("--tiles", choices=("auto", "single", "pair_mma", "inverse"), default="auto",
                    help="split paths: tiles on SMs (auto: the measured fastest; single: one 128-row tile per SM; "
                         "pair_mma: row-panel pairs as one 256-row product per 2-SM cluster; inverse: the "
                         "triangular product with L^-1 formed at set-up, row-panel pairs per cluster)")
    ap.add_argument("--no-substitution", action="store_true",
                    help="with --tiles auto: skip the kernel-only measurement of the blocked substitution (pair_mma)")
    ap.add_argument("--separate-sums", action="store_true",
                    help="inverse form: the per-SNP sums as a separate pass over X~ instead of inside the solve")
    ap.add_argument("--fp64-steps", type=int, default=None,
                    help="steps of the fp64 path when a split path is the headline (default 1)")
    ap.add_argument("--paper-scale-m", type=int, default=0,
                    help="also stream this many SNPs disk to disk from a 2-bit packed file of about "
                         "--paper-scale-gb GB, read pass after pass with the page cache dropped before each pass "
                         "(e.g. 190000000, the paper's m); not part of the default run")
    ap.add_argument("--paper-scale-gb", type=float, default=40.0)
    ap.add_argument("--disk-tier-gb", type=float, default=0.0,
                    help="also run the out-of-core forms from files of about this many GB on the local disk "
                         "(written, synced and dropped from the page cache first); not part of the default run")
    return ap.parse_args()


def workload(args):
    import gwas_synth
    w = dict(gwas_synth.WORKLOADS[WORKLOAD])
    if args.n:
        w["n"] = args.n
        w["k"] = max(2, args.n // 2)
    if args.bs:
        w["bs"] = args.bs
    return w


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """SM clock and throttle reasons sampled through NVML (or nvidia-smi)
    while running."""

    REASONS = {
        0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap", 0x8: "hw_slowdown",
        0x10: "sync_boost", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
        0x80: "hw_power_brake_slowdown", 0x100: "display_clock_setting",
    }

    def __init__(self, device_index: int, period_s: float = 0.005):
        self.period = period_s
        self.samples = []
        self.reasons = 0
        self._stop = threading.Event()
        self._thread = None
        self.max_mhz = None
        try:
            import pynvml
            pynvml.nvmlInit()
            self._nvml = pynvml
            self._h = pynvml.nvmlDeviceGetHandleByIndex(device_index)
            self.max_mhz = pynvml.nvmlDeviceGetMaxClockInfo(self._h, pynvml.NVML_CLOCK_SM)
        except Exception as e:  # no NVML binding: sample with nvidia-smi instead
            self._nvml = None
            self.error = repr(e)
        self._device_index = device_index
        self._proc = None

    def _run(self):
        nv = self._nvml
        while not self._stop.is_set():
            try:
                self.samples.append(nv.nvmlDeviceGetClockInfo(self._h, nv.NVML_CLOCK_SM))
                self.reasons |= nv.nvmlDeviceGetCurrentClocksEventReasons(self._h)
            except Exception:
                pass
            time.sleep(self.period)

    def _run_smi(self):
        import subprocess
        cmd = ["nvidia-smi", "-i", str(self._device_index),
               "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.active",
               "--format=csv,noheader,nounits", "-lms", "20"]
        try:
            self._proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception as e:
            self.error = repr(e)
            return
        for line in self._proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            try:
                self.samples.append(float(parts[0]))
                self.max_mhz = float(parts[1])
                self.reasons |= int(parts[2], 16)
            except Exception:
                pass

    def __enter__(self):
        self._thread = threading.Thread(target=self._run if self._nvml else self._run_smi, daemon=True)
        self._thread.start()
        if not self._nvml:
            time.sleep(0.3)  # let nvidia-smi start before the timed region
        return self

    def __exit__(self, *exc):
        self._stop.set()
        if self._proc is not None:
            time.sleep(0.05)
            self._proc.terminate()
        if self._thread:
            self._thread.join(timeout=5)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": [], "samples": 0,
                    "error": getattr(self, "error", "no samples")}
        reasons = [name for bit, name in self.REASONS.items() if self.reasons & bit and bit != 0x1]
        out = {"sm_mhz": float(np.median(self.samples)), "sm_max_mhz": self.max_mhz, "reasons": reasons,
               "samples": len(self.samples), "source": "nvml" if self._nvml else "nvidia-smi"}
        return out


# ------------------------------------------------------------------ peaks
def load_measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def measure_extra_peaks(torch, dev):
    """FP64 and TF32 GEMM rates (cuBLAS through torch) and pinned H2D GB/s,
    which the measured-peaks file does not hold."""
    out = {}

    def best_gemm(dtype, n, reps):
        a = torch.randn(n, n, device=dev, dtype=dtype)
        b = torch.randn(n, n, device=dev, dtype=dtype)
        torch.matmul(a, b)
        torch.cuda.synchronize()
        best = 1e9
        for _ in range(reps):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            torch.matmul(a, b)
            e.record()
            torch.cuda.synchronize()
            best = min(best, s.elapsed_time(e) / 1e3)
        return 2.0 * n ** 3 / best / 1e12

    out["fp64_tflops_cublas"] = best_gemm(torch.float64, 4096, 3)
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    out["tf32_tflops_cublas"] = best_gemm(torch.float32, 8192, 5)
    torch.backends.cuda.matmul.allow_tf32 = prev
    src = torch.empty(1 << 30, dtype=torch.uint8, pin_memory=True)
    dst = torch.empty(1 << 30, dtype=torch.uint8, device=dev)
    dst.copy_(src, non_blocking=True)
    torch.cuda.synchronize()
    best = 1e9
    for _ in range(5):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        dst.copy_(src, non_blocking=True)
        e.record()
        torch.cuda.synchronize()
        best = min(best, s.elapsed_time(e) / 1e3)
    out["h2d_gbs_pinned"] = (1 << 30) / best / 1e9
    del src, dst
    torch.cuda.empty_cache()
    return out


def source_digest(name: str) -> str:
    """sha256[:16] of a kernel source file and of every header of the library's
    CUDA sources (csrc/) it includes, directly or through another header, in
    a fixed order: a traffic record holds for the kernel only while none of
    them changed.  The public C header (declarations and their documentation,
    no device code) is not part of it."""
    csrc = os.path.join(ROOT, "paper_1302_4332_b300", "csrc")
    seen, todo = [], [name]
    while todo:
        f = todo.pop(0)
        path = os.path.join(csrc, f)
        if f in seen or "/" in f or not os.path.exists(path):
            continue
        seen.append(f)
        for line in open(path, encoding="utf-8", errors="replace"):
            t = line.strip()
            if t.startswith("#include \""):
                todo.append(t.split('"')[1])
    h = hashlib.sha256()
    for f in [seen[0]] + sorted(seen[1:]):
        h.update(f.encode() + b"\0" + open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def kernel_traffic(path: str, tiles: str = ""):
    """DRAM bytes per launch of the path's solve kernel (split paths: keyed by
    precision and tile mode) from the committed ncu summary, if that summary
    was taken on the current source (the kernel's file and its headers)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic_per_launch.json")) as f:
            rec = json.load(f).get(f"{path}/{tiles}" if tiles else path)
        if not rec:
            return None
        return rec["dram_bytes"] if source_digest(rec["source"]) == rec["sha256_16"] else None
    except Exception:
        return None


# ------------------------------------------------------------------ sharding
from paper_1302_4332_b300.shard import shard_block_starts  # noqa: E402  (rank r owns blocks r*nb ..)


def max_over_ranks(x: float, dist, device=None) -> float:
    """The slowest rank's time (the job's time); identity without a process group."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, units_per_rank: int, seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / seconds


# ------------------------------------------------------------------ ours
def run_ours(args, rank, world, local_rank, dist):
    import torch
    import gwas_synth
    import paper_1302_4332_b300 as gw
    from paper_1302_4332_b300 import build as gbuild

    gbuild.build()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    w = workload(args)
    n, p, bs = w["n"], w["p"], w["bs"]
    t0 = time.time()
    s = gwas_synth.study(n, p, w["k"], w["h"], w["sigma2"])
    # this rank's blocks: columns [ (rank*NB + i) * bs, ... )
    blocks_h = [gwas_synth.dosages(n, c0, c0 + bs) for c0 in shard_block_starts(rank, world, N_RESIDENT_BLOCKS, bs)]
    gen_s = time.time() - t0
    blocks_d = [torch.from_numpy(np.ascontiguousarray(b.T)).to(dev).T for b in blocks_h]

    peaks = load_measured_peaks()
    extra = measure_extra_peaks(torch, dev) if rank == 0 else {}

    built = list(getattr(gw, "BUILT_PRECISIONS", ("fp64",)))
    paths = built if args.paths == "auto" else [x for x in args.paths.split(",") if x]
    has_split = any(pp in paths for pp in SPLIT_PATHS)
    NB = N_RESIDENT_BLOCKS
    step_snps = NB * bs
    # (entry, precision, tile mode): the paths, then -- when the default tile
    # mode (the inverse form) is the headline -- the blocked substitution
    # (pair product) of each split path, kernel-only, for comparison
    jobs = [(pp, pp, args.tiles if pp != "fp64" else "auto") for pp in paths]
    if args.tiles == "auto" and not args.no_substitution:
        jobs += [(f"{pp}/pair_mma", pp, "pair_mma") for pp in paths if pp in ("bf16x3", "tf32x3")]
    results = {}
    for entry, path, tiles in jobs:
        steps, warm_blocks = args.steps, args.warmup * NB
        if path == "fp64" and has_split:
            # the FP64 path is two orders of magnitude slower: one step, a few warm-up blocks
            steps, warm_blocks = (args.fp64_steps or 1), args.warmup
        t_init = time.time()
        sg = STRIP_GROUP if args.strip_group is None else args.strip_group
        tc_split = path in SPLIT_PATHS  # the tile options apply to the split paths only
        gkw = dict(precision=path, bs=bs, strip_group=sg if tc_split else 0,
                   tiles=(tiles if path != "f16x2" or tiles == "auto" else "inverse") if tc_split else "auto",
                   separate_sums=args.separate_sums and tc_split)
        g = gw.GLS(s["Phi"], s["XL"], s["y"], w["h"], w["sigma2"], **gkw)
        init_s = time.time() - t_init
        b = torch.empty((bs, p), dtype=torch.float64, device=dev).T
        se = torch.empty((bs, p), dtype=torch.float64, device=dev).T
        st = torch.empty(bs, dtype=torch.int32, device=dev)
        for i in range(warm_blocks):
            g.solve_block(blocks_d[i % NB], b, se, st)
        g.synchronize()
        launches0 = g.kernel_launches
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local_rank) as clk:
            ev0.record()
            for i in range(steps * NB):
                g.solve_block(blocks_d[i % NB], b, se, st)
            ev1.record()
            torch.cuda.synchronize()
        g.synchronize()
        elapsed = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, dist, dev)
        if dist:
            dist.barrier()
        launches = g.kernel_launches - launches0
        # per-stage CUDA events (kept out of the timed region: events between
        # the kernels would also stop the solve and sums kernels from starting
        # early as programmatic dependents): one more pass over the blocks
        g.timing(True)
        steps_t = steps if path != "fp64" else 1
        for i in (range(steps_t * NB) if path != "fp64" else (NB - 1,)):  # ends on the block the error report reads
            g.solve_block(blocks_d[i % NB], b, se, st)
        g.synchronize()
        stages = g.timing_read()
        g.timing(False)
        res = dict(snps_per_s=job_rate(world, steps * step_snps, elapsed), ms_per_step=1e3 * elapsed / steps, steps=steps,
                   warmup_blocks=warm_blocks, snps_per_step=step_snps, init_s=init_s, gpu_launches=launches,
                   strip_group=(sg if tc_split else None),
                   solve_shape=dict(zip(("ctas", "cluster", "tiles"), g.solve_shape())),
                   clocks=clk.summary(),
                   stage_ms_per_block={k: v[0] / max(v[1], 1) for k, v in stages.items() if v[1]})
        # the solve kernel's own launches (CUDA events on its stream, recorded by
        # the library around the launch: the trsm stage also holds the pre-pass)
        st_solve = stages.get("solve", (0.0, 0))
        kernel_ms = st_solve[0] / st_solve[1] if st_solve[1] else stages["trsm"][0] / max(stages["trsm"][1], 1)
        alg_tflop = float(n) * n * bs / 1e12  # n^2 flops per SNP column (Sec. 2.2's trsm)
        achieved = alg_tflop / (kernel_ms / 1e3)
        mode = res["solve_shape"]["tiles"]
        if path == "sliced64":
            # five FP16 products of M^-1's triangle (10-bit slices) per algorithmic
            # product; FP16 runs at the BF16 rate
            pk = (peaks.get("bf16_tflops") or 1800.0) / SLICED_SLABS
            roof = dict(bound="tensor", achieved=achieved, peak=pk, unit="TFLOP/s", frac=achieved / pk,
                        traffic=kernel_traffic(path, "sliced"),
                        peak_basis=(f"bf16 dense tensor peak (of measured, burst; FP16 runs at that rate) / "
                                    f"{SLICED_SLABS}: {SLICED_SLABS} exact FP16 products of the sliced triangle of "
                                    "M^-1 per algorithmic product"))
        elif path == "fp64":
            pk = extra.get("fp64_tflops_cublas")
            roof = dict(bound="alu", achieved=achieved, peak=pk, unit="TFLOP/s",
                        frac=achieved / pk if pk else None, traffic=kernel_traffic(path),
                        peak_basis="FP64 dense GEMM rate measured with cuBLAS DGEMM on this GPU (of measured)")
        else:
            bf16 = peaks.get("bf16_tflops") or 1800.0
            # FP16 runs at the BF16 rate on the tensor cores
            base = bf16 if path in ("bf16x3", "f16x2") else (extra.get("tf32_tflops_cublas") or bf16 * 1.1 / 2.25)
            # tensor products per algorithmic product: the substitution multiplies
            # split operators by split X~ (hi*hi + hi*lo + lo*hi); the inverse form
            # multiplies the split L^-1 by the exact dosages (hi*X + lo*X)
            prods = 2 if mode == "inverse" else 3
            pk = base / prods
            roof = dict(bound="tensor", achieved=achieved, peak=pk, unit="TFLOP/s", frac=achieved / pk,
                        traffic=kernel_traffic(path, mode + ("_separate_sums" if args.separate_sums and
                                                             mode == "inverse" else "")),
                        peak_basis=(f"{'tf32' if path == 'tf32x3' else 'bf16'} dense tensor peak (of measured, "
                                    f"burst) / {prods}: {prods} split products per algorithmic product "
                                    f"({mode} tile mode)"))
        roof["kernel_ms"] = kernel_ms
        roof["timed"] = (f"mean CUDA-event duration of the solve kernel's {st_solve[1]} launches in a second timed "
                         f"region of the same {steps_t} steps right after the first, with the library's per-launch "
                         "events recorded on the kernel's stream (the first region has none: events between the "
                         "kernels stop the programmatic dependent launches from starting early)")
        res["roofline"] = roof
        res["trsm_ms_per_launch"] = stages["trsm"][0] / max(stages["trsm"][1], 1)  # with the pre-pass
        res["solve_kernel_ms_per_launch"] = kernel_ms
        # end to end: the 8 blocks, E2E_REPEATS times over, in pinned host memory
        # (one stream call of 32 blocks per step, so that filling and draining
        # the copy/compute pipeline is a small part of a call)
        if not args.no_e2e and "/" not in entry:
            reps = 1 if path == "fp64" else E2E_REPEATS  # FP64: compute-bound, the pipeline ends matter little
            # W whole calls untimed before the timed ones, as for the resident steps: the
            # host-packed stream runs 20-25 % slower in its first two or three calls of a
            # context (5.2, 5.9, 6.5, then 6.7-7.0 M SNPs/s, BF16x3) while int8 runs flat
            warm_calls = 0 if path == "fp64" else args.warmup
            e2e_snps = reps * step_snps
            Xh = torch.empty((e2e_snps, n), dtype=torch.int8, pin_memory=True)
            Xh_np = Xh.numpy()
            for r_ in range(reps):
                for i in range(NB):
                    Xh_np[(r_ * NB + i) * bs:(r_ * NB + i + 1) * bs] = blocks_h[i].T
            bh = torch.empty((e2e_snps, p), dtype=torch.float64, pin_memory=True)
            seh = torch.empty((e2e_snps, p), dtype=torch.float64, pin_memory=True)
            sth = torch.empty(e2e_snps, dtype=torch.int32, pin_memory=True)
            g.solve_stream(Xh_np[:bs].T, bh.numpy()[:bs].T, seh.numpy()[:bs].T, sth.numpy()[:bs])  # warm
            for _ in range(warm_calls):
                g.solve_stream(Xh_np.T, bh.numpy().T, seh.numpy().T, sth.numpy())
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            h0 = g.h2d_bytes
            t1 = time.perf_counter()
            for _ in range(steps):
                g.solve_stream(Xh_np.T, bh.numpy().T, seh.numpy().T, sth.numpy())
            e2e_s = max_over_ranks(time.perf_counter() - t1, dist, dev)
            h2d_step = (g.h2d_bytes - h0) // steps
            host_packed = h2d_step < e2e_snps * n  # the library packed the blocks on the host
            res["e2e"] = dict(value=job_rate(world, steps * e2e_snps, e2e_s), unit=UNIT,
                              h2d_bytes_per_step=h2d_step,
                              d2h_bytes_per_step=e2e_snps * (2 * p * 8 + 4), snps_per_step=e2e_snps,
                              step=f"one gwas_solve_stream call over {reps} x the {NB} resident blocks "
                                   "(int8 dosages in pinned host memory; " +
                                   ("each block packed to 2-bit codes by the library's host threads while "
                                    "earlier blocks solve, and sent as such" if host_packed else
                                    "sent as int8, one contiguous copy per block") + ")",
                              transport="2-bit codes packed on the host" if host_packed else "int8",
                              warmup_calls=warm_calls)
            if host_packed and (path in SPLIT_PATHS or path == "sliced64"):
                # the same call with the int8 transport (stream_pack = 0), for comparison
                with gw.GLS(s["Phi"], s["XL"], s["y"], w["h"], w["sigma2"], stream_pack=0, **gkw) as g8:
                    g8.solve_stream(Xh_np[:bs].T, bh.numpy()[:bs].T, seh.numpy()[:bs].T, sth.numpy()[:bs])
                    for _ in range(warm_calls):
                        g8.solve_stream(Xh_np.T, bh.numpy().T, seh.numpy().T, sth.numpy())
                    torch.cuda.synchronize()
                    h0 = g8.h2d_bytes
                    t1 = time.perf_counter()
                    for _ in range(steps):
                        g8.solve_stream(Xh_np.T, bh.numpy().T, seh.numpy().T, sth.numpy())
                    e8_s = max_over_ranks(time.perf_counter() - t1, dist, dev)
                    res["e2e_int8_transport"] = dict(
                        value=job_rate(world, steps * e2e_snps, e8_s), unit=UNIT,
                        h2d_bytes_per_step=(g8.h2d_bytes - h0) // steps, snps_per_step=e2e_snps,
                        step="the same calls with gwas_config.stream_pack = 0 (int8 over the link)")
            if path in SPLIT_PATHS or path == "sliced64":
                # the same SNPs held 2-bit packed in pinned host memory (hard calls
                # 0..3, four to a byte): the link carries ceil(n/4) bytes per SNP
                nbp = (n + 3) // 4
                Ph = torch.zeros((e2e_snps, (nbp + 15) // 16 * 16), dtype=torch.uint8, pin_memory=True)
                Ph.numpy()[:, :nbp] = gw.pack_dosages2(Xh_np.T).T  # columns 16-byte aligned: one copy a block
                g.solve_stream_packed(Ph.T[:, :bs], bh.numpy()[:bs].T, seh.numpy()[:bs].T, sth.numpy()[:bs])
                for _ in range(warm_calls):
                    g.solve_stream_packed(Ph.T, bh.numpy().T, seh.numpy().T, sth.numpy())
                torch.cuda.synchronize()
                h0 = g.h2d_bytes
                t1 = time.perf_counter()
                for _ in range(steps):
                    g.solve_stream_packed(Ph.T, bh.numpy().T, seh.numpy().T, sth.numpy())
                ep_s = max_over_ranks(time.perf_counter() - t1, dist, dev)
                res["e2e_packed_input"] = dict(
                    value=job_rate(world, steps * e2e_snps, ep_s), unit=UNIT,
                    h2d_bytes_per_step=(g.h2d_bytes - h0) // steps, snps_per_step=e2e_snps,
                    step="one gwas_solve_stream_packed call over the same SNPs held 2-bit packed in pinned "
                         "host memory (unpacked on the GPU)")
                del Ph
            del Xh, bh, seh, sth
        # keep a few results for the error report against the oracle
        res["_sample"] = (b[:, :64].cpu().numpy().copy(), se[:, :64].cpu().numpy().copy(),
                          st[:64].cpu().numpy().copy(), (steps * NB - 1) % NB)
        results[entry] = res
        g.close()
        torch.cuda.empty_cache()

    return dict(w=w, s=s, blocks_h=blocks_h, results=results, peaks=peaks, extra=extra, gen_s=gen_s)


STUDY_SIZES = (2000, 3500, 5000, 7000, 9000, 11000, 13500, 16000)  # the multi-study batching workload
BATCH_BS = 4096  # the most SNP columns of a study in one batched launch (the tuner's range: 512 .. BATCH_BS)


def measure_forms(args, out):
    """The other forms on one GPU (rank 0, N = 1): the multi-study batch (in
    memory and from files), disk streaming (to host memory and disk to disk),
    several phenotypes sharing one study, the adjoint and the REML fit."""
    import tempfile
    import torch
    import gwas_synth
    import paper_1302_4332_b300 as gw
    dev = torch.device("cuda", 0)
    forms = {}
    # --- batching: 8 studies of uneven n, one persistent graph-captured launch, autotuned
    t0 = time.time()
    studies = [gwas_synth.study(n, 4, 2000, 0.6, 1.0, study_id=i) for i, n in enumerate(STUDY_SIZES)]
    # each study's context holds up to BATCH_BS columns a launch; the tuner picks how many (512 .. BATCH_BS)
    gls = [gw.GLS(s["Phi"], s["XL"], s["y"], 0.6, 1.0, precision="bf16x3", bs=BATCH_BS) for s in studies]
    setup_s = time.time() - t0
    with gw.GLSBatch(gls) as B:
        tune = B.autotune_ex(reps=3)
        cols, order, tuned = tune["cols"], tune["order"], tune["snps_per_s"]
        blocks = [torch.from_numpy(np.ascontiguousarray(gwas_synth.dosages(n, 0, cols, study=i).T)).to(dev).T
                  for i, n in enumerate(STUDY_SIZES)]
        kk = 4  # k blocks of every study per graph replay (k batched launches captured together)
        steps = max(kk, args.steps // 2 // kk * kk)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

        def timed(fn, reps):
            fn()  # a switch between the two forms re-captures the graph: untimed
            B.synchronize()
            torch.cuda.synchronize()
            ev0.record()
            for _ in range(reps):
                fn()
            B.synchronize()
            ev1.record()
            torch.cuda.synchronize()
            return ev0.elapsed_time(ev1) / 1e3

        one = lambda: B.solve(blocks)
        k_steps = lambda: B.solve_k([blocks] * kk)
        one()
        B.synchronize()
        l0 = B.kernel_launches
        one()
        B.synchronize()
        per_step = B.kernel_launches - l0  # kernels of one single-step replay
        t_one = [timed(one, steps)]
        t_k = []
        for _ in range(2):  # the two forms in turn, the same number of block-steps each
            t_k.append(timed(k_steps, steps // kk))
            t_one.append(timed(one, steps))
        t = float(np.median(t_one))
        tk = float(np.median(t_k))
        rate = len(STUDY_SIZES) * cols * steps / t
        forms["batch"] = dict(
            workload="8 studies n=" + ",".join(map(str, STUDY_SIZES)) + ", p=4, bf16x3, int8 dosages",
            snps_per_s=rate, ms_per_step=1e3 * t / steps,
            snps_per_step=len(STUDY_SIZES) * cols, autotuned=tune,
            autotune_snps_per_s=tuned, autotune_over_timed=tuned / rate,
            k_block_replay=dict(blocks_per_study_per_replay=kk, snps_per_s=len(STUDY_SIZES) * cols * steps / tk),
            timing="median of 3 timed runs of single-step replays and of 2 of k-step replays, taken in turn "
                   "(the same block-steps each; the re-capture after each switch untimed)",
            gpu_launches=per_step * steps, steps=steps, setup_s=setup_s,
            algorithmic_tflops=sum(float(n) * n for n in STUDY_SIZES) * cols * steps / t / 1e12)
        # roofline of the whole step (casts, the batched solve and every study's sums):
        # n_i^2 flop per SNP of study i at the tuned tile mode's peak
        prods = 2 if tune["tile_mode"] == "inverse" else 3
        pk = (load_measured_peaks().get("bf16_tflops") or 1800.0) / prods
        forms["batch"]["roofline"] = dict(
            bound="tensor", achieved=forms["batch"]["algorithmic_tflops"], peak=pk, unit="TFLOP/s",
            frac=forms["batch"]["algorithmic_tflops"] / pk,
            peak_basis=f"bf16 dense tensor peak (of measured, burst) / {prods}; achieved over whole steps")
        # every study's results of one step against the FP64 GPU path on its first 64 SNPs
        outs = B.solve(blocks)
        worst = {"b_norm": 0.0, "se_rel": 0.0}
        for s_, X, o in zip(studies, blocks, outs):
            with gw.GLS(s_["Phi"], s_["XL"], s_["y"], 0.6, 1.0, precision="fp64", bs=64) as g64:
                b64, se64, st64 = g64.solve_block(X[:, :64])
                g64.synchronize()
            b64, se64 = b64.cpu().numpy(), se64.cpu().numpy()
            bb, ss = o[0][:, :64].cpu().numpy(), o[1][:, :64].cpu().numpy()
            okc = st64.cpu().numpy() == 0
            worst["b_norm"] = max(worst["b_norm"], float(np.max(np.linalg.norm(bb[:, okc] - b64[:, okc], axis=0) /
                                                                  np.linalg.norm(b64[:, okc], axis=0))))
            worst["se_rel"] = max(worst["se_rel"], float(np.max(np.abs(ss[:, okc] - se64[:, okc]) / se64[:, okc])))
        forms["batch"]["error_vs_fp64_path"] = dict(
            worst, sample="first 64 SNPs of every study, one batched step against the FP64 GPU path "
                          "(itself held to 1e-10 of the oracle by the tests)")
        # --- the same batch out of core: each study's dosages in its own file (its block
        # written REPS times), streamed disk -> pinned host (a reader thread per study) -> GPU
        reps_f = 4
        with tempfile.TemporaryDirectory() as td:
            paths = []
            for i, X in enumerate(blocks):
                paths.append(os.path.join(td, f"study{i}.bin"))
                raw = np.ascontiguousarray(X.cpu().numpy().T).tobytes()
                with open(paths[-1], "wb") as f:
                    for _ in range(reps_f):
                        f.write(raw)
            B.solve_files(paths, [cols] * len(paths), cols)  # warm
            t1 = time.perf_counter()
            B.solve_files(paths, [reps_f * cols] * len(paths), cols)
            t = time.perf_counter() - t1
            forms["batch_disk_e2e"] = dict(
                snps_per_s=len(paths) * reps_f * cols / t, snps=len(paths) * reps_f * cols,
                bytes_read=reps_f * cols * sum(STUDY_SIZES), steps=reps_f,
                note="8 files just written: served from the page cache; H2D and D2H inside the timing")
    for g in gls:
        g.close()
    del studies, gls, blocks
    torch.cuda.empty_cache()
    # --- disk -> pinned host -> GPU for the headline path (the 8 resident blocks in one file)
    w, s = out["w"], out["s"]
    n, bs = w["n"], w["bs"]
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "dosages.bin")
        with open(path, "wb") as f:
            for X in out["blocks_h"]:
                f.write(np.ascontiguousarray(X.T).tobytes())
        m = len(out["blocks_h"]) * bs
        with gw.GLS(s["Phi"], s["XL"], s["y"], w["h"], w["sigma2"], precision="bf16x3", bs=bs) as g:
            g.solve_file(path, bs)  # warm
            t1 = time.perf_counter()
            reps = 3
            for _ in range(reps):
                g.solve_file(path, m)
            t = time.perf_counter() - t1
            # disk to disk: the same columns with the results written back (and checkpointed)
            out_path = os.path.join(td, "results.bin")
            t1 = time.perf_counter()
            done = g.solve_file_out(path, m, out_path)
            t_out = time.perf_counter() - t1
        forms["disk_e2e"] = dict(snps_per_s=reps * m / t, snps=m * reps, bytes_read=reps * m * n,
                                 note="file just written: served from the page cache")
        forms["disk_to_disk_e2e"] = dict(snps_per_s=done / t_out, snps=done, bytes_read=done * n,
                                         bytes_written=64 + done * (16 * w["p"] + 8),
                                         note="gwas_solve_file_out: results written to a file with checkpoints "
                                              "every 16 blocks (fdatasync); input from the page cache")
    # --- several phenotypes sharing the study (the headline workload, 5 phenotype columns):
    # one triangular solve per SNP block serves all of them
    t_ph = 5
    rng = np.random.default_rng(11)
    Y = np.asfortranarray(np.column_stack([s["y"]] + [0.5 * s["y"] + rng.standard_normal(n) for _ in range(t_ph - 1)]))
    blocks_d = [torch.from_numpy(np.ascontiguousarray(X.T)).to(dev).T for X in out["blocks_h"]]
    with gw.GLS(s["Phi"], s["XL"], Y, w["h"], w["sigma2"], precision="f16x2", bs=bs) as g:
        b = torch.empty((t_ph, bs, w["p"]), dtype=torch.float64, device=dev).permute(2, 1, 0)
        se = torch.empty((bs, w["p"]), dtype=torch.float64, device=dev).T
        st = torch.empty(bs, dtype=torch.int32, device=dev)
        for X in blocks_d:
            g.solve_block(X, b, se, st)
        g.synchronize()
        reps = max(3, args.steps // 2)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(reps):
            for X in blocks_d:
                g.solve_block(X, b, se, st)
        ev1.record()
        torch.cuda.synchronize()
        t_s = ev0.elapsed_time(ev1) / 1e3
    snps = reps * len(blocks_d) * bs
    forms["phenotypes"] = dict(workload=f"n={n}, p={w['p']}, {t_ph} phenotypes sharing M, f16x2, 4096-SNP blocks",
                               snps_per_s=snps / t_s, snp_phenotype_tests_per_s=snps * t_ph / t_s,
                               ms_per_block=1e3 * t_s / (reps * len(blocks_d)))
    del blocks_d
    # --- the differentiation workload: n = 5,000, p = 4, FP64 adjoint of one 4096-SNP block
    s4 = gwas_synth.study(5000, 4, 5000, 0.5, 1.0, study_id=4)
    X4 = torch.from_numpy(np.ascontiguousarray(gwas_synth.dosages(5000, 0, 4096, study=4).T)).to(dev).T
    with gw.GLS(s4["Phi"], s4["XL"], s4["y"], 0.5, 1.0, bs=4096) as g:
        chi2 = torch.zeros(4096, dtype=torch.float64, device=dev)
        dch = torch.zeros(4096, dtype=torch.float64, device=dev)
        dh = torch.zeros(1, dtype=torch.float64, device=dev)
        dy = torch.zeros(5000, dtype=torch.float64, device=dev)
        g.adjoint_block(X4, dh, dy, chi2, dch)
        g.synchronize()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for _ in range(2):
            g.adjoint_block(X4, dh, dy, chi2, dch)
        g.synchronize()
        t = (time.perf_counter() - t1) / 2
    forms["adjoint_fp64"] = dict(workload="n=5000, p=4, 4096 SNPs per block", snps_per_s=4096 / t,
                                 ms_per_block=1e3 * t)
    # the split adjoint: block solve and transpose solve on the tensor cores
    with gw.GLS(s4["Phi"], s4["XL"], s4["y"], 0.5, 1.0, bs=4096, precision="bf16x3") as g:
        g.adjoint_block(X4, dh, dy, chi2, dch)
        g.synchronize()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for _ in range(5):
            g.adjoint_block(X4, dh, dy, chi2, dch)
        g.synchronize()
        t = (time.perf_counter() - t1) / 5
    forms["adjoint_bf16x3"] = dict(workload="n=5000, p=4, 4096 SNPs per block", snps_per_s=4096 / t,
                                   ms_per_block=1e3 * t)
    # the differentiation workload at its full size: d(sum chi2)/dh and d/dy over all m = 100,000
    # SNPs (25 blocks, the last one ragged), split and FP64, the split result against the FP64 one
    m4 = 100_000
    blocks4 = [torch.from_numpy(np.ascontiguousarray(
        gwas_synth.dosages(5000, c0, min(c0 + 4096, m4), study=4).T)).to(dev).T for c0 in range(0, m4, 4096)]

    def full_adjoint(precision):
        with gw.GLS(s4["Phi"], s4["XL"], s4["y"], 0.5, 1.0, bs=4096, precision=precision) as g:
            dh_w = torch.zeros(1, dtype=torch.float64, device=dev)
            dy_w = torch.zeros(5000, dtype=torch.float64, device=dev)
            g.adjoint_block(blocks4[0], dh_w, dy_w, chi2, dch)  # set-up and warm-up
            g.synchronize()
            dh_f = torch.zeros(1, dtype=torch.float64, device=dev)
            dy_f = torch.zeros(5000, dtype=torch.float64, device=dev)
            c2 = [torch.empty(X.shape[1], dtype=torch.float64, device=dev) for X in blocks4]
            dc = [torch.empty(X.shape[1], dtype=torch.float64, device=dev) for X in blocks4]
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            for X, a, d_ in zip(blocks4, c2, dc):
                g.adjoint_block(X, dh_f, dy_f, a, d_)
            g.synchronize()
            return (time.perf_counter() - t1, float(dh_f[0]), dy_f.cpu().numpy(), torch.cat(c2).cpu().numpy(),
                    torch.cat(dc).cpu().numpy())

    ts, dhs, dys, c2s, dcs = full_adjoint("bf16x3")
    t64, dh64, dy64, c264, dc64 = full_adjoint("fp64")
    ok = np.isfinite(c264) & np.isfinite(c2s)
    forms["adjoint_full_m100k"] = dict(
        workload="n=5000, p=4, m=100,000 SNPs (25 blocks of 4096), loss = sum of the Wald chi2",
        bf16x3_seconds=ts, bf16x3_snps_per_s=m4 / ts, fp64_seconds=t64, fp64_snps_per_s=m4 / t64,
        dloss_dh=dhs, dloss_dh_fp64=dh64,
        rel_err_vs_fp64={"dloss_dh": abs(dhs - dh64) / abs(dh64),
                         "dloss_dy_norm": float(np.linalg.norm(dys - dy64) / np.linalg.norm(dy64)),
                         "chi2_max": float(np.max(np.abs(c2s[ok] - c264[ok]) / np.abs(c264[ok]))),
                         "dchi2_dh_norm": float(np.linalg.norm(dcs[ok] - dc64[ok]) / np.linalg.norm(dc64[ok]))})
    del blocks4
    t1 = time.perf_counter()
    h_hat, ll, evals = gw.reml_fit(s4["Phi"], s4["XL"][:, :3], s4["y"], h0=0.2, tol=1e-8)
    forms["reml_fit"] = dict(workload="null model n=5000, q=3, true h=0.5, from h0=0.2", h_hat=h_hat,
                             loglik=ll, likelihood_evaluations=evals, seconds=time.perf_counter() - t1)
    return forms


def _drop_cached(path):
    """Flushes a file to the device and drops its pages from the page cache,
    so that the next reads come from the disk (the reads themselves still go
    through the page cache: no O_DIRECT)."""
    fd = os.open(path, os.O_RDONLY)
    try:
        os.fsync(fd)
        os.posix_fadvise(fd, 0, 0, os.POSIX_FADV_DONTNEED)
    finally:
        os.close(fd)


def _write_repeated(path, raw, reps):
    with open(path, "wb") as f:
        for _ in range(reps):
            f.write(raw)
        f.flush()
        os.fdatasync(f.fileno())


def measure_disk_tier(args, out):
    """The out-of-core forms at the scale the local disk holds (Sec. 3.1's
    disk -> main memory -> GPU, results written back): one study's dosage file
    of about --disk-tier-gb GB (the 8 resident blocks repeated), solved disk to
    disk with checkpoints; then the 8-study batching workload from 8 files of
    that total size (each study's first block repeated).  Files are written,
    synced and dropped from the page cache before each timed read."""
    import shutil
    import tempfile
    import torch
    import gwas_synth
    import paper_1302_4332_b300 as gw
    w, s = out["w"], out["s"]
    n, bs, p = w["n"], w["bs"], w["p"]
    res = {}
    root = tempfile.mkdtemp(prefix="gwas_disk_", dir=os.environ.get("TMPDIR", "/tmp"))
    try:
        free = shutil.disk_usage(root).free
        target = min(args.disk_tier_gb * 1e9, 0.8 * free)
        raw = b"".join(np.ascontiguousarray(X.T).tobytes() for X in out["blocks_h"])  # 8 blocks, column-major
        reps = max(1, int(target // len(raw)))
        m = reps * len(out["blocks_h"]) * bs
        path = os.path.join(root, "dosages.bin")
        t0 = time.perf_counter()
        _write_repeated(path, raw, reps)
        write_s = time.perf_counter() - t0
        _drop_cached(path)
        rpath = os.path.join(root, "results.bin")
        head_path = "f16x2" if "f16x2" in gw.BUILT_PRECISIONS else "fp64"
        with gw.GLS(s["Phi"], s["XL"], s["y"], w["h"], w["sigma2"], precision=head_path, bs=bs) as g:
            t1 = time.perf_counter()
            done = g.solve_file_out(path, m, rpath)
            t_run = time.perf_counter() - t1
            # check: the file's first and last block against the in-memory solve of the same columns
            head, b_all, se_all, st_all = gw.read_results(rpath)
            nb = m // bs
            checks = []
            for blk in (0, nb - 1):
                b_ref, se_ref, st_ref = g.solve_block(out["blocks_h"][blk % len(out["blocks_h"])])
                sl = slice(blk * bs, (blk + 1) * bs)
                checks.append(bool(np.array_equal(b_all[:, sl], b_ref) and np.array_equal(se_all[:, sl], se_ref)
                                   and np.array_equal(st_all[sl], st_ref)))
        res["one_study_disk_to_disk"] = dict(
            workload=f"n={n}, p={p}, {head_path}, m={m} SNPs ({m * n / 1e9:.1f} GB int8 file, the 8 resident "
                     f"blocks repeated {reps} times)", snps=done, seconds=t_run, snps_per_s=done / t_run,
            read_gbs=done * n / t_run / 1e9, results_gb=(64 + done * (16 * p + 8)) / 1e9,
            file_write_gbs=m * n / write_s / 1e9,
            page_cache="dropped before the run (fsync + POSIX_FADV_DONTNEED); reads through the page cache, "
                       "not O_DIRECT",
            matches_in_memory_solve=all(checks))
        os.remove(path)
        # the same SNPs from a 2-bit packed file (a quarter of the bytes from disk and over the link)
        nbp = (n + 3) // 4
        rawp = b"".join(np.ascontiguousarray(gw.pack_dosages2(X).T).tobytes() for X in out["blocks_h"])
        ppath = os.path.join(root, "dosages.2bit")
        t0 = time.perf_counter()
        _write_repeated(ppath, rawp, reps)
        writep_s = time.perf_counter() - t0
        _drop_cached(ppath)
        rppath = os.path.join(root, "results_packed.bin")
        with gw.GLS(s["Phi"], s["XL"], s["y"], w["h"], w["sigma2"], precision=head_path, bs=bs) as g:
            t1 = time.perf_counter()
            donep = g.solve_file_out(ppath, m, rppath, packed=True)
            tp_run = time.perf_counter() - t1
        _, bp_all, sep_all, stp_all = gw.read_results(rppath)
        same = bool(np.array_equal(bp_all, b_all) and np.array_equal(sep_all, se_all) and np.array_equal(stp_all, st_all))
        res["one_study_disk_to_disk_packed"] = dict(
            workload=f"the same m={m} SNPs from a 2-bit packed file ({m * nbp / 1e9:.1f} GB)", snps=donep,
            seconds=tp_run, snps_per_s=donep / tp_run, read_gbs=donep * nbp / tp_run / 1e9,
            file_write_gbs=m * nbp / writep_s / 1e9, results_equal_int8_file_run=same,
            page_cache="dropped before the run (fsync + POSIX_FADV_DONTNEED)")
        del b_all, se_all, st_all, bp_all, sep_all, stp_all
        os.remove(ppath)
        for q in (rpath, rppath):
            os.remove(q)
            if os.path.exists(q + ".ckpt"):
                os.remove(q + ".ckpt")
        # the batching workload, 8 studies of uneven n, from files of the same total size
        studies = [gwas_synth.study(ni, 4, 2000, 0.6, 1.0, study_id=i) for i, ni in enumerate(STUDY_SIZES)]
        gls = [gw.GLS(st_["Phi"], st_["XL"], st_["y"], 0.6, 1.0, precision="bf16x3", bs=4096) for st_ in studies]
        cols = 4096
        per = int(target // sum(STUDY_SIZES) // cols) * cols  # SNPs per study
        paths = []
        t0 = time.perf_counter()
        for i, ni in enumerate(STUDY_SIZES):
            blk = np.ascontiguousarray(gwas_synth.dosages(ni, 0, cols, study=i).T).tobytes()
            paths.append(os.path.join(root, f"study{i}.bin"))
            _write_repeated(paths[-1], blk, per // cols)
        write_s = time.perf_counter() - t0
        for pth in paths:
            _drop_cached(pth)
        with gw.GLSBatch(gls) as B:
            t1 = time.perf_counter()
            outs = B.solve_files(paths, [per] * len(paths), cols)
            t_run = time.perf_counter() - t1
        res["batch_8_studies_from_disk"] = dict(
            workload="8 studies n=" + ",".join(map(str, STUDY_SIZES)) + f", p=4, bf16x3, {per} SNPs per study "
                     f"({per / 2e6:.2f} of the 2,000,000 the batching workload names; "
                     f"{per * sum(STUDY_SIZES) / 1e9:.1f} GB of int8 files on the local disk)",
            snps=per * len(paths), seconds=t_run, snps_per_s=per * len(paths) / t_run,
            read_gbs=per * sum(STUDY_SIZES) / t_run / 1e9, file_write_gbs=per * sum(STUDY_SIZES) / write_s / 1e9,
            page_cache="dropped before the run (fsync + POSIX_FADV_DONTNEED); reads through the page cache",
            all_finite=bool(all(np.isfinite(o[0][:, o[2] == 0]).all() for o in outs)))
        for pth in paths:
            os.remove(pth)
        # the batching workload at its full 2,000,000 SNPs per study, from 2-bit packed files
        # (a quarter of the int8 bytes: ~33.5 GB where int8 files need 134 GB)
        nbp_all = sum((ni + 3) // 4 for ni in STUDY_SIZES)
        per_p = min(2_000_000, int(0.8 * shutil.disk_usage(root).free // nbp_all // cols) * cols)
        nblk_p = -(-per_p // cols)
        ppaths = []
        t0 = time.perf_counter()
        for i, ni in enumerate(STUDY_SIZES):
            blk = gw.pack_dosages2(gwas_synth.dosages(ni, 0, cols, study=i))
            ppaths.append(os.path.join(root, f"study{i}.2bit"))
            _write_repeated(ppaths[-1], np.ascontiguousarray(blk.T).tobytes(), nblk_p)
        writep_s = time.perf_counter() - t0
        for pth in ppaths:
            _drop_cached(pth)
        with gw.GLSBatch(gls) as B:
            t1 = time.perf_counter()
            outs_p = B.solve_files(ppaths, [per_p] * len(ppaths), cols, packed=True)
            tp_run = time.perf_counter() - t1
        k = min(per, per_p)  # the columns both runs solved (the same repeated block)
        same = all(np.array_equal(a[0][:, :k], q[0][:, :k]) and np.array_equal(a[1][:, :k], q[1][:, :k])
                   and np.array_equal(a[2][:k], q[2][:k]) for a, q in zip(outs, outs_p))
        res["batch_8_studies_from_disk_packed"] = dict(
            workload="8 studies n=" + ",".join(map(str, STUDY_SIZES)) + f", p=4, bf16x3, {per_p} SNPs per study "
                     f"({per_p / 2e6:.2f} of the 2,000,000 the batching workload names; "
                     f"{per_p * nbp_all / 1e9:.1f} GB of 2-bit packed files on the local disk)",
            snps=per_p * len(ppaths), seconds=tp_run, snps_per_s=per_p * len(ppaths) / tp_run,
            read_gbs=per_p * nbp_all / tp_run / 1e9, file_write_gbs=per_p * nbp_all / writep_s / 1e9,
            page_cache="dropped before the run (fsync + POSIX_FADV_DONTNEED); reads through the page cache",
            results_equal_int8_files_on_common_columns=bool(same),
            all_finite=bool(all(np.isfinite(o[0][:, o[2] == 0]).all() for o in outs_p)))
        del outs, outs_p
        for g in gls:
            g.close()
    finally:
        shutil.rmtree(root, ignore_errors=True)
    torch.cuda.empty_cache()
    return res


def measure_paper_scale(args, out):
    """Sustained disk-to-disk streaming at the paper's scale in SNPs (Sec. 1.4,
    m ~ 1.9e8 at n = 10^4): a 2-bit packed dosage file (the 8 resident blocks
    repeated) is solved disk to disk with checkpoints
    pass after pass (the page cache dropped before each pass) until
    --paper-scale-m SNPs are done; one study context throughout (file size:
    --paper-scale-gb)."""
    import shutil
    import tempfile
    import paper_1302_4332_b300 as gw
    w, s = out["w"], out["s"]
    n, bs, p = w["n"], w["bs"], w["p"]
    nbp = (n + 3) // 4
    root = tempfile.mkdtemp(prefix="gwas_paper_", dir=os.environ.get("TMPDIR", "/tmp"))
    res = {}
    try:
        free = shutil.disk_usage(root).free
        rawp = b"".join(np.ascontiguousarray(gw.pack_dosages2(X).T).tobytes() for X in out["blocks_h"])
        results_per_snp = 16 * p + 8
        target = min(args.paper_scale_gb * 1e9, 0.7 * free - 4e9)
        reps = max(1, int(target // (len(rawp) + len(out["blocks_h"]) * bs * results_per_snp)))
        m_file = reps * len(out["blocks_h"]) * bs
        ppath = os.path.join(root, "dosages.2bit")
        _write_repeated(ppath, rawp, reps)
        head_path = "f16x2" if "f16x2" in gw.BUILT_PRECISIONS else "fp64"
        rates, total, t_all = [], 0, 0.0
        ok = True
        with gw.GLS(s["Phi"], s["XL"], s["y"], w["h"], w["sigma2"], precision=head_path, bs=bs) as g:
            refs = [g.solve_block(X) for X in (out["blocks_h"][0], out["blocks_h"][-1])]
            while total < args.paper_scale_m:
                m = min(m_file, args.paper_scale_m - total)
                _drop_cached(ppath)
                rpath = os.path.join(root, "results.bin")
                t1 = time.perf_counter()
                done = g.solve_file_out(ppath, m, rpath, packed=True)
                dt = time.perf_counter() - t1
                t_all += dt
                total += done
                rates.append(done / dt)
                if done != m:
                    ok = False
                    break
                # the pass's first block and (for a whole pass) its last against the in-memory solve
                _, b_all, se_all, st_all = gw.read_results(rpath)
                for (b_ref, se_ref, st_ref), blk in zip(refs, (0, m // bs - 1)):
                    if (blk + 1) * bs > m or (blk != 0 and blk % len(out["blocks_h"]) != len(out["blocks_h"]) - 1):
                        continue
                    sl = slice(blk * bs, (blk + 1) * bs)
                    ok &= bool(np.array_equal(b_all[:, sl], b_ref) and np.array_equal(se_all[:, sl], se_ref)
                               and np.array_equal(st_all[sl], st_ref))
                del b_all, se_all, st_all
                os.remove(rpath)
                if os.path.exists(rpath + ".ckpt"):
                    os.remove(rpath + ".ckpt")
        res = dict(workload=f"n={n}, p={p}, {head_path}, {total} SNPs disk to disk from a {m_file * nbp / 1e9:.1f} GB "
                            f"2-bit packed file ({m_file} SNPs, the 8 resident blocks repeated) read {len(rates)} "
                            "times, results and checkpoints written every pass",
                   snps=total, seconds=t_all, snps_per_s=total / t_all, passes=len(rates),
                   pass_snps_per_s_min=min(rates), pass_snps_per_s_max=max(rates),
                   read_gbs=total * nbp / t_all / 1e9, results_gb=total * results_per_snp / 1e9,
                   page_cache="dropped before every pass (fsync + POSIX_FADV_DONTNEED); reads through the page "
                              "cache, not O_DIRECT",
                   blocks_match_in_memory_solve=ok)
    finally:
        shutil.rmtree(root, ignore_errors=True)
    return res


def cpu_baseline(w, s, X_sample, target_s=12.0):
    """The oracle as it stands on the host cores: Cholesky first (not timed,
    as the paper leaves set-up out), then per-SNP GLS on a bounded sample."""
    import oracle
    t0 = time.time()
    L = oracle.potrf(oracle.form_m(s["Phi"], w["h"], w["sigma2"]))
    chol_s = time.time() - t0
    # calibrate on one group of 16 SNPs per thread (the oracle's unit of parallel
    # work), then time a whole number of such rounds lasting about target_s
    cores = oracle.num_threads()
    grp = 16 * cores
    t1 = time.time()
    oracle.gls(L, s["XL"], s["y"], X_sample[:, :grp])
    rate = grp / max(time.time() - t1, 1e-9)
    m = int(min(X_sample.shape[1], max(grp, rate * target_s)))
    m -= m % grp if m > grp else 0
    t2 = time.time()
    r, se, _, st = oracle.gls(L, s["XL"], s["y"], X_sample[:, :m])
    dt = time.time() - t2
    # the same oracle on one core, on the first 16 SNPs of the sample
    oracle.set_num_threads(1)
    try:
        t3 = time.time()
        oracle.gls(L, s["XL"], s["y"], X_sample[:, :16])
        one_core = 16 / max(time.time() - t3, 1e-9)
    finally:
        oracle.set_num_threads(cores)
    return dict(value=m / dt, unit=UNIT, cores=cores, kind="oracle", value_1core=one_core, nproc=os.cpu_count(),
                sample=f"first {m} SNPs of one bs block at n={w['n']}, p={w['p']} ({cores} threads; 1 thread: "
                       f"first 16); Cholesky ({chol_s:.1f} s) excluded"), \
        (L, r, se, st)


def error_report(res_path, oracle_out, blocks_h, s, w):
    """Max / median error of b and se against the FP64 oracle on 64 SNPs."""
    import oracle
    from oracle.metrics import compare
    b, se, st, blk = res_path["_sample"]
    L = oracle_out[0]
    r, se_o, _, st_o = oracle.gls(L, s["XL"], s["y"], blocks_h[blk][:, :64])
    return compare(b, se, st, r, se_o, st_o)


def storage_precision_study(oracle_out, blocks_h, s, w, errors):
    """Whether single precision is enough to store the operator: b and se of
    the sampled SNPs against the FP64 oracle with L^-1 held as its split pair
    (the split paths as measured) and as its hi piece alone (one BF16, TF32
    or row-scaled FP16 rounding: `single_piece`), next to the FP64 path."""
    import paper_1302_4332_b300 as gw
    import oracle
    from oracle.metrics import compare
    X = np.asfortranarray(blocks_h[0][:, :64])
    r, se_o, _, st_o = oracle.gls(oracle_out[0], s["XL"], s["y"], X)
    study = {"sample": "first 64 SNPs of block 0, n=%d, p=%d" % (w["n"], w["p"]),
             "fp64": errors.get("fp64")}
    for path in ("bf16x3", "tf32x3", "f16x2"):
        if path not in gw.BUILT_PRECISIONS:
            continue
        with gw.GLS(s["Phi"], s["XL"], s["y"], w["h"], w["sigma2"], precision=path, bs=64,
                    single_piece=True) as g:
            b, se, st = g.solve_block(X)
        study[path] = {"split_pair": errors.get(path), "single_piece": compare(b, se, st, r, se_o, st_o)}
    return study


def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return 0
        return run_reference(args, world)

    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
        dist = tdist
    out = run_ours(args, rank, world, local_rank, dist)
    w, results = out["w"], out["results"]
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    forms = None
    if world == 1 and not args.no_forms:
        try:
            forms = measure_forms(args, out)
        except Exception as e:  # report, do not hide
            forms = {"error": repr(e)}
    if world == 1 and args.disk_tier_gb > 0:
        try:
            forms = dict(forms or {})
            forms["disk_tier"] = measure_disk_tier(args, out)
        except Exception as e:  # report, do not hide
            forms["disk_tier"] = {"error": repr(e)}
    if world == 1 and args.paper_scale_m > 0:
        try:
            forms = dict(forms or {})
            forms["paper_scale"] = measure_paper_scale(args, out)
        except Exception as e:  # report, do not hide
            forms["paper_scale"] = {"error": repr(e)}
    cpu = None
    oracle_out = None
    if world == 1 and not args.no_cpu_baseline:
        cpu, oracle_out = cpu_baseline(w, out["s"], out["blocks_h"][0])
    errors = {}
    if oracle_out is not None:
        for path, res in results.items():
            try:
                errors[path] = error_report(res, oracle_out, out["blocks_h"], out["s"], w)
            except Exception as e:  # report, do not hide
                errors[path] = {"error": repr(e)}
    storage = None
    if oracle_out is not None:
        try:
            storage = storage_precision_study(oracle_out, out["blocks_h"], out["s"], w, errors)
        except Exception as e:  # report, do not hide
            storage = {"error": repr(e)}

    split = [pp for pp in SPLIT_PATHS if pp in results]
    # the headline: the fastest split path; else the FP64 path; else whatever ran
    head = max(split, key=lambda pp: results[pp]["snps_per_s"]) if split else ("fp64" if "fp64" in results
                                                                             else next(iter(results)))
    hr = results[head]
    paths_out = {}
    for path, res in results.items():
        r = {k: v for k, v in res.items() if not k.startswith("_")}
        if path in errors:
            r["error_vs_oracle"] = errors[path]
        paths_out[path] = r
    # the path's roofline: the slower of the solve's flops at the path's peak
    # (n^2 algorithmic flop per SNP) and the SNP's n int8 bytes over the
    # measured pinned host->device link (beside it: the link term of 2-bit
    # packed input, ceil(n/4) bytes per SNP)
    n_ = float(w["n"])
    trsm_bound = hr["roofline"]["peak"] * 1e12 / (n_ * n_) if hr["roofline"].get("peak") else None
    h2d = out["extra"].get("h2d_gbs_pinned")
    h2d_bound = h2d * 1e9 / n_ if h2d else None
    terms = [t for t in (trsm_bound, h2d_bound) if t]
    slower = min(terms) if terms else None
    path_roofline = {"trsm_snps_per_s": trsm_bound, "h2d_snps_per_s": h2d_bound,
                     "bound": None if slower is None else ("trsm" if slower == trsm_bound else "h2d"),
                     "frac": hr["snps_per_s"] / (slower * world) if slower else None,
                     "e2e_frac": (hr["e2e"]["value"] / (slower * world)) if slower and hr.get("e2e") else None,
                     "basis": "per GPU: n^2 flop/SNP at the roofline peak; n B/SNP over the measured pinned H2D link"}
    if h2d and trsm_bound and hr.get("e2e", {}).get("transport", "int8") != "int8":
        # the e2e call sent 2-bit codes packed on the host: its link term is ceil(n/4) B/SNP
        link_p = h2d * 1e9 / ((n_ + 3) // 4)
        e2e_bound = min(trsm_bound, link_p)
        path_roofline["e2e_frac"] = hr["e2e"]["value"] / (e2e_bound * world)
        path_roofline["e2e_bound"] = "trsm" if e2e_bound == trsm_bound else "h2d (2-bit codes)"
        path_roofline["e2e_basis"] = ("the e2e call's blocks crossed the link as 2-bit codes packed on the host: "
                                      "the slower of the solve term and ceil(n/4) B/SNP over the link")
    if h2d and hr.get("e2e_packed_input") and trsm_bound:
        packed_bound = min(trsm_bound, h2d * 1e9 / ((n_ + 3) // 4))
        path_roofline["packed_input"] = {
            "h2d_snps_per_s": h2d * 1e9 / ((n_ + 3) // 4),
            "bound": "trsm" if packed_bound == trsm_bound else "h2d",
            "e2e_frac": hr["e2e_packed_input"]["value"] / (packed_bound * world)}
    # the FP64 bar two ways: the FP64 ALU path and the sliced tensor-core path
    fp64_class = None
    if "fp64" in results and "sliced64" in results:
        f, sl = results["fp64"], results["sliced64"]
        fp64_class = {"fp64_snps_per_s": f["snps_per_s"], "sliced64_snps_per_s": sl["snps_per_s"],
                      "sliced64_over_fp64": sl["snps_per_s"] / f["snps_per_s"],
                      "sliced64_e2e": sl.get("e2e"), "sliced64_roofline": sl["roofline"],
                      "error_vs_oracle": {"fp64": errors.get("fp64"), "sliced64": errors.get("sliced64")}}
    line = {
        "metric": METRIC, "value": hr["snps_per_s"], "unit": UNIT, "n_gpus": world, "steps": hr["steps"],
        "warmup": args.warmup, "ms_per_step": hr["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp64": "f64", "bf16x3": "bf16x3", "tf32x3": "tf32x3", "f16x2": "f16x2",
                                                                   "sliced64": "f16"}[head],
        "data": "synthetic (seeded kinship, covariates, phenotype and int8 dosages shaped like the paper's n=1e4, p=4 workload)",
        "config": {"workload": WORKLOAD, "n": w["n"], "p": w["p"], "bs": w["bs"],
                   "snps_per_step": N_RESIDENT_BLOCKS * w["bs"],
                   "headline_path": head, "parallelism": f"snp-shard x{world}",
                   "l2": "inputs larger than L2: 8 resident int8 blocks (328 MB) per step plus the n x n operator (split L^-1 or block operator, 204 MB) streamed every block"},
        "roofline": hr["roofline"], "path_roofline": path_roofline, "e2e": hr.get("e2e"),
        "gpu_launches": hr["gpu_launches"],
        "clocks": hr["clocks"], "cpu_baseline": cpu, "fp64_class": fp64_class, "paths": paths_out, "forms": forms,
        "storage_precision": storage,
        "peaks": {"measured_file": {k: out["peaks"].get(k) for k in ("hbm_gbs", "bf16_tflops", "bf16_tflops_sustained")},
                  "measured_here": out["extra"]},
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_reference(args, world):
    """The oracle arm: the FP64 CPU oracle as it stands, on the host cores."""
    import gwas_synth
    import oracle
    w = workload(args)
    n, p, bs = w["n"], w["p"], w["bs"]
    s = gwas_synth.study(n, p, w["k"], w["h"], w["sigma2"])
    # the oracle parallelises over groups of 16 SNPs (one L stream per group): eight rounds of one
    # group per thread a step -- each call also solves X~_L and y~ (~0.34 s at n = 1e4, one
    # thread), so a single round per call measured ~40 % below the steady rate, eight ~9 %
    threads = oracle.num_threads()
    per_step = 16 * threads * (8 if n >= 5000 else 64)
    X = gwas_synth.dosages(n, 0, per_step * (args.warmup + args.steps))
    L = oracle.potrf(oracle.form_m(s["Phi"], w["h"], w["sigma2"]))
    for i in range(args.warmup):
        oracle.gls(L, s["XL"], s["y"], X[:, i * per_step:(i + 1) * per_step])
    t0 = time.time()
    for i in range(args.warmup, args.warmup + args.steps):
        oracle.gls(L, s["XL"], s["y"], X[:, i * per_step:(i + 1) * per_step])
    dt = time.time() - t0
    v = args.steps * per_step / dt
    sample = (f"{per_step} SNPs per step = {per_step // 16} groups of 16 on {threads} threads, at n={n}, p={p} "
              f"(one bs={bs} block would take {bs / v:.0f} s); Cholesky excluded")
    line = {
        "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": WORKLOAD, "n": n, "p": p, "bs": bs, "snps_per_step": per_step,
                   "headline_path": "oracle-fp64-cpu", "parallelism": "host cores"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
                         "snp_groups_per_step": per_step // 16},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
