"""A small, self-contained case for kernel profilers (ncu): one study and a
few SNP blocks on the device, solved a few times -- only the buffers the
profiled kernels need, so that a capture with many replay passes stays small.

    python -m paper_1302_4332_b300.profile_case --path bf16x3 --tiles pair_mma --blocks 3
    python -m paper_1302_4332_b300.profile_case --path f16x2 --adjoint --n 5000

Prints one line with the per-call time (CUDA events) of the last repetition;
the profiler's numbers come from its own capture, not from this line.
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--path", default="f16x2", choices=("fp64", "bf16x3", "tf32x3", "f16x2", "sliced64"))
    ap.add_argument("--tiles", default="auto", choices=("auto", "single", "pair_mma", "inverse"))
    ap.add_argument("--n", type=int, default=10000)
    ap.add_argument("--bs", type=int, default=4096)
    ap.add_argument("--blocks", type=int, default=3, help="solve calls (each a full block)")
    ap.add_argument("--adjoint", action="store_true", help="profile the adjoint block instead of the solve")
    ap.add_argument("--separate-sums", action="store_true")
    a = ap.parse_args(argv)

    import torch

    import gwas_synth
    import paper_1302_4332_b300 as gw

    torch.cuda.set_device(0)
    s = gwas_synth.study(a.n, 4, max(2, a.n // 2), 0.5, 1.0)
    X = torch.from_numpy(np.ascontiguousarray(gwas_synth.dosages(a.n, 0, a.bs).T)).cuda().T
    with gw.GLS(s["Phi"], s["XL"], s["y"], 0.5, 1.0, precision=a.path, bs=a.bs, tiles=a.tiles,
                separate_sums=a.separate_sums) as g:
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if a.adjoint:
            dh = torch.zeros(1, dtype=torch.float64, device="cuda")
            dy = torch.zeros(a.n, dtype=torch.float64, device="cuda")
            chi2 = torch.empty(a.bs, dtype=torch.float64, device="cuda")
            dch = torch.empty(a.bs, dtype=torch.float64, device="cuda")
            call = lambda: g.adjoint_block(X, dh, dy, chi2, dch)
        else:
            b = torch.empty((a.bs, 4), dtype=torch.float64, device="cuda").T
            se = torch.empty((a.bs, 4), dtype=torch.float64, device="cuda").T
            st = torch.empty(a.bs, dtype=torch.int32, device="cuda")
            call = lambda: g.solve_block(X, b, se, st)
        for i in range(a.blocks):
            if i == a.blocks - 1:
                ev0.record()
            call()
        ev1.record()
        g.synchronize()
        torch.cuda.synchronize()
        print(f"{a.path} {a.tiles} n={a.n} bs={a.bs} {'adjoint' if a.adjoint else 'solve'}: "
              f"{ev0.elapsed_time(ev1):.3f} ms per call")


if __name__ == "__main__":
    main()
