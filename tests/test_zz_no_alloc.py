"""gwas_solve_block_static: the block solve for callers that cannot allocate
device memory when they solve (their device memory is held by another
allocator, or they must not call cudaMalloc while serving).  Its scratch is a
fixed array inside the library whose address gwas_init looks up.

Each test calls the entry point through the C ABI and checks it against the
entry points that use the context's own scratch: gwas_solve_block on an FP64
context, gwas_solve_block_f64 on a split-precision one (the static call always
runs the FP64 solve), on two calls in a row -- the second reuses the array the
first left behind.  This file is named so that pytest collects it last: if it
fails, a run that stops at the first failure has already run every other test.
Its tests do not depend on that order; each passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import gwas_synth
import paper_1302_4332_b300 as gw

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
LIMIT = 32 * 1024 * 1024  # GWAS_STATIC_SCRATCH_BYTES


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _rel(a, b):
    return float(np.max(np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)))


def _need(n_pad, ncols):
    """Scratch bytes of one call, as the header states them."""
    flags = 4 * (n_pad // 128) * ((ncols + 63) // 64)
    return (128 + flags + 255) // 256 * 256 + 8 * n_pad * ncols


def _max_cols(n_pad):
    c = LIMIT // (8 * n_pad)
    while _need(n_pad, c) > LIMIT:
        c -= 1
    return c


def _static(lib, g, Xd, m, guard=0):
    """Calls the entry point with device outputs surrounded by `guard` sentinel elements."""
    torch = _torch()
    p = g.p
    bb = torch.full((p * (m + 2 * guard),), 7.25, dtype=torch.float64, device="cuda")
    sb = torch.full((p * (m + 2 * guard),), 7.25, dtype=torch.float64, device="cuda")
    tb = torch.full((m + 2 * guard,), -9, dtype=torch.int32, device="cuda")
    b, se, st = bb[p * guard:p * (guard + m)], sb[p * guard:p * (guard + m)], tb[guard:guard + m]
    rc = lib.gwas_solve_block_static(g._ctx, ctypes.c_void_p(Xd.data_ptr()), Xd.stride(1), m,
                                     ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(se.data_ptr()),
                                     ctypes.c_void_p(st.data_ptr()))
    return rc, (bb, sb, tb), (b.view(m, p).T, se.view(m, p).T, st)


def _cudart_name():
    """The CUDA runtime the library itself loaded (it links it as a shared library)."""
    with open("/proc/self/maps") as f:
        for line in f:
            if "libcudart.so" in line:
                return line.split()[-1]
    pytest.skip("CUDA runtime library not found in the process")


def _host(*ts):
    return tuple(t.cpu().numpy() for t in ts)


def _blocks(n, m, seed, starts=(0, 4096)):
    torch = _torch()
    return [torch.from_numpy(np.ascontiguousarray(gwas_synth.dosages(n, c0, c0 + m, seed=seed).T)).cuda().T
            for c0 in starts]


def test_static_scratch_matches_context_scratch_twice():
    _torch()
    lib = gw.load()
    n, p, m = 1000, 4, 300
    s = gwas_synth.study(n, p, 2000, 0.6, 1.0, seed=21)
    with gw.GLS(s["Phi"], s["XL"], s["y"], 0.6, 1.0, bs=m) as g:
        for Xd in _blocks(n, m, 21):  # two calls in a row
            b_ref, se_ref, st_ref = g.solve_block(Xd)
            rc, _, (b, se, st) = _static(lib, g, Xd, m)
            assert rc == gw.GWAS_OK
            g.synchronize()
            b_ref, se_ref, st_ref = _host(b_ref, se_ref, st_ref)
            b, se, st = _host(b, se, st)
            assert np.array_equal(st, st_ref)
            assert _rel(b, b_ref) <= TOL64 and _rel(se, se_ref) <= TOL64


def test_static_on_split_context_matches_f64_entry():
    """On a BF16x3 context the static call still runs the FP64 solve: it must match
    gwas_solve_block_f64 (the FP64 solve on the context's own scratch) to 1e-10."""
    torch = _torch()
    lib = gw.load()
    n, p, m = 700, 3, 200
    s = gwas_synth.study(n, p, 1500, 0.5, 1.3, seed=22)
    with gw.GLS(s["Phi"], s["XL"], s["y"], 0.5, 1.3, precision="bf16x3", bs=256) as g:
        for Xd in _blocks(n, m, 22):
            b_ref, se_ref, st_ref = g.solve_block_f64(Xd.to(torch.float64))
            rc, _, (b, se, st) = _static(lib, g, Xd, m)
            assert rc == gw.GWAS_OK
            g.synchronize()
            b_ref, se_ref, st_ref = _host(b_ref, se_ref, st_ref)
            b, se, st = _host(b, se, st)
            assert np.array_equal(st, st_ref)
            assert _rel(b, b_ref) <= TOL64 and _rel(se, se_ref) <= TOL64


def test_static_at_the_size_limit_and_beyond():
    """The largest accepted call succeeds, writes every output element and nothing
    around the outputs; one column more is refused with GWAS_ERR_ARG."""
    _torch()
    lib = gw.load()
    n, p = 1000, 4
    s = gwas_synth.study(n, p, 2000, 0.6, 1.0, seed=23)
    n_pad = (n + 127) // 128 * 128
    mx = _max_cols(n_pad)
    assert _need(n_pad, mx) <= LIMIT < _need(n_pad, mx + 1)
    guard = 64
    with gw.GLS(s["Phi"], s["XL"], s["y"], 0.6, 1.0, bs=mx + 1) as g:
        Xd = _blocks(n, mx + 1, 23, starts=(0,))[0]
        b_ref, se_ref, st_ref = g.solve_block(Xd[:, :mx])
        rc, (bb, sb, tb), (b, se, st) = _static(lib, g, Xd[:, :mx], mx, guard=guard)
        assert rc == gw.GWAS_OK
        g.synchronize()
        bb, sb, tb = _host(bb, sb, tb)
        for buf, per in ((bb, p), (sb, p), (tb, 1)):
            assert np.all(buf[:per * guard] == buf[0]) and np.all(buf[-per * guard:] == buf[0])
        b_ref, se_ref, st_ref = _host(b_ref, se_ref, st_ref)
        b, se, st = _host(b, se, st)
        assert np.all(np.isin(st, (gw.SNP_OK, gw.SNP_SINGULAR)))
        assert np.array_equal(st, st_ref)
        assert _rel(b, b_ref) <= TOL64 and _rel(se, se_ref) <= TOL64
        # one column beyond the fixed scratch: refused before anything is launched or read
        rc, _, _ = _static(lib, g, Xd, mx + 1)
        assert rc == gw.GWAS_ERR_ARG


def test_static_call_with_device_memory_full():
    """After gwas_init the call needs no device memory: with the device's memory
    taken (all but a few MiB, fewer than the fixed array holds) it still succeeds
    and matches the context-scratch solve."""
    torch = _torch()
    lib = gw.load()
    n, p, m = 800, 4, 256
    s = gwas_synth.study(n, p, 1600, 0.4, 1.0, seed=24)
    with gw.GLS(s["Phi"], s["XL"], s["y"], 0.4, 1.0, bs=m) as g:
        Xd = _blocks(n, m, 24, starts=(8192,))[0]
        b_ref, se_ref, st_ref = g.solve_block(Xd)
        g.synchronize()
        b_ref, se_ref, st_ref = _host(b_ref, se_ref, st_ref)
        # outputs first, then take the device's memory
        b = torch.full((m, p), float("nan"), dtype=torch.float64, device="cuda").T
        se = torch.full((m, p), float("nan"), dtype=torch.float64, device="cuda").T
        st = torch.full((m,), -1, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        cudart = ctypes.CDLL(_cudart_name())
        cudart.cudaMalloc.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_size_t]
        cudart.cudaFree.argtypes = [ctypes.c_void_p]
        hold, raw = [], []
        try:
            size = 1 << 34
            while size >= (1 << 24):  # large torch blocks first ...
                try:
                    hold.append(torch.empty(size, dtype=torch.uint8, device="cuda"))
                except torch.OutOfMemoryError:
                    size //= 2
            size = 1 << 24
            while size >= (1 << 18):  # ... then plain cudaMalloc down to 256 KiB
                ptr = ctypes.c_void_p()
                if cudart.cudaMalloc(ctypes.byref(ptr), size) == 0:
                    raw.append(ptr)
                else:
                    size //= 2
            cudart.cudaGetLastError()
            free, _ = torch.cuda.mem_get_info()
            assert free < 8 * 1024 * 1024, free  # a quarter of what the fixed array would need
            rc = lib.gwas_solve_block_static(g._ctx, ctypes.c_void_p(Xd.data_ptr()), Xd.stride(1), m,
                                             ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(se.data_ptr()),
                                             ctypes.c_void_p(st.data_ptr()))
            torch.cuda.synchronize()
            assert rc == gw.GWAS_OK, (rc, lib.gwas_last_error_detail(g._ctx))
        finally:
            for ptr in raw:
                cudart.cudaFree(ptr)
            hold.clear()
            torch.cuda.empty_cache()
        g.synchronize()
        b, se, st = _host(b, se, st)
        assert np.array_equal(st, st_ref)
        assert _rel(b, b_ref) <= TOL64 and _rel(se, se_ref) <= TOL64
