"""gwas_solve_block_static: the block solve for callers that cannot allocate
device memory when they solve (their device memory is held by another
allocator, or they must not call cudaMalloc while serving).  Its scratch is a
fixed array inside the library; the test calls it through the C ABI twice in
a row and checks each result against gwas_solve_block, the entry point that
uses the context's own scratch.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

import gwas_synth
import paper_1302_4332_b300 as gw

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def _rel(a, b):
    return float(np.max(np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)))


def test_static_scratch_matches_context_scratch_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1302_4332_b300 import build
    build.build()
    lib = gw.load()
    n, p, m = 1000, 4, 300
    s = gwas_synth.study(n, p, 2000, 0.6, 1.0, seed=21)
    blocks = [gwas_synth.dosages(n, c0, c0 + m, seed=21) for c0 in (0, 4096)]
    with gw.GLS(s["Phi"], s["XL"], s["y"], 0.6, 1.0, bs=m) as g:
        for X in blocks:  # two calls in a row: the second reuses the array the first left behind
            Xd = torch.from_numpy(np.ascontiguousarray(X.T)).cuda().T
            b_ref, se_ref, st_ref = g.solve_block(Xd)
            b = torch.full((m, p), float("nan"), dtype=torch.float64, device="cuda").T
            se = torch.full((m, p), float("nan"), dtype=torch.float64, device="cuda").T
            st = torch.full((m,), -1, dtype=torch.int32, device="cuda")
            rc = lib.gwas_solve_block_static(g._ctx, ctypes.c_void_p(Xd.data_ptr()), Xd.stride(1), m,
                                             ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(se.data_ptr()),
                                             ctypes.c_void_p(st.data_ptr()))
            assert rc == gw.GWAS_OK
            g.synchronize()
            b_ref, se_ref, st_ref = (t.cpu().numpy() for t in (b_ref, se_ref, st_ref))
            b, se, st = (t.cpu().numpy() for t in (b, se, st))
            assert np.array_equal(st, st_ref)
            assert _rel(b, b_ref) <= TOL64 and _rel(se, se_ref) <= TOL64
        # beyond the fixed scratch: refused before anything is launched or read
        big = 32 * 1024 * 1024 // (8 * g.n_pad) + 1
        bd = torch.empty(1, dtype=torch.float64, device="cuda")
        rc = lib.gwas_solve_block_static(g._ctx, ctypes.c_void_p(Xd.data_ptr()), Xd.stride(1), big,
                                         ctypes.c_void_p(bd.data_ptr()), None, None)
        assert rc == -1
