"""Failure detection and bounds, on the GPU without a fault.

* Bounded device-side waits: a wait on a flag (or an mbarrier phase) that
  nothing ever provides runs out after its limit, the device records it, the
  host reports GWAS_ERR_TIMEOUT and clears it, and the context keeps working.
* Output bounds: every output buffer sits between guard regions filled with a
  sentinel; after ragged solves (column counts off every tile and chunk size)
  the guards are untouched, in every path and both forms of the per-SNP sums."""
import time

import numpy as np
import pytest

import gwas_synth
import oracle
import paper_1302_4332_b300 as gw
from oracle.metrics import compare

pytestmark = pytest.mark.gpu

GWAS_ERR_ARG, GWAS_ERR_TIMEOUT = -1, -4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1302_4332_b300 import build
    build.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(scope="module")
def study():
    s = gwas_synth.study(300, 4, 600, 0.5, 1.0, seed=41)
    X = gwas_synth.dosages(300, 0, 600, seed=41)
    L = oracle.potrf(oracle.form_m(s["Phi"], 0.5, 1.0))
    return s, X, oracle.gls(L, s["XL"], s["y"], X)


@pytest.mark.parametrize("prec", ("fp64", "f16x2"))
@pytest.mark.parametrize("kind", (0, 1))
def test_bounded_wait_reports_and_recovers(study, prec, kind):
    s, X, (r, se, _, st) = study
    with gw.GLS(s["Phi"], s["XL"], s["y"], 0.5, 1.0, precision=prec, bs=600) as g:
        t0 = time.perf_counter()
        assert g.check_timeout(kind, 20000) == GWAS_ERR_TIMEOUT  # 20 ms
        assert time.perf_counter() - t0 < 5.0
        assert g.check_timeout(2, 20000) == GWAS_ERR_ARG and g.check_timeout(kind, 0) == GWAS_ERR_ARG
        b, se_g, st_g = g.solve_block(X)  # the context is still usable, with the status cleared
        g.synchronize()
    e = compare(b, se_g, st_g, r, se, st)
    assert e["b_norm"] <= (1e-10 if prec == "fp64" else 1e-5), e


SENT_F = np.frombuffer(np.uint64(0x7FF4DEADBEEF0001).tobytes(), dtype=np.float64)[0]  # a NaN payload
SENT_I = 0x5A5A5A5A
G = 37  # guard elements on each side


def _guarded(torch, shape_cols, p, on_dev):
    """b, se (p x cols column-major) and status views into buffers with G guard
    columns (elements) before and after, all filled with the sentinel."""
    if on_dev:
        fb = torch.full(((shape_cols + 2 * G) * p,), 0.0, dtype=torch.float64, device="cuda")
        fb.view(torch.int64).fill_(0x7FF4DEADBEEF0001)
        fs = fb.clone()
        fi = torch.full((shape_cols + 2 * G,), SENT_I, dtype=torch.int32, device="cuda")
        b = fb[G * p:(G + shape_cols) * p].view(shape_cols, p).T
        se = fs[G * p:(G + shape_cols) * p].view(shape_cols, p).T
        st = fi[G:G + shape_cols]
        return (fb, fs, fi), (b, se, st)
    fb = np.full((shape_cols + 2 * G) * p, SENT_F)
    fs = fb.copy()
    fi = np.full(shape_cols + 2 * G, SENT_I, dtype=np.int32)
    b = fb[G * p:(G + shape_cols) * p].reshape(shape_cols, p).T
    se = fs[G * p:(G + shape_cols) * p].reshape(shape_cols, p).T
    st = fi[G:G + shape_cols]
    return (fb, fs, fi), (b, se, st)


def _guards_intact(bufs, cols, p):
    fb, fs, fi = [x.cpu().numpy() if hasattr(x, "cpu") else x for x in bufs]
    sent = np.uint64(0x7FF4DEADBEEF0001)
    for f in (fb, fs):
        u = f.view(np.uint64)
        if not (np.all(u[:G * p] == sent) and np.all(u[(G + cols) * p:] == sent)):
            return False
        if np.any(u[G * p:(G + cols) * p] == sent):  # every output element written
            return False
    return bool(np.all(fi[:G] == SENT_I) and np.all(fi[G + cols:] == SENT_I))


@pytest.mark.parametrize("prec,sep", [("fp64", False), ("bf16x3", False), ("bf16x3", True), ("tf32x3", False),
                                      ("f16x2", False), ("f16x2", True)])
@pytest.mark.parametrize("on_dev", (True, False))
def test_output_guards(study, prec, sep, on_dev):
    import torch
    s, X, (r, se, _, st) = study
    with gw.GLS(s["Phi"], s["XL"], s["y"], 0.5, 1.0, precision=prec, bs=600, separate_sums=sep) as g:
        for cols in (1, 15, 17, 255, 257, 511, 600):
            bufs, (b, se_o, st_o) = _guarded(torch, cols, 4, on_dev)
            Xc = X[:, :cols]
            if on_dev:
                Xc = torch.from_numpy(np.ascontiguousarray(Xc.T)).cuda().T
            g.solve_block(Xc, b, se_o, st_o)
            g.synchronize()
            assert _guards_intact(bufs, cols, 4), (prec, sep, on_dev, cols)
            bb = b.cpu().numpy() if on_dev else b
            ss = se_o.cpu().numpy() if on_dev else se_o
            tt = st_o.cpu().numpy() if on_dev else st_o
            e = compare(bb, ss, tt, r[:, :cols], se[:, :cols], st[:cols])
            assert e["b_norm"] <= (1e-10 if prec == "fp64" else 1e-5), (prec, cols, e)
