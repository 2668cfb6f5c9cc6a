"""Paths that only large studies take: n > 16,384 (n_pad = 16,512, 129 row
panels), where the split inverse form's cast reads each column twice (its
register-held form covers n <= 16,384), the sliced solve's integer totals
approach their bound, and the split adjoint sums ||x^'||^2 in FP64 (its exact
int64 form needs 512 max|x'| n_pad <= 2^24).  The reference factor is LAPACK's
Cholesky (numpy; the oracle's own potrf is pinned to it on small cases), the
per-SNP GLS the oracle's."""
import numpy as np
import pytest

import gwas_synth
import oracle
import paper_1302_4332_b300 as gw
from oracle.metrics import compare

pytestmark = pytest.mark.gpu

N, P, H, S2 = 16500, 4, 0.5, 1.3
TOL = {"fp64": 1e-10, "sliced64": 1e-10, "bf16x3": 1e-5, "f16x2": 1e-5, "tf32x3": 1e-5}


@pytest.fixture(scope="module")
def case():
    from paper_1302_4332_b300 import build
    build.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    s = gwas_synth.study(N, P, 500, H, S2, seed=17)
    X = gwas_synth.dosages(N, 0, 300, seed=17)
    L = np.linalg.cholesky(oracle.form_m(s["Phi"], H, S2))
    cols = np.r_[0:16, 284:300]  # first and last SNPs of the block
    r, se, _, st = oracle.gls(L, s["XL"], s["y"], np.asfortranarray(X[:, cols]))
    return s, X, cols, (r, se, st)


@pytest.mark.parametrize("prec", ["fp64", "f16x2", "bf16x3", "sliced64"])
def test_solve_beyond_16384_rows(case, prec):
    s, X, cols, (r, se, st) = case
    with gw.GLS(s["Phi"], s["XL"], s["y"], H, S2, precision=prec, bs=300) as g:
        b, se_g, st_g = g.solve_block(X)
    e = compare(b[:, cols], se_g[:, cols], st_g[cols], r, se, st)
    print(prec, e)
    assert e["b_norm"] <= TOL[prec] and e["se_rel"] <= TOL[prec], (prec, e)
    assert np.array_equal(st_g[cols], st)


def test_split_adjoint_beyond_16384_rows(case):
    """The split adjoint (exact products; ||x^'||^2 summed in FP64 at this n)
    against the FP64 adjoint on the same block at the gradient bar, 1e-6."""
    s, X, _, _ = case
    out = {}
    for prec in ("fp64", "bf16x3"):
        with gw.GLS(s["Phi"], s["XL"], s["y"], H, S2, precision=prec, bs=300) as g:
            out[prec] = g.adjoint_block(X)
    chi2, dch, dh, dy = out["bf16x3"]
    chi2_r, dch_r, dh_r, dy_r = out["fp64"]
    ok = np.isfinite(chi2_r)
    assert np.max(np.abs(chi2[ok] - chi2_r[ok]) / np.abs(chi2_r[ok])) <= 1e-6
    assert np.linalg.norm(dch[ok] - dch_r[ok]) / np.linalg.norm(dch_r[ok]) <= 1e-6
    assert abs(dh[0] - dh_r[0]) / abs(dh_r[0]) <= 1e-6
    assert np.linalg.norm(dy - dy_r) / np.linalg.norm(dy_r) <= 1e-6
