"""The differentiation form on the GPU (FP64) against the oracle's dense-form
gradients, central differences, and the REML fit of h against the oracle."""
import numpy as np
import pytest

import gwas_synth
import oracle
import paper_1302_4332_b300 as gw

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1302_4332_b300 import build
    build.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("n,p,m,h,sigma2", [(300, 4, 70, 0.5, 1.3), (129, 2, 65, 0.8, 1.0), (257, 6, 40, 0.3, 0.7)])
def test_adjoint_matches_oracle(n, p, m, h, sigma2):
    s = gwas_synth.study(n, p, 2 * n, h, sigma2, seed=5)
    X = gwas_synth.dosages(n, 0, m, seed=5)
    L = oracle.potrf(oracle.form_m(s["Phi"], h, sigma2))
    c_ref, dh_ref, dy_ref = oracle.gls_grad(L, s["Phi"], h, sigma2, s["XL"], s["y"], X)
    with gw.GLS(s["Phi"], s["XL"], s["y"], h, sigma2, bs=64) as g:
        dh, dy = np.zeros(1), np.zeros(n)
        chi2, dch = [], []
        for c0 in range(0, m, 64):
            c, d, dh, dy = g.adjoint_block(X[:, c0:c0 + 64], dh_accum=dh, dy_accum=dy)
            chi2.append(c.copy())
            dch.append(d.copy())
    chi2, dch = np.concatenate(chi2), np.concatenate(dch)
    assert _rel(chi2, c_ref) <= 1e-10
    assert _rel(dch, dh_ref) <= 1e-9
    assert abs(dh[0] - dh_ref.sum()) <= 1e-9 * np.abs(dh_ref).sum()
    assert _rel(dy, dy_ref) <= 1e-9


def test_autograd_matches_central_differences():
    import torch
    from paper_1302_4332_b300.autograd import wald_chi2_sum
    n, p, m = 200, 4, 96
    s = gwas_synth.study(n, p, 400, 0.6, 1.0, seed=8)
    blocks = [gwas_synth.dosages(n, 0, 48, seed=8), gwas_synth.dosages(n, 48, m, seed=8)]
    h = torch.tensor(0.6, dtype=torch.float64, requires_grad=True)
    y = torch.tensor(s["y"], dtype=torch.float64, requires_grad=True)
    loss = wald_chi2_sum(h, y, s["Phi"], s["XL"], blocks, bs=64)
    loss.backward()
    f = lambda hh, yy: float(wald_chi2_sum(torch.tensor(hh, dtype=torch.float64),
                                           torch.tensor(yy, dtype=torch.float64), s["Phi"], s["XL"], blocks, bs=64))
    d = 1e-6
    fd_h = (f(0.6 + d, s["y"]) - f(0.6 - d, s["y"])) / (2 * d)
    assert abs(h.grad.item() - fd_h) <= 1e-6 * abs(fd_h)
    for j in (0, 57, 199):
        yp, ym = s["y"].copy(), s["y"].copy()
        yp[j] += d
        ym[j] -= d
        fd = (f(0.6, yp) - f(0.6, ym)) / (2 * d)
        assert abs(y.grad[j].item() - fd) <= 1e-6 * max(1.0, abs(fd)), (j, y.grad[j].item(), fd)


def test_adjoint_paper_scale_n5000():
    """The differentiation workload: n = 5,000, p = 4, h = 0.5, one 512-SNP block."""
    n, p, m = 5000, 4, 512
    s = gwas_synth.study(n, p, 5000, 0.5, 1.0, seed=4)
    X = gwas_synth.dosages(n, 0, m, seed=4)
    L = oracle.potrf(oracle.form_m(s["Phi"], 0.5, 1.0))
    c_ref, dh_ref, dy_ref = oracle.gls_grad(L, s["Phi"], 0.5, 1.0, s["XL"], s["y"], X)
    with gw.GLS(s["Phi"], s["XL"], s["y"], 0.5, 1.0, bs=m) as g:
        chi2, dch, dh, dy = g.adjoint_block(X)
    assert _rel(chi2, c_ref) <= 1e-10
    assert _rel(dch, dh_ref) <= 1e-6 and abs(dh[0] - dh_ref.sum()) <= 1e-6 * np.abs(dh_ref).sum()
    assert _rel(dy, dy_ref) <= 1e-6


# ---------------------------------------------------------- split precision
# The split contexts' adjoint forms every per-SNP input from one exact integer
# product on the tensor cores (sliced M^-1 and linear functionals times the
# shifted dosages, FP16 slices, FP32 accumulation kept below 2^24), then the
# per-SNP adjoint arithmetic in FP64: the gradient bar is the FP64 one.
SPLIT_ADJ_TOL = {"bf16x3": 1e-6, "tf32x3": 1e-6, "f16x2": 1e-6}


@pytest.mark.parametrize("prec,tiles", [("bf16x3", "pair_mma"), ("bf16x3", "inverse"), ("tf32x3", "pair_mma"),
                                        ("tf32x3", "inverse"), ("f16x2", "inverse")])
@pytest.mark.parametrize("n,p,m,h,sigma2", [(300, 4, 300, 0.5, 1.3), (1000, 3, 513, 0.7, 1.0)])
def test_split_adjoint_matches_oracle(prec, n, p, m, h, sigma2, tiles):
    s = gwas_synth.study(n, p, 2 * n, h, sigma2, seed=6)
    X = gwas_synth.dosages(n, 0, m, seed=6)
    L = oracle.potrf(oracle.form_m(s["Phi"], h, sigma2))
    c_ref, dh_ref, dy_ref = oracle.gls_grad(L, s["Phi"], h, sigma2, s["XL"], s["y"], X)
    with gw.GLS(s["Phi"], s["XL"], s["y"], h, sigma2, bs=512, precision=prec, tiles=tiles) as g:
        dh, dy = np.zeros(1), np.zeros(n)
        chi2, dch = [], []
        for c0 in range(0, m, 512):
            c, d, dh, dy = g.adjoint_block(X[:, c0:c0 + 512], dh_accum=dh, dy_accum=dy)
            chi2.append(c.copy())
            dch.append(d.copy())
    chi2, dch = np.concatenate(chi2), np.concatenate(dch)
    errs = dict(chi2=_rel(chi2, c_ref), dchi2_dh=_rel(dch, dh_ref),
                dh_sum=abs(dh[0] - dh_ref.sum()) / np.abs(dh_ref).sum(), dy=_rel(dy, dy_ref))
    print(prec, tiles, n, "split adjoint", errs)
    tol = SPLIT_ADJ_TOL[prec]
    assert all(v <= tol for v in errs.values()), (prec, tiles, errs)


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
def test_split_adjoint_paper_scale_n5000(prec):
    n, p, m = 5000, 4, 512
    s = gwas_synth.study(n, p, 5000, 0.5, 1.0, seed=4)
    X = gwas_synth.dosages(n, 0, m, seed=4)
    L = oracle.potrf(oracle.form_m(s["Phi"], 0.5, 1.0))
    c_ref, dh_ref, dy_ref = oracle.gls_grad(L, s["Phi"], 0.5, 1.0, s["XL"], s["y"], X)
    with gw.GLS(s["Phi"], s["XL"], s["y"], 0.5, 1.0, bs=m, precision=prec) as g:
        chi2, dch, dh, dy = g.adjoint_block(X)
    errs = dict(chi2=_rel(chi2, c_ref), dchi2_dh=_rel(dch, dh_ref),
                dh_sum=abs(dh[0] - dh_ref.sum()) / np.abs(dh_ref).sum(), dy=_rel(dy, dy_ref))
    print(prec, n, "split adjoint", errs)
    tol = SPLIT_ADJ_TOL[prec]
    assert all(v <= tol for v in errs.values()), (prec, errs)


def test_split_adjoint_config4_sample_across_m100k():
    """The differentiation workload's scale: n = 5,000, p = 4, h = 0.5, SNPs
    from m = 100,000; 2,048 of them in 8 seeded 256-column chunks spread over
    the whole range, every one against the oracle's FP64 gradient (chi2,
    d chi2/dh per SNP and summed, d/dy of the sample's sum)."""
    n, p, m = 5000, 4, 100_000
    s = gwas_synth.study(n, p, 5000, 0.5, 1.0, study_id=4)
    rng = np.random.default_rng(20130218)
    chunks = np.sort(rng.choice(m // gwas_synth.CHUNK, 8, replace=False))
    X = np.asfortranarray(np.column_stack([gwas_synth.dosages(n, c * gwas_synth.CHUNK, (c + 1) * gwas_synth.CHUNK,
                                                              study=4) for c in chunks]))
    L = oracle.potrf(oracle.form_m(s["Phi"], 0.5, 1.0))
    c_ref, dh_ref, dy_ref = oracle.gls_grad(L, s["Phi"], 0.5, 1.0, s["XL"], s["y"], X)
    for prec in ("bf16x3", "f16x2"):
        with gw.GLS(s["Phi"], s["XL"], s["y"], 0.5, 1.0, bs=1024, precision=prec) as g:
            dh, dy = np.zeros(1), np.zeros(n)
            chi2, dch = [], []
            for c0 in range(0, X.shape[1], 1024):
                c, d, dh, dy = g.adjoint_block(X[:, c0:c0 + 1024], dh_accum=dh, dy_accum=dy)
                chi2.append(c.copy())
                dch.append(d.copy())
        chi2, dch = np.concatenate(chi2), np.concatenate(dch)
        errs = dict(chi2=_rel(chi2, c_ref), dchi2_dh=_rel(dch, dh_ref),
                    dh_sum=abs(dh[0] - dh_ref.sum()) / np.abs(dh_ref).sum(), dy=_rel(dy, dy_ref))
        print(prec, "config-4 sample", errs)
        assert all(v <= SPLIT_ADJ_TOL[prec] for v in errs.values()), (prec, errs)


def test_split_adjoint_wide_integer_values():
    """Columns of arbitrary int8 values (|x - c| up to ~120): the exact products
    then split each tile's 3 K-blocks over two TMEM partials (at most 256 /
    120 K-blocks per partial); the result still meets the FP64 gradient bar."""
    n, p, m = 300, 3, 96
    s = gwas_synth.study(n, p, 600, 0.4, 1.1, seed=13)
    rng = np.random.default_rng(13)
    X = np.asfortranarray(rng.integers(-120, 121, size=(n, m)).astype(np.int8))
    L = oracle.potrf(oracle.form_m(s["Phi"], 0.4, 1.1))
    c_ref, dh_ref, dy_ref = oracle.gls_grad(L, s["Phi"], 0.4, 1.1, s["XL"], s["y"], X)
    with gw.GLS(s["Phi"], s["XL"], s["y"], 0.4, 1.1, bs=m, precision="bf16x3") as g:
        chi2, dch, dh, dy = g.adjoint_block(X)
    errs = dict(chi2=_rel(chi2, c_ref), dchi2_dh=_rel(dch, dh_ref), dy=_rel(dy, dy_ref))
    assert all(v <= 1e-6 for v in errs.values()), errs


def test_split_autograd_matches_central_differences():
    """The split adjoint's gradient against central differences of the split
    forward loss itself (both sides on the tensor cores)."""
    import torch
    from paper_1302_4332_b300.autograd import wald_chi2_sum
    n, m = 300, 128
    s = gwas_synth.study(n, 4, 600, 0.6, 1.0, seed=9)
    blocks = [gwas_synth.dosages(n, 0, m, seed=9)]
    h = torch.tensor(0.6, dtype=torch.float64, requires_grad=True)
    loss = wald_chi2_sum(h, torch.tensor(s["y"]), s["Phi"], s["XL"], blocks, bs=m, precision="tf32x3")
    loss.backward()
    f = lambda hh: float(wald_chi2_sum(torch.tensor(hh, dtype=torch.float64), torch.tensor(s["y"]), s["Phi"],
                                       s["XL"], blocks, bs=m, precision="tf32x3"))
    # the split loss moves in steps of ~1e-9 relative as the slices of M^-1
    # round differently with h: a wider step than FP64's keeps that below 1e-5
    d = 1e-4
    fd_h = (f(0.6 + d) - f(0.6 - d)) / (2 * d)
    print("split autograd", h.grad.item(), fd_h)
    assert abs(h.grad.item() - fd_h) <= 5e-5 * abs(fd_h)


@pytest.mark.parametrize("h", [0.2, 0.5, 0.9])
def test_reml_eval_matches_oracle(h):
    s = gwas_synth.study(400, 3, 800, 0.5, seed=6)
    l, dl, s2 = gw.reml_eval(s["Phi"], s["XL"], s["y"], h)
    lo, dlo, s2o = oracle.reml(s["Phi"], s["XL"], s["y"], h)
    assert abs(l - lo) <= 1e-9 * abs(lo)
    assert abs(dl - dlo) <= 1e-8 * max(1.0, abs(dlo))
    assert abs(s2 - s2o) <= 1e-10 * s2o


def test_reml_fit_matches_oracle_argmax():
    s = gwas_synth.study(600, 3, 1200, 0.5, seed=10)
    h_hat, ll, evals = gw.reml_fit(s["Phi"], s["XL"], s["y"], h0=0.2, tol=1e-9)
    h_ref = oracle.reml_argmax(s["Phi"], s["XL"], s["y"], tol=1e-9)
    assert abs(h_hat - h_ref) <= 1e-6, (h_hat, h_ref, evals)


def test_reml_fit_n2000_oracle_gradient_changes_sign():
    """A larger null model: the oracle's dense dl/dh changes sign across the GPU fit."""
    s = gwas_synth.study(2000, 3, 2000, 0.5, seed=12)
    h_hat, ll, evals = gw.reml_fit(s["Phi"], s["XL"], s["y"], h0=0.2, tol=1e-9)
    g_lo = oracle.reml(s["Phi"], s["XL"], s["y"], h_hat - 1e-6)[1]
    g_hi = oracle.reml(s["Phi"], s["XL"], s["y"], h_hat + 1e-6)[1]
    assert g_lo > 0 > g_hi, (h_hat, g_lo, g_hi)
