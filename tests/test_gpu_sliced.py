"""The sliced solve (GWAS_SLICED64) against the FP64 oracle at the FP64 bar.

Eq. 1's X_i^T M^-1 X_i and X_i^T M^-1 y from exact integer products of a
sliced M^-1 with the shifted int8 dosages on the tensor cores; the only error
is the 44-bit representation of M^-1's triangle, so every check here uses the
FP64 path's tolerance: per-SNP normwise b, b in units of se, and se
component-wise, all <= 1e-10, statuses identical."""
import numpy as np
import pytest

import gwas_synth
import oracle
import paper_1302_4332_b300 as gw
from oracle.metrics import compare

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1302_4332_b300 import build
    build.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _case(n, p, k, h, sigma2=1.0, m=64, seed=11, c0=0):
    s = gwas_synth.study(n, p, k, h, sigma2, seed=seed)
    X = gwas_synth.dosages(n, c0, c0 + m, seed=seed)
    L = oracle.potrf(oracle.form_m(s["Phi"], h, sigma2))
    return s, X, L


def _check(b, se_g, st_g, r, se, st, what):
    e = compare(b, se_g, st_g, r, se, st)
    print(what, e)
    assert e["b_norm"] <= TOL64 and e["b_se_scaled"] <= TOL64 and e["se_rel"] <= TOL64, (what, e)
    return e


# n: 1 (one panel, one pair holding the appended rows), 127 / 129 (a ragged
# last row panel), 255 / 257 / 640 (odd and even numbers of row panels), 1000;
# p = 1 (no intercept: no shift), 16 (the most covariates); m ragged against
# the 256-column strips
@pytest.mark.parametrize("n,p,m", [(1, 1, 3), (5, 2, 1), (127, 4, 63), (129, 4, 65), (255, 3, 257),
                                   (257, 1, 129), (300, 7, 300), (640, 16, 70), (1000, 4, 513)])
def test_ragged_shapes(n, p, m):
    s, X, L = _case(n, p, max(2 * n, 4), 0.5, sigma2=1.3, m=m)
    r, se, _, st = oracle.gls(L, s["XL"], s["y"], X)
    with gw.GLS(s["Phi"], s["XL"] if p > 1 else None, s["y"], 0.5, 1.3, precision="sliced64", bs=max(m, 1)) as g:
        b, se_g, st_g = g.solve_block(X)
    _check(b, se_g, st_g, r, se, st, (n, p, m))


def test_blocks_stream_and_device_io():
    """Several blocks of one context (the last one short), the stream form over
    the same columns bit for bit, device tensors in and out, an unaligned
    device leading dimension."""
    import torch
    s, X, L = _case(1000, 4, 2000, 0.6, m=1500)
    r, se, _, st = oracle.gls(L, s["XL"], s["y"], X)
    with gw.GLS(s["Phi"], s["XL"], s["y"], 0.6, 1.0, precision="sliced64", bs=512) as g:
        outs = [g.solve_block(X[:, c0:c0 + 512]) for c0 in range(0, 1500, 512)]
        b = np.concatenate([o[0] for o in outs], axis=1)
        se_g = np.concatenate([o[1] for o in outs], axis=1)
        st_g = np.concatenate([o[2] for o in outs])
        _check(b, se_g, st_g, r, se, st, "blocks")
        b_s, se_s, st_s = g.solve_stream(np.asfortranarray(X))
        assert np.array_equal(b, b_s) and np.array_equal(se_g, se_s) and np.array_equal(st_g, st_s)
        buf = torch.zeros((300, 1003), dtype=torch.int8, device="cuda")
        buf[:, :1000] = torch.from_numpy(np.ascontiguousarray(X[:, :300].T)).cuda()
        Xd = buf.T[:1000]
        bd, sed, std = g.solve_block(Xd)
        g.synchronize()
        assert np.array_equal(bd.cpu().numpy(), b[:, :300]) and np.array_equal(sed.cpu().numpy(), se_g[:, :300])
        assert np.array_equal(std.cpu().numpy(), st_g[:300])


def test_singular_and_near_singular():
    """A monomorphic SNP and an all-zero SNP are flagged; a SNP with one
    deviating sample is a valid, ill-conditioned design (S_BR / d^2 ~ 4n)."""
    s, X, L = _case(200, 4, 400, 0.6, m=6)
    X[:, 1] = 2
    X[:, 2] = 0
    X[:, 3] = 2
    X[17, 3] = 1
    r, se, _, st = oracle.gls(L, s["XL"], s["y"], X)
    assert st.tolist() == [0, 1, 1, 0, 0, 0]
    with gw.GLS(s["Phi"], s["XL"], s["y"], 0.6, 1.0, precision="sliced64", bs=64) as g:
        b, se_g, st_g = g.solve_block(X)
    assert st_g.tolist() == st.tolist()
    assert np.isnan(b[:, 1]).all() and np.isnan(b[:, 2]).all()
    _check(b, se_g, st_g, r, se, st, "with the near-singular SNP")


def test_arbitrary_int8_values():
    """Columns of arbitrary int8 values (|x - c| up to ~250): the partial sums
    of the product stay exact with one K-block per TMEM partial."""
    n, p, m = 640, 4, 200
    s, _, L = _case(n, p, 2 * n, 0.5, m=1)
    rng = np.random.default_rng(5)
    X = np.asfortranarray(rng.integers(-128, 128, size=(n, m)).astype(np.int8))
    X[:, 0] = 127
    X[::2, 0] = -128  # the largest spread about the shift
    X[:, 1] = rng.integers(0, 3, size=n)  # dosages beside them
    X[:, 2] = 127
    X[:10, 2] = -128  # shift 123, |x - c| = 251: one K-block per partial
    r, se, _, st = oracle.gls(L, s["XL"], s["y"], X)
    with gw.GLS(s["Phi"], s["XL"], s["y"], 0.5, 1.0, precision="sliced64", bs=m) as g:
        b, se_g, st_g = g.solve_block(X)
    _check(b, se_g, st_g, r, se, st, "int8")


@pytest.mark.parametrize("h", (0.0, 1.0, 0.5))
@pytest.mark.parametrize("sigma2", (1e-6, 1.0, 1e4))
def test_h_and_sigma2_edges(h, sigma2):
    """h = 0 (M = sigma2 I), h = 1 (M = sigma2 Phi, condition ~3e3 here) and
    extreme sigma2: the power-of-two scales of the slices absorb any magnitude
    of M^-1.  At sigma2 = 1e-6 the z-scores b / se reach ~1e5, so b in units of
    se carries FP64's own rounding times z: there the bar is the FP64 path's
    own error on the same SNPs (x 10), next to the normwise 1e-10."""
    s, X, L = _case(300, 4, 600, h, sigma2=sigma2, m=50)
    r, se, _, st = oracle.gls(L, s["XL"], s["y"], X)
    with gw.GLS(s["Phi"], s["XL"], s["y"], h, sigma2, precision="sliced64", bs=64) as g:
        b, se_g, st_g = g.solve_block(X)
    with gw.GLS(s["Phi"], s["XL"], s["y"], h, sigma2, precision="fp64", bs=64) as g:
        b64, se64, st64 = g.solve_block(X)
    e = compare(b, se_g, st_g, r, se, st)
    e64 = compare(b64, se64, st64, r, se, st)
    print((h, sigma2), "sliced", e, "fp64", e64)
    assert e["b_norm"] <= TOL64 and e["se_rel"] <= TOL64, e
    assert e["b_se_scaled"] <= max(TOL64, 10 * e64["b_se_scaled"]), (e, e64)


def test_options_that_do_not_apply():
    s, X, L = _case(200, 4, 400, 0.6, m=8)
    for kw in (dict(tiles="pair_mma"), dict(tiles="inverse"), dict(strip_group=4), dict(separate_sums=True),
               dict(single_piece=True)):
        with pytest.raises(gw.GwasError) as e:
            gw.GLS(s["Phi"], s["XL"], s["y"], 0.6, 1.0, precision="sliced64", bs=64, **kw)
        assert e.value.name == "GWAS_ERR_ARG", kw
    with gw.GLS(s["Phi"], s["XL"], s["y"], 0.6, 1.0, precision="sliced64", bs=64) as g:
        ctas, cluster, mode = g.solve_shape()
        assert cluster == 2 and ctas >= 2 and ctas % 2 == 0 and mode == "auto"
        with pytest.raises(gw.GwasError):
            gw.GLSBatch([g])  # batches take the split precisions only
        # the FP64 entry point runs the FP64 solve on any context
        b, se_g, st_g = g.solve_block_f64(X.astype(np.float64))
        r, se, _, st = oracle.gls(L, s["XL"], s["y"], X)
        _check(b, se_g, st_g, r, se, st, "f64 input")


def test_adjoint_on_a_sliced_context():
    """The adjoint on a sliced context runs the exact-product adjoint; its
    chi2 and gradients match the oracle's at the adjoint's bar (1e-6)."""
    n, m = 300, 64
    s, X, L = _case(n, 4, 2 * n, 0.5, m=m)
    chi2_o, dh_o, dy_o = oracle.gls_grad(L, s["Phi"], 0.5, 1.0, s["XL"], s["y"], X)
    with gw.GLS(s["Phi"], s["XL"], s["y"], 0.5, 1.0, precision="sliced64", bs=m) as g:
        chi2, dch, dh_acc, dy_acc = g.adjoint_block(X)
    assert np.max(np.abs(chi2 - chi2_o) / np.abs(chi2_o)) <= 1e-6
    assert np.linalg.norm(dch - dh_o) / np.linalg.norm(dh_o) <= 1e-6
    assert abs(dh_acc[0] - dh_o.sum()) / abs(dh_o.sum()) <= 1e-6
    assert np.linalg.norm(dy_acc - dy_o) / np.linalg.norm(dy_o) <= 1e-6


def test_int8_range_limit():
    """The int32 product totals bound max|x - c| * 1024 * n_pad below 2^31:
    a column with |x - c| = 255 is solved exactly at n = 8,192 (n_pad = 8,192)
    and refused with GWAS_ERR_ARG one row panel later (n_pad = 8,320), where
    dosage columns still solve."""
    for n, ok in ((8192, True), (8193, False)):
        s = gwas_synth.study(n, 4, 256, 0.5, 1.0, seed=3)
        X = np.asfortranarray(gwas_synth.dosages(n, 0, 6, seed=3))
        Xw = X.copy(order="F")
        Xw[:, 2] = 127
        Xw[:10, 2] = -128  # shift 127: |x - c| = 255
        with gw.GLS(s["Phi"], s["XL"], s["y"], 0.5, 1.0, precision="fp64", bs=8) as g:
            b64, se64, st64 = g.solve_block(Xw)
        with gw.GLS(s["Phi"], s["XL"], s["y"], 0.5, 1.0, precision="sliced64", bs=8) as g:
            if ok:
                b, se_g, st_g = g.solve_block(Xw)
                _check(b, se_g, st_g, b64, se64, st64, ("int8 extremes", n))
            else:
                with pytest.raises(gw.GwasError) as e:
                    g.solve_block(Xw)
                assert e.value.name == "GWAS_ERR_ARG"
                b, se_g, st_g = g.solve_block(X)  # the context stays usable
                with gw.GLS(s["Phi"], s["XL"], s["y"], 0.5, 1.0, precision="fp64", bs=8) as g64:
                    r, se, st = g64.solve_block(X)
                _check(b, se_g, st_g, r, se, st, ("dosages", n))
