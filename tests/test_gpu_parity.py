"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerance of the FP64 path: per-SNP normwise relative error of b <= 1e-10 and
component-wise relative error of se <= 1e-10; statuses identical."""
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
    r, se, _, st = oracle.gls(L, s["XL"], s["y"], X)
    return s, X, L, (r, se, st)


@pytest.fixture(scope="module")
def small_study():
    """n = 1000, p = 4, h = 0.6: the small FP64-dosage workload, all of its m = 10,000 SNPs."""
    return _case(1000, 4, 2000, 0.6, m=10000)


def test_fp64_dosages_full_parity(small_study):
    s, X, L, (r, se, st) = small_study
    with gw.GLS(s["Phi"], s["XL"], s["y"], s["h"], s["sigma2"], bs=X.shape[1]) as g:
        b, se_g, st_g = g.solve_block_f64(X.astype(np.float64))
    e = compare(b, se_g, st_g, r, se, st)
    assert e["b_norm"] <= TOL64 and e["se_rel"] <= TOL64, e


def test_int8_dosages_parity_and_factor(small_study):
    s, X, L, (r, se, st) = small_study
    with gw.GLS(s["Phi"], s["XL"], s["y"], s["h"], s["sigma2"], bs=1024) as g:
        Lg = g.factor()
        outs = [g.solve_block(X[:, c0:c0 + 1024]) for c0 in range(0, X.shape[1], 1024)]
    np.testing.assert_allclose(Lg, L, rtol=0, atol=1e-12 * np.abs(L).max())
    b = np.concatenate([o[0] for o in outs], axis=1)
    se_g = np.concatenate([o[1] for o in outs], axis=1)
    st_g = np.concatenate([o[2] for o in outs])
    e = compare(b, se_g, st_g, r, se, st)
    assert e["b_norm"] <= TOL64 and e["se_rel"] <= TOL64, e


@pytest.mark.parametrize("n,p,m", [(1, 1, 3), (5, 2, 1), (127, 4, 63), (129, 4, 65), (300, 7, 300),
                                   (257, 1, 129), (640, 16, 70)])
def test_ragged_shapes(n, p, m):
    s, X, L, (r, se, st) = _case(n, p, max(2 * n, 4), 0.5, sigma2=1.3, m=m)
    with gw.GLS(s["Phi"], s["XL"] if p > 1 else None, s["y"], 0.5, 1.3, bs=max(m, 1)) as g:
        b, se_g, st_g = g.solve_block(X)
    e = compare(b, se_g, st_g, r, se, st)
    assert e["b_norm"] <= TOL64 and e["se_rel"] <= TOL64, e


def test_given_factor_matches(small_study):
    s, X, L, (r, se, st) = small_study
    with gw.GLS(L, s["XL"], s["y"], s["h"], s["sigma2"], is_L=True, bs=512) as g:
        b, se_g, st_g = g.solve_block(X[:, :512])
    e = compare(b, se_g, st_g, r[:, :512], se[:, :512], st[:512])
    assert e["b_norm"] <= TOL64 and e["se_rel"] <= TOL64, e


def test_singular_and_degenerate_snps():
    s, X, L, _ = _case(200, 4, 400, 0.6, m=6)
    X[:, 1] = 2          # monomorphic: collinear with the intercept
    X[:, 2] = 0          # all zero
    X[:, 3] = 2
    X[17, 3] = 1         # one sample differs: a valid design
    r, se, _, st = oracle.gls(L, s["XL"], s["y"], X)
    assert st.tolist() == [0, 1, 1, 0, 0, 0]
    with gw.GLS(s["Phi"], s["XL"], s["y"], 0.6, 1.0, bs=16) as g:
        b, se_g, st_g = g.solve_block(X)
    e = compare(b, se_g, st_g, r, se, st)
    assert e["b_norm"] <= TOL64, e


def test_h0_and_h1_edges():
    for h in (0.0, 1.0):
        s, X, L, (r, se, st) = _case(300, 4, 600, h, m=50)
        with gw.GLS(s["Phi"], s["XL"], s["y"], h, 1.0, bs=64) as g:
            b, se_g, st_g = g.solve_block(X)
        e = compare(b, se_g, st_g, r, se, st)
        assert e["b_norm"] <= TOL64 and e["se_rel"] <= TOL64, (h, e)


def test_not_spd_and_bad_arguments():
    n = 200
    Phi = np.eye(n)
    Phi[150, 150] = -5.0   # M_150,150 = 0.5 * -5 + 0.5 < 0
    with pytest.raises(gw.NotSPDError) as e:
        gw.GLS(Phi, np.ones((n, 1)), np.ones(n), 0.5)
    assert e.value.index == 150
    XL = np.column_stack([np.ones(n), 2 * np.ones(n)])  # collinear covariates
    with pytest.raises(gw.NotSPDError):
        gw.GLS(np.eye(n), XL, np.ones(n), 0.5)
    with pytest.raises(gw.GwasError) as e:
        gw.GLS(np.eye(n), np.ones((n, 1)), np.ones(n), 1.5)
    assert e.value.name == "GWAS_ERR_ARG"
    with gw.GLS(np.eye(n), np.ones((n, 1)), np.ones(n), 0.5, bs=8) as g:
        with pytest.raises(gw.GwasError) as e:
            g.solve_block(np.zeros((n, 9), dtype=np.int8))  # more columns than bs
        assert e.value.name == "GWAS_ERR_ARG"
        b, se, st = g.solve_block(np.zeros((n, 0), dtype=np.int8))
        assert b.shape == (2, 0)


def test_device_tensors_async(small_study):
    import torch
    s, X, L, (r, se, st) = small_study
    Xd = torch.from_numpy(np.ascontiguousarray(X.T)).cuda().T  # n x m, column-major on the device
    with gw.GLS(s["Phi"], s["XL"], s["y"], s["h"], s["sigma2"], bs=X.shape[1]) as g:
        b, se_g, st_g = g.solve_block(Xd)
        g.synchronize()
        e = compare(b.cpu().numpy(), se_g.cpu().numpy(), st_g.cpu().numpy(), r, se, st)
    assert e["b_norm"] <= TOL64 and e["se_rel"] <= TOL64, e


def test_stream_matches_blocks(small_study):
    s, X, L, (r, se, st) = small_study
    Xh = np.asfortranarray(X[:, :1900])
    with gw.GLS(s["Phi"], s["XL"], s["y"], s["h"], s["sigma2"], bs=256, ring_depth=3) as g:
        b, se_g, st_g = g.solve_stream(Xh)
    e = compare(b, se_g, st_g, r[:, :1900], se[:, :1900], st[:1900])
    assert e["b_norm"] <= TOL64 and e["se_rel"] <= TOL64, e


@pytest.mark.parametrize("prec", ("fp64", "f16x2", "sliced64"))
def test_stream_packed_input(small_study, prec):
    """gwas_solve_stream_packed: the same columns held 2-bit packed in host
    memory give bit for bit gwas_solve_stream's results while the link carries
    ceil(n/4) bytes per SNP; a packed leading dimension that is not a multiple
    of 16 (ldp = ceil(n/4) + 3) goes through the pitched copy."""
    s, X, L, (r, se, st) = small_study
    n, m, bs = X.shape[0], 1100, 256
    Xh = np.asfortranarray(X[:, :m].astype(np.int8))
    P = gw.pack_dosages2(Xh)
    nb = (n + 3) // 4
    Pw = np.zeros((nb + 3, m), dtype=np.uint8, order="F")
    Pw[:nb] = P
    with gw.GLS(s["Phi"], s["XL"], s["y"], s["h"], s["sigma2"], precision=prec, bs=bs, stream_pack=0) as g:
        ref = g.solve_stream(Xh)  # int8 over the link
        h0 = g.h2d_bytes
        out = g.solve_stream_packed(P)
        moved = g.h2d_bytes - h0
        out_w = g.solve_stream_packed(Pw)
    assert moved == nb * m, moved
    for a_, b_ in zip(ref, out):
        assert np.array_equal(a_, b_, equal_nan=True)
    for a_, b_ in zip(ref, out_w):
        assert np.array_equal(a_, b_, equal_nan=True)
    tol = TOL64 if prec in ("fp64", "sliced64") else 1e-5
    e = compare(*out, r[:, :m], se[:, :m], st[:m])
    assert e["b_norm"] <= tol and e["se_rel"] <= tol, e


@pytest.mark.parametrize("prec", ("fp64", "f16x2", "bf16x3", "sliced64"))
def test_stream_packed_ragged_rows_and_padding_bits(prec):
    """n = 301 (the last packed byte holds one row): packed columns whose
    padding bits are set (rows past n) give the int8 stream's results bit for
    bit -- the split inverse form reads the codes in its cast, the other
    precisions unpack them; rows past n count as 0 either way."""
    n, m = 301, 300
    s = gwas_synth.study(n, 4, 600, 0.6, 1.0, seed=9)
    X = np.asfortranarray(gwas_synth.dosages(n, 0, m, seed=9))
    P = gw.pack_dosages2(X)
    P[-1, :] |= 0xFC  # rows 301..303 of the last byte: garbage
    with gw.GLS(s["Phi"], s["XL"], s["y"], 0.6, 1.0, precision=prec, bs=128, stream_pack=0) as g:
        ref = g.solve_stream(X)
        out = g.solve_stream_packed(P)
    for a_, b_ in zip(ref, out):
        assert np.array_equal(a_, b_, equal_nan=True)


# ---------------------------------------------------------------- split precision
TOL_SPLIT = 1e-5
SPLITS = ("bf16x3", "tf32x3", "f16x2")
# how the tensor-core solve's tiles map onto SMs: one per SM, row-panel pairs on
# a 2-SM cluster with shared loads, row-panel pairs as one 256-row product (the
# substitution), and the product with L^-1 formed at set-up
TILES = ("single", "pair_mma", "inverse")
# f16x2 exists in the inverse form only
SPLIT_TILES = [(p, t) for p in SPLITS for t in TILES if p != "f16x2" or t == "inverse"]
FULL_CASES = [("fp64", "auto"), ("sliced64", "auto")] + [(p, t) for p in SPLITS for t in ("auto",) + TILES
                                                          if p != "f16x2" or t in ("auto", "inverse")]


@pytest.mark.parametrize("prec,tiles,ring", [("fp64", "auto", 3), ("f16x2", "auto", 3), ("bf16x3", "auto", 3),
                                             ("bf16x3", "pair_mma", 3), ("sliced64", "auto", 3),
                                             ("f16x2", "auto", 2)])
def test_stream_host_packing(prec, tiles, ring):
    """gwas_solve_stream with stream_pack = 1: int8 host blocks whose values lie
    in 0..3 are packed by the host threads and cross the link as 2-bit codes
    (the split inverse form reads them in its cast, the others unpack them);
    a block holding another value crosses as int8.  Results bit for bit those
    of the int8 transport; the link's bytes counted per block."""
    n, bs = 1001, 256
    m = 3 * bs + 77  # four blocks, the last ragged
    s = gwas_synth.study(n, 4, 2 * n, 0.6, 1.0, seed=21)
    X = np.asfortranarray(gwas_synth.dosages(n, 0, m, seed=21))
    X[5, 300] = 3    # block 1: still packable
    X[9, 600] = 5    # block 2: int8
    nb, ldp = (n + 3) // 4, ((n + 3) // 4 + 15) // 16 * 16
    outs, moved = {}, {}
    for mode in (0, 1):
        with gw.GLS(s["Phi"], s["XL"], s["y"], 0.6, 1.0, precision=prec, bs=bs, tiles=tiles,
                    ring_depth=ring, stream_pack=mode) as g:
            h0 = g.h2d_bytes
            outs[mode] = g.solve_stream(X)
            moved[mode] = g.h2d_bytes - h0
            again = g.solve_stream(X)  # the pool and slots reused
            for a_, b_ in zip(outs[mode], again):
                assert np.array_equal(a_, b_, equal_nan=True)
    for a_, b_ in zip(outs[0], outs[1]):
        assert np.array_equal(a_, b_, equal_nan=True)
    assert moved[0] == n * m
    assert moved[1] == ldp * (2 * bs + 77) + n * bs  # blocks 0, 1, 3 packed; block 2 as int8


@pytest.mark.parametrize("prec,tiles", SPLIT_TILES)
def test_split_precision_parity(small_study, prec, tiles):
    s, X, L, (r, se, st) = small_study
    with gw.GLS(s["Phi"], s["XL"], s["y"], s["h"], s["sigma2"], precision=prec, bs=1024, tiles=tiles) as g:
        ctas, cluster, mode = g.solve_shape()
        assert mode == tiles and cluster == (1 if tiles == "single" else 2) and 0 < ctas <= 148
        outs = [g.solve_block(X[:, c0:c0 + 1024]) for c0 in range(0, X.shape[1], 1024)]
    b = np.concatenate([o[0] for o in outs], axis=1)
    se_g = np.concatenate([o[1] for o in outs], axis=1)
    st_g = np.concatenate([o[2] for o in outs])
    e = compare(b, se_g, st_g, r, se, st)
    print(prec, e)
    assert e["b_norm"] <= TOL_SPLIT and e["se_rel"] <= TOL_SPLIT, e


@pytest.mark.parametrize("prec,tiles", SPLIT_TILES)
@pytest.mark.parametrize("n,p,m", [(1, 1, 3), (127, 4, 63), (129, 2, 257), (300, 7, 300), (1000, 4, 513),
                                   (1200, 3, 300)])
def test_split_ragged_shapes(prec, tiles, n, p, m):
    # n = 1..129: one or two row panels (a pair with and without its second
    # panel); n = 300, 1000, 1200: 3, 8 and 10 panels, odd and even counts
    s, X, L, (r, se, st) = _case(n, p, max(2 * n, 4), 0.5, sigma2=1.3, m=m)
    with gw.GLS(s["Phi"], s["XL"] if p > 1 else None, s["y"], 0.5, 1.3, precision=prec, bs=max(m, 1),
                tiles=tiles) as g:
        b, se_g, st_g = g.solve_block(X)
    e = compare(b, se_g, st_g, r, se, st)
    assert e["b_norm"] <= TOL_SPLIT and e["se_rel"] <= TOL_SPLIT, (prec, tiles, e)


@pytest.mark.parametrize("prec,tiles", SPLIT_TILES)
def test_split_grouped_tile_order(small_study, prec, tiles):
    """Tiles handed out over groups of 2 column strips (a device order table; in
    the pair modes its rows are row-panel pairs): same parity."""
    s, X, L, (r, se, st) = small_study
    with gw.GLS(s["Phi"], s["XL"], s["y"], s["h"], s["sigma2"], precision=prec, bs=1024, tiles=tiles,
                strip_group=2) as g:
        b, se_g, st_g = g.solve_block(X[:, :1000])
    e = compare(b, se_g, st_g, r[:, :1000], se[:, :1000], st[:1000])
    assert e["b_norm"] <= TOL_SPLIT and e["se_rel"] <= TOL_SPLIT, (prec, tiles, e)


@pytest.mark.parametrize("prec", SPLITS)
@pytest.mark.parametrize("sigma2", (1e-6, 1e4))
def test_split_extreme_sigma2(prec, sigma2):
    """L^-1 scales as sigma2^-1/2 (entries ~1e3 and ~1e-2 here): the FP16 pieces
    of f16x2 keep their precision through the per-row power-of-two scaling
    (unscaled, 1e-2-sized entries would put the lo pieces among FP16's
    subnormals); b does not depend on sigma2, se scales with its square root.
    (At sigma2 = 1e6 the noise-dominated fit amplifies the operand error:
    BF16x3 reaches 8e-6 normwise there, TF32x3 and F16x2 5e-7.)"""
    s, X, L, (r, se, st) = _case(640, 4, 1280, 0.5, sigma2=sigma2, m=300)
    with gw.GLS(s["Phi"], s["XL"], s["y"], 0.5, sigma2, precision=prec, bs=300) as g:
        b, se_g, st_g = g.solve_block(X)
    e = compare(b, se_g, st_g, r, se, st)
    print(prec, sigma2, e)
    assert e["b_norm"] <= TOL_SPLIT and e["se_rel"] <= TOL_SPLIT, (prec, sigma2, e)


def _phenotypes(s, t, seed=5):
    """t phenotype columns: the study's y, then y shifted and mixed with independent noise."""
    rng = np.random.default_rng(seed)
    cols = [s["y"]] + [0.5 * s["y"] + 0.3 * k + rng.standard_normal(s["n"]) for k in range(1, t)]
    return np.asfortranarray(np.column_stack(cols))


@pytest.mark.parametrize("prec", ("fp64", "sliced64") + SPLITS)
@pytest.mark.parametrize("n,p,m,t", [(640, 4, 300, 5), (300, 2, 130, 3), (257, 6, 65, 11)])
def test_several_phenotypes(prec, n, p, m, t):
    """t phenotypes sharing one study: b of each equals its own single-phenotype
    GLS (the oracle run per column of Y); se and status are shared."""
    s, X, L, _ = _case(n, p, 2 * n, 0.5, m=m)
    Y = _phenotypes(s, t)
    tol = TOL64 if prec in ("fp64", "sliced64") else TOL_SPLIT
    with gw.GLS(s["Phi"], s["XL"] if p > 1 else None, Y, 0.5, 1.0, precision=prec, bs=m) as g:
        b, se_g, st_g = g.solve_block(X)
        b_s, se_s, st_s = g.solve_stream(np.asfortranarray(X))
    assert b.shape == (p, m, t)
    assert np.array_equal(b, b_s) and np.array_equal(se_g, se_s) and np.array_equal(st_g, st_s)
    for k in range(t):
        r, se, _, st = oracle.gls(L, s["XL"], Y[:, k], X)
        e = compare(b[:, :, k], se_g, st_g, r, se, st)
        assert e["b_norm"] <= tol and e["se_rel"] <= tol, (prec, k, e)


@pytest.mark.parametrize("prec", SPLITS)
@pytest.mark.parametrize("n,p,m,t", [(1000, 4, 1000, 1), (300, 2, 257, 3), (640, 4, 300, 5), (129, 2, 65, 1)])
def test_fused_and_separate_sums(prec, n, p, m, t):
    """Inverse form: the per-SNP sums formed in the solve's epilogue (the
    default; one plane per row panel when p - 1 + t <= 4, per row quarter up to
    8) against the separate pass over a stored X~: both at the oracle's bar, and
    equal to each other up to summation order.  A block solved for the adjoint
    (which stores X~) in between leaves the next block's fused sums intact."""
    s, X, L, _ = _case(n, p, 2 * n, 0.5, sigma2=1.3, m=m)
    Y = _phenotypes(s, t) if t > 1 else s["y"]
    XL = s["XL"] if p > 1 else None
    out = {}
    for sep in (False, True):
        with gw.GLS(s["Phi"], XL, Y, 0.5, 1.3, precision=prec, bs=m, tiles="inverse", separate_sums=sep) as g:
            out[sep] = g.solve_block(X)
            if t == 1 and p > 1:
                g.adjoint_block(X[:, : m // 2])
                again = g.solve_block(X)
                assert all(np.array_equal(a, c) for a, c in zip(out[sep], again))
    for k in range(t):
        yk = Y[:, k] if t > 1 else Y
        r, se, _, st = oracle.gls(L, s["XL"], yk, X)
        for sep in (False, True):
            b = out[sep][0][:, :, k] if t > 1 else out[sep][0]
            e = compare(b, out[sep][1], out[sep][2], r, se, st)
            assert e["b_norm"] <= TOL_SPLIT and e["se_rel"] <= TOL_SPLIT, (prec, sep, k, e)
    assert np.array_equal(out[False][2], out[True][2])
    ok = out[True][2] == 0
    assert np.allclose(out[False][1][:, ok], out[True][1][:, ok], rtol=1e-6, atol=0)


def test_several_phenotypes_device_outputs_and_limits():
    import torch
    s, X, L, _ = _case(300, 4, 600, 0.5, m=64)
    Y = _phenotypes(s, 4)
    with gw.GLS(s["Phi"], s["XL"], Y, 0.5, 1.0, precision="f16x2", bs=64) as g:
        Xd = torch.from_numpy(np.ascontiguousarray(X.T)).cuda().T
        b, se_g, st_g = g.solve_block(Xd)
        g.synchronize()
        assert tuple(b.shape) == (4, 64, 4) and b.is_cuda
        b_h, se_h, st_h = g.solve_block(X)
        assert np.array_equal(b.cpu().numpy(), b_h)
        with pytest.raises(gw.GwasError) as e:
            g.adjoint_block(X)
        assert e.value.name == "GWAS_ERR_UNSUPPORTED"
    with pytest.raises(gw.GwasError):  # q + t > 16 columns
        gw.GLS(s["Phi"], s["XL"], _phenotypes(s, 14), 0.5, 1.0, bs=64)


@pytest.mark.parametrize("tiles", ("single", "pair_mma"))
def test_f16x2_needs_the_inverse_form(small_study, tiles):
    s, *_ = small_study
    with pytest.raises(gw.GwasError):
        gw.GLS(s["Phi"], s["XL"], s["y"], s["h"], s["sigma2"], precision="f16x2", bs=256, tiles=tiles)


@pytest.mark.parametrize("prec", SPLITS)
def test_split_unaligned_device_input(prec):
    import torch
    s, X, L, (r, se, st) = _case(200, 4, 400, 0.6, m=40)
    # device input with a leading dimension that is not a multiple of 16
    buf = torch.zeros((40, 203), dtype=torch.int8, device="cuda")
    buf[:, :200] = torch.from_numpy(np.ascontiguousarray(X.T)).cuda()
    Xd = buf.T[:200]
    assert Xd.stride(1) == 203
    with gw.GLS(s["Phi"], s["XL"], s["y"], 0.6, 1.0, precision=prec, bs=64) as g:
        b, se_g, st_g = g.solve_block(Xd)
        g.synchronize()
    e = compare(b.cpu().numpy(), se_g.cpu().numpy(), st_g.cpu().numpy(), r, se, st)
    assert e["b_norm"] <= TOL_SPLIT and e["se_rel"] <= TOL_SPLIT, e


@pytest.mark.parametrize("prec", SPLITS)
def test_split_singular_and_near_singular(prec):
    """A monomorphic SNP is flagged; a SNP with one deviating sample is a valid
    but ill-conditioned design (S_BR / d^2 ~ 4n): its b is checked against the
    oracle in units of the oracle's standard error."""
    s, X, L, _ = _case(200, 4, 400, 0.6, m=6)
    X[:, 1] = 2
    X[:, 3] = 2
    X[17, 3] = 1
    r, se, _, st = oracle.gls(L, s["XL"], s["y"], X)
    with gw.GLS(s["Phi"], s["XL"], s["y"], 0.6, 1.0, precision=prec, bs=64) as g:
        b, se_g, st_g = g.solve_block(X)
    assert st_g.tolist() == st.tolist() == [0, 1, 0, 0, 0, 0]
    assert np.isnan(b[:, 1]).all()
    well = [0, 2, 4, 5]
    e = compare(b[:, well], se_g[:, well], st_g[well], r[:, well], se[:, well], st[well])
    assert e["b_norm"] <= TOL_SPLIT and e["se_rel"] <= TOL_SPLIT, e
    e3 = compare(b[:, [3]], se_g[:, [3]], st_g[[3]], r[:, [3]], se[:, [3]], st[[3]])
    print(prec, "near-singular", e3)
    assert e3["b_se_scaled"] <= 1e-3 and e3["se_rel"] <= 1e-3, e3


@pytest.mark.parametrize("prec", SPLITS)
def test_split_stream(small_study, prec):
    s, X, L, (r, se, st) = small_study
    with gw.GLS(s["Phi"], s["XL"], s["y"], s["h"], s["sigma2"], precision=prec, bs=512, ring_depth=3) as g:
        b, se_g, st_g = g.solve_stream(np.asfortranarray(X[:, :1800]))
    e = compare(b, se_g, st_g, r[:, :1800], se[:, :1800], st[:1800])
    assert e["b_norm"] <= TOL_SPLIT and e["se_rel"] <= TOL_SPLIT, e


# ------------------------------------------------------- full size (n = 10,000)
@pytest.fixture(scope="module")
def paper_scale():
    """The paper-scale workload: n = 10,000, p = 4, h = 0.5, kinship from k = 5,000
    genotypes, m = 1,000,000 SNPs in blocks of 4,096 (the last block holds 576)."""
    w = gwas_synth.WORKLOADS["n10k_p4_m1M_int8"]
    s = gwas_synth.study(w["n"], w["p"], w["k"], w["h"], w["sigma2"])
    L = oracle.potrf(oracle.form_m(s["Phi"], w["h"], w["sigma2"]))
    first = gwas_synth.dosages(w["n"], 0, w["bs"])
    last0 = (w["m"] // w["bs"]) * w["bs"]
    last = gwas_synth.dosages(w["n"], last0, w["m"])
    rng = np.random.default_rng(7)
    pick_first = np.sort(rng.choice(w["bs"], 48, replace=False))
    pick_last = np.r_[0, np.sort(rng.choice(np.arange(1, last.shape[1] - 1), 14, replace=False)), last.shape[1] - 1]
    ref_first = oracle.gls(L, s["XL"], s["y"], first[:, pick_first])
    ref_last = oracle.gls(L, s["XL"], s["y"], last[:, pick_last])
    return w, s, first, last, pick_first, pick_last, ref_first, ref_last


@pytest.fixture(scope="module")
def paper_scale_sample(paper_scale):
    """2,000 SNPs of the m = 1,000,000 drawn by seed across the whole range:
    16 from each of 125 generator chunks (256 columns) picked by seed, so each
    column is regenerated alone; oracle results for all of them."""
    w, s, *_ = paper_scale
    rng = np.random.default_rng(20130218)
    nchunks = w["m"] // gwas_synth.CHUNK
    chunks = np.sort(rng.choice(nchunks, 125, replace=False))
    cols = []
    for ch in chunks:
        c0 = int(ch) * gwas_synth.CHUNK
        blk = gwas_synth.dosages(w["n"], c0, c0 + gwas_synth.CHUNK)
        pick = np.sort(rng.choice(gwas_synth.CHUNK, 16, replace=False))
        cols.append(blk[:, pick])
    Xs = np.asfortranarray(np.concatenate(cols, axis=1))
    L = oracle.potrf(oracle.form_m(s["Phi"], w["h"], w["sigma2"]))
    ref = oracle.gls(L, s["XL"], s["y"], Xs)
    return Xs, ref


@pytest.mark.parametrize("prec,tiles", FULL_CASES)
def test_full_size_seeded_sample(paper_scale, paper_scale_sample, prec, tiles):
    """The 2,000 sampled SNPs solved as one block, every one against the oracle."""
    import torch
    w, s, *_ = paper_scale
    Xs, (r, se, _, st) = paper_scale_sample
    tb, ts = FULL_TOL[prec]
    with gw.GLS(s["Phi"], s["XL"], s["y"], w["h"], w["sigma2"], precision=prec, bs=w["bs"], tiles=tiles) as g:
        Xd = torch.from_numpy(np.ascontiguousarray(Xs.T)).cuda().T
        b, se_g, st_g = g.solve_block(Xd)
        g.synchronize()
        b, se_g, st_g = b.cpu().numpy(), se_g.cpu().numpy(), st_g.cpu().numpy()
    e = compare(b, se_g, st_g, r, se, st)
    print(prec, tiles, "sample", e)
    assert e["b_norm"] <= tb and e["se_rel"] <= ts, (prec, tiles, e)
    if prec != "fp64":
        # stricter extra: component by component on components with |b_j| >= se_j.
        # BF16x3 operands carry ~17 bits (hi + lo of 8 each): the dropped lo*lo term
        # and the representation residual are each ~2^-18, and the worst component
        # of the 2,000 SNPs sits at ~1.1e-5; TF32x3 (~22 bits) stays near 2e-6; F16x2's
        # pieces carry ~22 bits as well
        assert e["b_comp_max"] <= COMP_TOL[prec], (prec, tiles, e)


# b: per-SNP normwise relative error (the stated bar: 1e-10 FP64, 1e-5 split);
# se: component-wise relative error, same bars.
FULL_TOL = {"fp64": (1e-10, 1e-10), "sliced64": (1e-10, 1e-10), "bf16x3": (1e-5, 1e-5), "tf32x3": (1e-5, 1e-5),
            "f16x2": (1e-5, 1e-5)}
# the sliced path carries the FP64 bar component by component too
COMP_TOL = {"sliced64": 1e-10, "bf16x3": 2e-5, "tf32x3": 1e-5, "f16x2": 1e-5}


@pytest.mark.parametrize("prec,tiles", FULL_CASES)
def test_full_size_sampled(paper_scale, prec, tiles):
    import torch
    w, s, first, last, pf, pl, ref_first, ref_last = paper_scale
    tb, ts = FULL_TOL[prec]
    with gw.GLS(s["Phi"], s["XL"], s["y"], w["h"], w["sigma2"], precision=prec, bs=w["bs"], tiles=tiles) as g:
        for X, pick, (r, se, _, st) in ((first, pf, ref_first), (last, pl, ref_last)):
            Xd = torch.from_numpy(np.ascontiguousarray(X.T)).cuda().T
            b, se_g, st_g = g.solve_block(Xd)
            g.synchronize()
            b, se_g, st_g = b.cpu().numpy()[:, pick], se_g.cpu().numpy()[:, pick], st_g.cpu().numpy()[pick]
            e = compare(b, se_g, st_g, r, se, st)
            print(prec, X.shape[1], e)
            assert e["b_norm"] <= tb and e["se_rel"] <= ts, (prec, e)
            if prec != "fp64":  # significant components, one by one (see COMP_TOL)
                assert e["b_comp_max"] <= COMP_TOL[prec], (prec, e)


@pytest.mark.parametrize("prec", ("fp64", "f16x2"))
def test_stage_timing(small_study, prec):
    """Per-stage CUDA-event timers: the solve kernel's launches are timed on
    their own (inside the trsm stage, which also holds the split pre-pass)."""
    s, X, L, _ = small_study
    with gw.GLS(s["Phi"], s["XL"], s["y"], s["h"], s["sigma2"], precision=prec, bs=512) as g:
        g.timing(True)
        for c0 in (0, 512):
            g.solve_block(X[:, c0:c0 + 512])
        st = g.timing_read()
        g.timing(False)
    assert set(st) == {"h2d", "trsm", "reduce", "d2h", "solve"}
    assert st["trsm"][1] == st["solve"][1] == st["reduce"][1] == 2
    assert 0.0 < st["solve"][0] <= st["trsm"][0] and st["reduce"][0] > 0.0


@pytest.mark.parametrize("prec", SPLITS)
def test_single_piece_study_switch(small_study, prec):
    """The precision-study switch keeps L^-1 as its hi piece alone: results
    stay finite with the same statuses, their error against the oracle grows
    by orders of magnitude over the split pair's, and the switch is refused
    outside the inverse form."""
    s, X, L, (r, se, st) = small_study
    Xs = X[:, :256]
    e = {}
    for single in (False, True):
        with gw.GLS(s["Phi"], s["XL"], s["y"], s["h"], s["sigma2"], precision=prec, bs=256,
                    single_piece=single) as g:
            b, se_g, st_g = g.solve_block(Xs)
        assert np.array_equal(st_g, st[:256]) and np.all(np.isfinite(b[:, st_g == 0]))
        e[single] = compare(b, se_g, st_g, r[:, :256], se[:, :256], st[:256])
    assert e[False]["b_norm"] <= TOL_SPLIT
    assert e[True]["b_norm"] > 10 * e[False]["b_norm"], e
    for bad in (dict(precision="fp64"), dict(precision=prec, tiles="pair_mma")):
        if bad.get("tiles") and prec == "f16x2":
            continue
        with pytest.raises(gw.GwasError):
            gw.GLS(s["Phi"], s["XL"], s["y"], s["h"], s["sigma2"], bs=256, single_piece=True, **bad)
