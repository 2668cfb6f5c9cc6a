"""The batching form: studies of uneven n in one persistent launch (CUDA
graph), against each study solved alone and against the FP64 oracle."""
import numpy as np
import pytest

import gwas_synth
import oracle
import paper_1302_4332_b300 as gw
from oracle.metrics import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1302_4332_b300 import build
    build.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


NS = (300, 700, 129, 1000)  # uneven study sizes, one of them a single ragged panel + 1


def _studies(prec, bs=512, tiles="auto"):
    out = []
    for i, n in enumerate(NS):
        s = gwas_synth.study(n, 4, 2 * n, 0.5, 1.0, seed=30, study_id=i)
        out.append((s, gw.GLS(s["Phi"], s["XL"], s["y"], 0.5, 1.0, precision=prec, bs=bs, tiles=tiles)))
    return out


@pytest.mark.parametrize("prec,tiles", [("bf16x3", "auto"), ("bf16x3", "pair_mma"), ("tf32x3", "auto"),
                                        ("tf32x3", "pair_mma"), ("f16x2", "auto")])
def test_batch_matches_single_and_oracle(prec, tiles):
    studies = _studies(prec, tiles=tiles)
    gls = [g for _, g in studies]
    try:
        with gw.GLSBatch(gls) as B:
            for rep, c0 in enumerate((0, 512)):  # two steps: the captured graph replays with new data
                blocks = [gwas_synth.dosages(s["n"], c0, c0 + m, seed=30, study=i)
                          for i, ((s, _), m) in enumerate(zip(studies, (512, 300, 64, 511)))]
                outs = B.solve(blocks)
                for i, ((s, g), X, (b, se, st)) in enumerate(zip(studies, blocks, outs)):
                    b1, se1, st1 = g.solve_block(X)
                    np.testing.assert_array_equal(st, st1)
                    assert np.array_equal(b, b1) and np.array_equal(se, se1), (prec, i, rep)
                    L = oracle.potrf(oracle.form_m(s["Phi"], 0.5, 1.0))
                    pick = np.arange(0, X.shape[1], 17)
                    r, se_o, _, st_o = oracle.gls(L, s["XL"], s["y"], X[:, pick])
                    e = compare(b[:, pick], se[:, pick], st[pick], r, se_o, st_o)
                    assert e["b_norm"] <= 1e-5 and e["se_rel"] <= 1e-5, (prec, tiles, i, e)
            # study-after-study order: the same results
            B.set_order(1)
            outs2 = B.solve(blocks)
            for (b, se, st), (b2, se2, st2) in zip(outs, outs2):
                assert np.array_equal(b, b2) and np.array_equal(st, st2)
    finally:
        for g in gls:
            g.close()


@pytest.mark.parametrize("prec", ("bf16x3", "f16x2"))
def test_batch_studies_of_different_p(prec):
    """Studies with p = 2, 4, 6, 8 in one launch: their per-SNP sums take both
    widths of W in the solve's epilogue (4 and 8 columns; per row panel or per
    row quarter) side by side.  Each equals its own context's block solve bit
    for bit and the oracle within the split bar."""
    ps, ns = (2, 4, 6, 8), (300, 520, 129, 700)
    studies = []
    for i, (n, p) in enumerate(zip(ns, ps)):
        s = gwas_synth.study(n, p, 2 * n, 0.5, 1.0, seed=31, study_id=i)
        studies.append((s, gw.GLS(s["Phi"], s["XL"], s["y"], 0.5, 1.0, precision=prec, bs=256)))
    gls = [g for _, g in studies]
    try:
        with gw.GLSBatch(gls) as B:
            blocks = [gwas_synth.dosages(s["n"], 0, m, seed=31, study=i)
                      for i, ((s, _), m) in enumerate(zip(studies, (256, 200, 97, 256)))]
            outs = B.solve(blocks)
            for i, ((s, g), X, (b, se, st)) in enumerate(zip(studies, blocks, outs)):
                assert b.shape == (ps[i], X.shape[1])
                b1, se1, st1 = g.solve_block(X)
                assert np.array_equal(b, b1) and np.array_equal(se, se1) and np.array_equal(st, st1), (prec, i)
                L = oracle.potrf(oracle.form_m(s["Phi"], 0.5, 1.0))
                r, se_o, _, st_o = oracle.gls(L, s["XL"], s["y"], X)
                e = compare(b, se, st, r, se_o, st_o)
                assert e["b_norm"] <= 1e-5 and e["se_rel"] <= 1e-5, (prec, i, e)
    finally:
        for g in gls:
            g.close()


@pytest.mark.parametrize("prec,tiles", [("bf16x3", "auto"), ("tf32x3", "pair_mma"), ("f16x2", "auto")])
def test_batch_autotune_then_oracle_and_skipped_study(prec, tiles):
    """The autotuner tries columns, tile mode (inverse form / pair product,
    except for FP16 pieces), stages and orders on seeded dosages; solves
    after it, in whatever configuration it kept, still meet the oracle."""
    studies = _studies(prec, bs=1024, tiles=tiles)
    gls = [g for _, g in studies]
    try:
        with gw.GLSBatch(gls) as B:
            t = B.autotune_ex(reps=2)
            assert t["cols"] in (512, 1024) and t["snps_per_s"] > 0 and t["stages"] in (6, 8)
            assert t["tile_mode"] in (("inverse",) if prec == "f16x2" else ("inverse", "pair_mma"))
            blocks = [gwas_synth.dosages(s["n"], 1024, 1024 + m, seed=30, study=i)
                      for i, ((s, _), m) in enumerate(zip(studies, (t["cols"], 300, 64, 511)))]
            outs = B.solve(blocks)
            for i, ((s, g), X, (b, se, st)) in enumerate(zip(studies, blocks, outs)):
                L = oracle.potrf(oracle.form_m(s["Phi"], 0.5, 1.0))
                pick = np.arange(0, X.shape[1], 13)
                r, se_o, _, st_o = oracle.gls(L, s["XL"], s["y"], X[:, pick])
                e = compare(b[:, pick], se[:, pick], st[pick], r, se_o, st_o)
                assert e["b_norm"] <= 1e-5 and e["se_rel"] <= 1e-5, (prec, t, i, e)
            s0, g0 = studies[0]
            X = blocks[0]
            outs = B.solve([X, None, None, None])
            assert outs[1] is None
            b1, se1, st1 = g0.solve_block(X)
            if t["tile_mode"] == (g0.solve_shape()[2]):  # the same kernels as the study's own solve
                assert np.array_equal(outs[0][0], b1)
    finally:
        for g in gls:
            g.close()


@pytest.mark.parametrize("prec", ("bf16x3", "f16x2"))
def test_batch_k_blocks_per_replay(prec):
    """Three blocks of every study through one graph replay (three batched
    launches captured together): each block equals the one-block batch solve
    bit for bit, and the oracle on a sample; a later call with other column
    counts re-captures."""
    studies = _studies(prec, bs=512)
    gls = [g for _, g in studies]
    Ls = [oracle.potrf(oracle.form_m(s["Phi"], 0.5, 1.0)) for s, _ in studies]
    try:
        with gw.GLSBatch(gls) as B:
            for ms in ((512, 300, 64, 511), (100, 512, 129, 7)):
                steps = [[gwas_synth.dosages(s["n"], 512 * j, 512 * j + m, seed=32, study=i)
                          for i, ((s, _), m) in enumerate(zip(studies, ms))] for j in range(3)]
                outs = B.solve_k(steps)
                assert len(outs) == 3
                for j in range(3):
                    one = B.solve(steps[j])
                    for i, ((s, g), X) in enumerate(zip(studies, steps[j])):
                        b, se, st = outs[j][i]
                        assert np.array_equal(b, one[i][0]) and np.array_equal(se, one[i][1]), (j, i)
                        assert np.array_equal(st, one[i][2])
                        pick = np.r_[0, np.arange(1, X.shape[1], 29), X.shape[1] - 1]
                        r, se_o, _, st_o = oracle.gls(Ls[i], s["XL"], s["y"], X[:, pick])
                        e = compare(b[:, pick], se[:, pick], st[pick], r, se_o, st_o)
                        assert e["b_norm"] <= 1e-5 and e["se_rel"] <= 1e-5, (prec, j, i, e)
    finally:
        for g in gls:
            g.close()


def test_batch_takes_one_phenotype_per_study():
    s = gwas_synth.study(300, 4, 600, 0.5, 1.0, seed=30)
    Y = np.asfortranarray(np.column_stack([s["y"], s["y"]]))
    with gw.GLS(s["Phi"], s["XL"], Y, 0.5, 1.0, precision="bf16x3", bs=256) as g:
        with pytest.raises(gw.GwasError) as e:
            gw.GLSBatch([g])
        assert e.value.name == "GWAS_ERR_UNSUPPORTED"


def test_batch_solve_files_matches_in_memory(tmp_path):
    """Out of core: each study's dosages in its own file (own leading dimension
    and header); the streamed batch equals the in-memory batch step by step and
    the oracle on a sample; a study that runs out of columns drops out."""
    studies = _studies("bf16x3")
    gls = [g for _, g in studies]
    cols, ms = 256, (700, 1000, 300, 513)
    paths, lds, heads, Xs = [], [], [], []
    for i, ((s, _), m) in enumerate(zip(studies, ms)):
        X = gwas_synth.dosages(s["n"], 0, m, seed=31, study=i)
        ld, head = s["n"] + 5 + i, 16 * i
        raw = np.zeros((m, ld), dtype=np.int8)
        raw[:, :s["n"]] = X.T
        path = tmp_path / f"study{i}.bin"
        with open(path, "wb") as f:
            f.write(b"\x55" * head)
            f.write(raw.tobytes())
        paths.append(str(path)); lds.append(ld); heads.append(head); Xs.append(X)
    try:
        with gw.GLSBatch(gls) as B:
            outs = B.solve_files(paths, ms, cols, ldx=lds, header_bytes=heads)
            nsteps = max((m + cols - 1) // cols for m in ms)
            for k in range(nsteps):
                blocks = [X[:, k * cols:(k + 1) * cols] if k * cols < X.shape[1] else None for X in Xs]
                ref = B.solve(blocks)
                for i, r in enumerate(ref):
                    if r is None:
                        continue
                    sl = slice(k * cols, k * cols + r[0].shape[1])
                    assert np.array_equal(outs[i][0][:, sl], r[0]) and np.array_equal(outs[i][2][sl], r[2]), (i, k)
            for i, ((s, _), X, (b, se, st)) in enumerate(zip(studies, Xs, outs)):
                L = oracle.potrf(oracle.form_m(s["Phi"], 0.5, 1.0))
                pick = np.arange(0, X.shape[1], 23)
                r, se_o, _, st_o = oracle.gls(L, s["XL"], s["y"], X[:, pick])
                e = compare(b[:, pick], se[:, pick], st[pick], r, se_o, st_o)
                assert e["b_norm"] <= 1e-5 and e["se_rel"] <= 1e-5, (i, e)
            # a file that is too short is an IO error, not a hang
            with pytest.raises(gw.GwasError) as err:
                B.solve_files(paths, [m + 300 for m in ms], cols, ldx=lds, header_bytes=heads)
            assert err.value.name == "GWAS_ERR_IO"
    finally:
        for g in gls:
            g.close()


def test_batch_solve_files_packed_equals_int8_files(tmp_path):
    """The batch over files of 2-bit packed columns (own leading dimensions and
    headers, junk in the padding bits past n): every study's results equal the
    int8 files' bit for bit and the oracle on a sample; a leading dimension
    below ceil(n/4) is refused, a short file is an IO error."""
    studies = _studies("f16x2")
    gls = [g for _, g in studies]
    cols, ms = 256, (700, 1000, 300, 513)
    p8, pp, ld8, ldp, heads, Xs = [], [], [], [], [], []
    rng = np.random.default_rng(4)
    for i, ((s, _), m) in enumerate(zip(studies, ms)):
        n = s["n"]
        X = gwas_synth.dosages(n, 0, m, seed=32, study=i)
        X[::2, 5] = 3  # the largest hard call
        X[:, 6] = 1  # a monomorphic SNP: singular, NaN outputs
        head = 8 * i + 3
        raw = np.ascontiguousarray(X.T)
        P = gw.pack_dosages2(X)  # ceil(n/4) x m
        nb = (n + 3) // 4
        lp = nb + 1 + i
        rawp = rng.integers(0, 256, size=(m, lp), dtype=np.uint8)  # junk beyond each column's bytes
        rawp[:, :nb] = P.T
        if n % 4:  # junk in the bits of rows past n in each column's last byte
            keep = (1 << (2 * (n % 4))) - 1
            rawp[:, nb - 1] = (rawp[:, nb - 1] & keep) | (rng.integers(0, 256, size=m, dtype=np.uint8) & ~np.uint8(keep))
        for lst, data, tag in ((p8, raw, "bin"), (pp, rawp, "2bit")):
            path = tmp_path / f"study{i}.{tag}"
            with open(path, "wb") as f:
                f.write(b"\xa5" * head)
                f.write(data.tobytes())
            lst.append(str(path))
        ld8.append(n); ldp.append(lp); heads.append(head); Xs.append(X)
    try:
        with gw.GLSBatch(gls) as B:
            o8 = B.solve_files(p8, ms, cols, ldx=ld8, header_bytes=heads)
            op = B.solve_files(pp, ms, cols, ldx=ldp, header_bytes=heads, packed=True)
            for i, (a, q) in enumerate(zip(o8, op)):
                assert all(np.array_equal(u, v, equal_nan=True) for u, v in zip(a, q)), i
                assert a[2][6] == 1 and np.isnan(q[0][:, 6]).all()
            for i, ((s, _), X, (b, se, st)) in enumerate(zip(studies, Xs, op)):
                L = oracle.potrf(oracle.form_m(s["Phi"], 0.5, 1.0))
                pick = np.r_[np.arange(0, X.shape[1], 29), X.shape[1] - 1]
                r, se_o, _, st_o = oracle.gls(L, s["XL"], s["y"], X[:, pick])
                e = compare(b[:, pick], se[:, pick], st[pick], r, se_o, st_o)
                assert e["b_norm"] <= 1e-5 and e["se_rel"] <= 1e-5, (i, e)
            bad = list(ldp)
            bad[2] = (NS[2] + 3) // 4 - 1
            with pytest.raises(gw.GwasError) as err:
                B.solve_files(pp, ms, cols, ldx=bad, header_bytes=heads, packed=True)
            assert err.value.name == "GWAS_ERR_ARG"
            with pytest.raises(gw.GwasError) as err:
                B.solve_files(pp, [m + 300 for m in ms], cols, ldx=ldp, header_bytes=heads, packed=True)
            assert err.value.name == "GWAS_ERR_IO"
    finally:
        for g in gls:
            g.close()
