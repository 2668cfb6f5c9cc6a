"""Out-of-core streaming: disk -> pinned host (reader thread) -> device ring -> solve."""
import ctypes
import os

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


@pytest.fixture(scope="module")
def dosage_file(tmp_path_factory):
    n, m, ld, header = 1000, 2200, 1003, 64
    X = gwas_synth.dosages(n, 0, m, seed=40)
    raw = np.zeros((m, ld), dtype=np.int8)
    raw[:, :n] = X.T
    path = tmp_path_factory.mktemp("geno") / "dosages.bin"
    with open(path, "wb") as f:
        f.write(b"\x7f" * header)
        f.write(raw.tobytes())
    return str(path), n, m, ld, header, X


TOL = {"fp64": 1e-10, "sliced64": 1e-10, "bf16x3": 1e-5, "f16x2": 1e-5}


@pytest.fixture(scope="module")
def oracle_results(dosage_file):
    """The FP64 oracle over every column of the file (b, se, status)."""
    path, n, m, ld, header, X = dosage_file
    s = gwas_synth.study(n, 4, 2000, 0.6, seed=40)
    L = oracle.potrf(oracle.form_m(s["Phi"], 0.6, 1.0))
    r, se, _, st = oracle.gls(L, s["XL"], s["y"], X)
    return r, se, st


def _check_oracle(b, se, st, ref, cols, prec):
    """Columns `cols` of the file against the oracle; b, se, st hold those columns in order."""
    r, se_o, st_o = ref
    e = compare(b, se, st, r[:, cols], se_o[:, cols], st_o[cols])
    assert e["b_norm"] <= TOL[prec] and e["se_rel"] <= TOL[prec], (prec, e)


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_solve_file_matches_blocks_and_resumes(dosage_file, oracle_results, prec):
    path, n, m, ld, header, X = dosage_file
    s = gwas_synth.study(n, 4, 2000, 0.6, seed=40)
    with gw.GLS(s["Phi"], s["XL"], s["y"], 0.6, 1.0, precision=prec, bs=512) as g:
        b, se, st = g.solve_file(path, m, ldx=ld, header_bytes=header)
        _check_oracle(b, se, st, oracle_results, np.arange(m), prec)  # every column, first and last of each block
        ref = [g.solve_block(X[:, c0:c0 + 512]) for c0 in range(0, m, 512)]
        b_ref = np.concatenate([r[0] for r in ref], axis=1)
        st_ref = np.concatenate([r[2] for r in ref])
        assert np.array_equal(b, b_ref) and np.array_equal(st, st_ref)
        # resume from a column cursor
        b2, se2, st2 = g.solve_file(path, m - 1100, ldx=ld, col0=1100, header_bytes=header)
        _check_oracle(b2, se2, st2, oracle_results, np.arange(1100, m), prec)
        assert np.array_equal(b2, b_ref[:, 1100:]) and np.array_equal(se2, se[:, 1100:])


@pytest.mark.parametrize("prec", ["fp64", "f16x2"])
def test_solve_file_out_writes_results_and_resumes(dosage_file, oracle_results, tmp_path, prec):
    """Disk to disk: the result file holds exactly what the in-memory stream
    returns; a run resumed from a checkpoint recomputes what follows it and
    ends with the same file."""
    path, n, m, ld, header, X = dosage_file
    s = gwas_synth.study(n, 4, 2000, 0.6, seed=40)
    out = str(tmp_path / "results.bin")
    with gw.GLS(s["Phi"], s["XL"], s["y"], 0.6, 1.0, precision=prec, bs=128) as g:
        b, se, st = g.solve_file(path, m - 300, ldx=ld, col0=300, header_bytes=header)
        done = g.solve_file_out(path, m - 300, out, ldx=ld, col0=300, header_bytes=header)
        assert done == m - 300
        head, b2, se2, st2 = gw.read_results(out)
        assert head == dict(p=4, n=n, col0=300, m=m - 300, record_bytes=72, precision=gw.PRECISIONS[prec])
        _check_oracle(b2, se2, st2, oracle_results, np.arange(300, m), prec)
        assert np.array_equal(b, b2) and np.array_equal(se, se2) and np.array_equal(st, st2)
        full = open(out, "rb").read()
        # an interrupted run: the checkpoint says 2 blocks, the records after them are garbage
        ck = bytearray(open(out + ".ckpt", "rb").read())
        assert ck[:8] == b"GWASCKP\0" and int.from_bytes(ck[48:56], "little") == m - 300
        ck[48:56] = (256).to_bytes(8, "little")
        open(out + ".ckpt", "wb").write(bytes(ck))
        with open(out, "r+b") as f:
            f.seek(64 + 256 * 72)
            f.write(b"\xee" * (72 * 500))
        assert g.solve_file_out(path, m - 300, out, ldx=ld, col0=300, header_bytes=header, resume=True) == m - 300
        assert open(out, "rb").read() == full
        _, b3, se3, st3 = gw.read_results(out)  # the resumed range against the oracle as well
        _check_oracle(b3[:, 256:], se3[:, 256:], st3[256:], oracle_results, np.arange(300 + 256, m), prec)
        # a checkpoint of another run is refused
        with pytest.raises(gw.GwasError) as e:
            g.solve_file_out(path, m - 301, out, ldx=ld, col0=300, header_bytes=header, resume=True)
        assert e.value.name == "GWAS_ERR_ARG"
        with pytest.raises(gw.GwasError) as e:
            g.solve_file_out(path, 10, str(tmp_path / "no_such_dir" / "r.bin"), ldx=ld, header_bytes=header)
        assert e.value.name == "GWAS_ERR_IO"


@pytest.mark.parametrize("prec", ["fp64", "f16x2", "sliced64"])
def test_solve_file_out_packed_input(dosage_file, oracle_results, tmp_path, prec):
    """Disk to disk from a 2-bit packed file (GWAS_PACKED_INPUT; columns of
    ceil(n/4) bytes at a stride of 257 bytes after a 64-byte header): the
    result file equals the one from the int8 file byte for byte, a quarter of
    the bytes crossed the link, and a packed run resumes from a checkpoint."""
    path, n, m, ld, header, X = dosage_file
    nb = (n + 3) // 4
    ldp = nb + 7
    raw = np.zeros((m, ldp), dtype=np.uint8)
    raw[:, :nb] = gw.pack_dosages2(X).T
    ppath = str(tmp_path / "dosages.2bit")
    with open(ppath, "wb") as f:
        f.write(b"\x5a" * 64)
        f.write(raw.tobytes())
    s = gwas_synth.study(n, 4, 2000, 0.6, seed=40)
    out8, outp = str(tmp_path / "r8.bin"), str(tmp_path / "rp.bin")
    with gw.GLS(s["Phi"], s["XL"], s["y"], 0.6, 1.0, precision=prec, bs=256) as g:
        assert g.solve_file_out(path, m - 100, out8, ldx=ld, col0=100, header_bytes=header) == m - 100
        h0 = g.h2d_bytes
        assert g.solve_file_out(ppath, m - 100, outp, ldx=ldp, col0=100, header_bytes=64, packed=True) == m - 100
        assert g.h2d_bytes - h0 == nb * (m - 100)
        full = open(outp, "rb").read()
        assert full == open(out8, "rb").read()
        _, b2, se2, st2 = gw.read_results(outp)
        _check_oracle(b2, se2, st2, oracle_results, np.arange(100, m), prec)
        ck = bytearray(open(outp + ".ckpt", "rb").read())
        ck[48:56] = (512).to_bytes(8, "little")
        open(outp + ".ckpt", "wb").write(bytes(ck))
        with open(outp, "r+b") as f:
            f.seek(64 + 512 * 72)
            f.write(b"\xee" * (72 * 300))
        assert g.solve_file_out(ppath, m - 100, outp, ldx=ldp, col0=100, header_bytes=64, packed=True,
                                resume=True) == m - 100
        assert open(outp, "rb").read() == full
        with pytest.raises(gw.GwasError) as e:  # a packed stride below ceil(n/4)
            g.solve_file_out(ppath, 10, outp, ldx=nb - 1, header_bytes=64, packed=True)
        assert e.value.name == "GWAS_ERR_ARG"


def test_solve_file_several_phenotypes(dosage_file, tmp_path):
    """t phenotypes through the file forms: b is p x m x t, the result file
    holds every phenotype's b in each record."""
    path, n, m, ld, header, X = dosage_file
    s = gwas_synth.study(n, 4, 2000, 0.6, seed=40)
    rng = np.random.default_rng(3)
    Y = np.asfortranarray(np.column_stack([s["y"], s["y"] + rng.standard_normal(n), rng.standard_normal(n)]))
    out = str(tmp_path / "r3.bin")
    with gw.GLS(s["Phi"], s["XL"], Y, 0.6, 1.0, precision="bf16x3", bs=512) as g:
        b, se, st = g.solve_file(path, m, ldx=ld, header_bytes=header)
        assert b.shape == (4, m, 3)
        ref = [g.solve_block(X[:, c0:c0 + 512]) for c0 in range(0, m, 512)]
        assert np.array_equal(b, np.concatenate([r[0] for r in ref], axis=1))
        assert g.solve_file_out(path, m, out, ldx=ld, header_bytes=header) == m
    head, b2, se2, st2 = gw.read_results(out)
    assert head["traits"] == 3 and head["record_bytes"] == 8 * 4 * 4 + 8
    assert np.array_equal(b, b2) and np.array_equal(se, se2) and np.array_equal(st, st2)


def test_solve_file_errors(dosage_file):
    path, n, m, ld, header, X = dosage_file
    s = gwas_synth.study(n, 4, 2000, 0.6, seed=40)
    with gw.GLS(s["Phi"], s["XL"], s["y"], 0.6, 1.0, bs=512) as g:
        with pytest.raises(gw.GwasError) as e:
            g.solve_file(path + ".missing", 10, ldx=ld)
        assert e.value.name == "GWAS_ERR_IO"
        with pytest.raises(gw.GwasError) as e:
            g.solve_file(path, m + 5, ldx=ld, header_bytes=header)  # runs past the end of the file
        assert e.value.name == "GWAS_ERR_IO"


def test_reader_returns_file_blocks_in_order(dosage_file):
    path, n, m, ld, header, X = dosage_file
    block = 7 * ld
    nblk = (m + 6) // 7
    last = (m - 7 * (nblk - 1)) * ld
    with gw.Reader(path, header, block, nblk, last, depth=3) as r:
        for k in range(nblk):
            ptr, nbytes = r.next()
            assert nbytes == (last if k == nblk - 1 else block)
            got = np.ctypeslib.as_array((ctypes.c_int8 * nbytes).from_address(ptr)).reshape(-1, ld)[:, :n]
            assert np.array_equal(got, X[:, 7 * k:7 * k + got.shape[0]].T)
            r.release()
