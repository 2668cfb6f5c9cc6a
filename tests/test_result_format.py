"""The result file format of gwas_solve_file_out, as include/gwas_b300.h
documents it, against the binding's reader (no GPU)."""
import struct

import numpy as np
import pytest

import paper_1302_4332_b300 as gw


def _write(path, p, m, t, col0=5, n=123, precision=3):
    rec = 8 * p * (t + 1) + 8  # GWAS_RESULT_RECORD_BYTES_T(p, t); 16p + 8 for t = 1
    head = b"GWASRES\0" + struct.pack("<IIQQQII", 1, p, n, col0, m, rec, precision) + bytes(8) + \
        struct.pack("<Q", t if t > 1 else 0)
    assert len(head) == 64
    rng = np.random.default_rng(9)
    b = rng.standard_normal((m, t, p))
    se = rng.random((m, p))
    st = rng.integers(0, 2, m).astype(np.int32)
    with open(path, "wb") as f:
        f.write(head)
        for j in range(m):
            f.write(b[j].astype("<f8").tobytes() + se[j].astype("<f8").tobytes() + struct.pack("<ii", st[j], 0))
    return rec, b, se, st


@pytest.mark.parametrize("p,t", [(4, 1), (3, 2), (1, 5)])
def test_reader_matches_the_documented_layout(tmp_path, p, t):
    path = str(tmp_path / "r.bin")
    m = 17
    rec, b, se, st = _write(path, p, m, t)
    head, b2, se2, st2 = gw.read_results(path)
    assert head["p"] == p and head["m"] == m and head["col0"] == 5 and head["n"] == 123
    assert head["record_bytes"] == rec == (16 * p + 8 if t == 1 else 8 * p * (t + 1) + 8)
    assert head.get("traits", 1) == t
    if t == 1:
        assert b2.shape == (p, m) and np.array_equal(b2, b[:, 0, :].T)
    else:
        assert b2.shape == (p, m, t) and np.array_equal(b2, np.transpose(b, (2, 0, 1)))
    assert np.array_equal(se2, se.T) and np.array_equal(st2, st)


def test_reader_refuses_other_files(tmp_path):
    path = tmp_path / "x.bin"
    path.write_bytes(b"GWASCKP\0" + bytes(56))
    with pytest.raises(ValueError):
        gw.read_results(str(path))
