"""CPU checks of the C-ABI library: it loads, exports every symbol the header
declares, and refuses to compute without a CUDA device (no CPU fallback)."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

import paper_1302_4332_b300 as gw
from paper_1302_4332_b300 import build as gbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_symbols():
    syms = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        syms |= set(re.findall(r"\b(gwas_[a-z0-9_]+)\s*\(", text))
    return syms


@pytest.fixture(scope="module")
def lib():
    gbuild.build()
    return gw.load()


def test_library_exports_every_declared_symbol(lib):
    syms = _header_symbols()
    assert syms, "no declarations found"
    assert set(gw.EXPORTS) <= syms
    for s in sorted(syms):
        assert hasattr(lib, s), f"{s} declared in include/ but not exported"


def test_strerror_and_defaults(lib):
    assert lib.gwas_strerror(0) == b"ok"
    assert lib.gwas_strerror(-2) == b"matrix not positive definite"
    cfg = gw._Config()
    lib.gwas_config_default(ctypes.byref(cfg))
    assert (cfg.precision, cfg.bs, cfg.ring_depth, cfg.device) == (0, 4096, 3, -1)


def test_config_struct_matches_the_header(lib):
    """gwas_config_default writes exactly the C struct: as many bytes as the
    binding's _Config holds (a guard region after it stays untouched), and the
    fields the header lists, in its order, are the binding's."""
    size = ctypes.sizeof(gw._Config)
    buf = (ctypes.c_ubyte * (size + 64))(*([0xA5] * (size + 64)))
    lib.gwas_config_default(ctypes.cast(buf, ctypes.POINTER(gw._Config)))
    assert all(b == 0xA5 for b in bytes(buf)[size:]), "the C struct is larger than the binding's"
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "gwas_b300.h")).read(), flags=re.S)
    body = re.search(r"typedef struct \{(.*?)\} gwas_config;", text, flags=re.S).group(1)
    fields = re.findall(r"\bint\s+([a-z_0-9]+)\s*;", body)
    assert fields == [name for name, _ in gw._Config._fields_]
    zeros = gw._Config()
    lib.gwas_config_default(ctypes.byref(zeros))
    assert zeros.separate_sums == 0 and zeros.single_piece == 0 and zeros.traits == 0


def test_null_context_is_an_argument_error(lib):
    assert lib.gwas_synchronize(None) == -1
    assert lib.gwas_check_timeout(None, 0, 1000) == -1
    assert lib.gwas_solve_block(None, None, 0, 0, None, None, None) == -1
    lib.gwas_destroy(None)


def _has_gpu():
    import torch
    return torch.cuda.is_available()


@pytest.mark.skipif(_has_gpu(), reason="a GPU is present")
def test_no_device_fails_loudly(lib):
    n = 8
    with pytest.raises(gw.GwasError) as e:
        gw.GLS(np.eye(n), np.ones((n, 1)), np.ones(n), 0.5)
    assert e.value.name in ("GWAS_ERR_CUDA", "GWAS_ERR_UNSUPPORTED")


def test_tuning_struct_matches_the_header():
    """The binding's gwas_batch_tuning mirror has the header's fields, in order."""
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "gwas_b300.h")).read(), flags=re.S)
    body = re.search(r"typedef struct \{([^{}]*)\} gwas_batch_tuning;", text).group(1)
    fields = re.findall(r"\b(?:int|double)\s+([a-z_0-9]+)\s*;", body)
    assert fields == [name for name, _ in gw._Tuning._fields_]


def _pack_reference(X):
    """The 2-bit encoding written out: byte k of a column = sum_i X[4k + i] 4^i."""
    n, m = X.shape
    nb = (n + 3) // 4
    Xp = np.zeros((4 * nb, m), dtype=np.int64)
    Xp[:n] = X
    return (Xp[0::4] + 4 * Xp[1::4] + 16 * Xp[2::4] + 64 * Xp[3::4]).astype(np.uint8)


@pytest.mark.parametrize("n", [1, 3, 4, 5, 7, 8, 9, 15, 16, 17, 63, 64, 65, 127, 128, 129, 1000, 10001])
def test_pack_dosages2_encoding(lib, n):
    """The stream transport's host packing (host code, no device needed) against
    the encoding written out, on ragged n, values 0..3 (3 included)."""
    rng = np.random.default_rng(n)
    X = np.asfortranarray(rng.integers(0, 4, size=(n, 37)).astype(np.int8))
    P = gw.pack_dosages2(X)
    assert P.shape == ((n + 3) // 4, 37)
    np.testing.assert_array_equal(P, _pack_reference(X))


@pytest.mark.parametrize("bad", [4, -1, 127, -128])
def test_pack_dosages2_refuses_other_values(lib, bad):
    X = np.zeros((50, 5), dtype=np.int8, order="F")
    X[49, 3] = bad  # the last row of one column: the ragged end is checked too
    with pytest.raises(gw.GwasError) as e:
        gw.pack_dosages2(X)
    assert e.value.name == "GWAS_ERR_ARG"
    X[49, 3] = 2
    X[0, 4] = bad
    with pytest.raises(gw.GwasError):
        gw.pack_dosages2(X)
