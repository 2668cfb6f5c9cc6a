"""SNP sharding (Sec. 3.2: every GPU holds the study, the SNP blocks are split
between GPUs) checked on one GPU: the block assignment the multi-GPU bench
uses (shard_block_starts for 2 and 4 ranks) is solved as logical shards, one
after another, each shard with its own context as its rank would have.  The
per-shard results gathered into column order must equal one unsharded run bit
for bit (a block's results depend on that block alone), and match the FP64
oracle on a seeded sample of columns."""
import numpy as np
import pytest

import gwas_synth
import oracle
import paper_1302_4332_b300 as gw
from oracle.metrics import compare
from paper_1302_4332_b300.shard import assemble_columns, shard_block_starts

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


N, P, BS, NB = 1000, 4, 512, 2
TOL = {"fp64": 1e-10, "bf16x3": 1e-5, "f16x2": 1e-5}


@pytest.fixture(scope="module")
def study():
    s = gwas_synth.study(N, P, 2000, 0.6, 1.0, seed=51)
    L = oracle.potrf(oracle.form_m(s["Phi"], 0.6, 1.0))
    return s, L


def _solve_blocks(s, prec, starts):
    """One rank: its own context, its blocks (the dosages regenerated from their column range)."""
    out = []
    with gw.GLS(s["Phi"], s["XL"], s["y"], 0.6, 1.0, precision=prec, bs=BS) as g:
        for c0 in starts:
            X = gwas_synth.dosages(N, c0, c0 + BS, seed=51)
            out.append((c0, g.solve_block(X)))
    return out


@pytest.mark.parametrize("prec", ("fp64", "bf16x3", "f16x2"))
@pytest.mark.parametrize("world", (2, 4))
def test_logical_shards_equal_one_run(study, prec, world):
    s, L = study
    m = world * NB * BS
    whole = assemble_columns([_solve_blocks(s, prec, range(0, m, BS))])
    parts = [_solve_blocks(s, prec, shard_block_starts(r, world, NB, BS)) for r in range(world)]
    sharded = assemble_columns(parts)
    for a, b in zip(sharded, whole):
        assert a.shape == b.shape and np.array_equal(a, b)
    rng = np.random.default_rng(world)
    pick = np.unique(np.r_[0, m - 1, [c for c in range(0, m, BS)], [c - 1 for c in range(BS, m, BS)],
                           rng.choice(m, 40, replace=False)])
    X = np.asfortranarray(np.column_stack([gwas_synth.dosages(N, c, c + 1, seed=51)[:, 0] for c in pick]))
    r, se, _, st = oracle.gls(L, s["XL"], s["y"], X)
    b, se_g, st_g = sharded
    e = compare(b[:, pick], se_g[:, pick], st_g[pick], r, se, st)
    assert e["b_norm"] <= TOL[prec] and e["se_rel"] <= TOL[prec], e
