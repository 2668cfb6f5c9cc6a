"""SNP sharding over ranks (one process per GPU) for the per-SNP GLS.

SNPs are independent (Eq. 1 holds for each i on its own), so a multi-GPU run
splits the SNP columns into contiguous blocks, gives every rank the whole
study (its own copy of L and the loop-invariant part of Listing 1, as Sec. 3.2
of the paper replicates it on every GPU) and a disjoint set of blocks, and
exchanges nothing on the data path.  The only collective is the host-side
gather of the per-rank results into column order at the end.
"""
from __future__ import annotations

import numpy as np


def shard_block_starts(rank: int, world: int, nb: int, bs: int) -> list[int]:
    """First SNP column of each of this rank's nb blocks of bs columns: rank r
    owns blocks r*nb .. r*nb + nb - 1, so ranks never share a SNP."""
    return [(rank * nb + i) * bs for i in range(nb)]


def assemble_columns(parts) -> tuple[np.ndarray, ...]:
    """Concatenates per-rank results in SNP column order.

    parts: one entry per rank, each a list of (c0, arrays) with arrays a tuple
    of column blocks (2-D p x ncols, or 1-D ncols) whose first column is SNP c0.
    Returns each array concatenated over all ranks' blocks, sorted by c0; the
    blocks must tile the columns without gap or overlap."""
    blocks = sorted((c0, arrs) for rank_parts in parts for c0, arrs in rank_parts)
    if not blocks:
        return ()
    nxt = blocks[0][0]
    for c0, arrs in blocks:
        if c0 != nxt:
            raise ValueError(f"SNP blocks do not tile the columns: expected column {nxt}, got {c0}")
        nxt = c0 + np.shape(arrs[0])[-1]
    k = len(blocks[0][1])
    return tuple(np.concatenate([np.asarray(arrs[i]) for _, arrs in blocks], axis=-1) for i in range(k))


def gather_columns(dist, local_parts, dst: int = 0):
    """Host-side gather over a torch.distributed process group: every rank
    passes its list of (c0, arrays); rank `dst` gets the arrays in column
    order (assemble_columns), the other ranks None."""
    world = dist.get_world_size()
    got = [None] * world if dist.get_rank() == dst else None
    dist.gather_object(local_parts, got, dst=dst)
    return assemble_columns(got) if got is not None else None
