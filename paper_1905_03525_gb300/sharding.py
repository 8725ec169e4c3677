"""Multi-GPU use of the generator: range sharding, no collective.

Edges are independent given (table, seed, global edge index) -- the paper's
generation is communication-free (Sec. 3, parallelization) -- so rank r of W
generates its own range of the graph and nothing is exchanged on the data
path.  Weak scaling: every rank owns `per_rank` edges, the graph has
W * per_rank.  Strong scaling: a fixed m split into W near-equal ranges.
"""
from __future__ import annotations


def weak_range(rank: int, per_rank: int) -> tuple[int, int]:
    """(edge_offset, count) of `rank` when every rank owns per_rank edges."""
    return rank * per_rank, per_rank


def strong_range(rank: int, world: int, m: int) -> tuple[int, int]:
    """(edge_offset, count) of `rank` when m edges are split over `world` ranks
    (the first m % world ranks get one edge more)."""
    base, extra = divmod(m, world)
    start = rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)


def row_tiles(rank: int, world: int, tile_levels: int) -> tuple[int, int]:
    """(row_tile_begin, row_tile_end) of `rank` for a partitioned graph
    (Sec. 3): the 2^tile_levels tile rows split into `world` near-equal runs,
    so rank r holds every edge whose row falls in its run and nothing is
    exchanged."""
    return strong_range(rank, world, 1 << tile_levels)[0], sum(strong_range(rank, world, 1 << tile_levels))
