"""Tile sharding across processes (one process per GPU).

Tiles are independent (each is reconstructed on its own, Sec. 3.2), so a
slide's tiles split into contiguous ranges, one per rank, with no exchange on
the data path; only results are gathered where a caller wants them.
"""
from __future__ import annotations


def tile_range(rank: int, world: int, n_tiles: int) -> tuple[int, int]:
    """[start, stop) of the contiguous tile range of `rank` among `world` ranks.

    The first n_tiles % world ranks take one extra tile.
    """
    if world < 1 or not 0 <= rank < world or n_tiles < 0:
        raise ValueError("bad rank / world / n_tiles")
    base, extra = divmod(n_tiles, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)
