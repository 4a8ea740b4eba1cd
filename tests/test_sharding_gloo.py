"""Multi-process tile sharding on CPU (gloo, world size 2): the union of the
ranks' reconstructions equals the single-process run, with no collective
other than the final gather of results."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2407_20469_gb300.shard import tile_range  # noqa: E402

N_TILES, N = 5, 32


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _tiles():
    from helpers import make_tiles
    return make_tiles(N, N_TILES, seed=123, scale=0.3)[0]


def _reconstruct(I):
    from helpers import oracle_tile
    out = []
    for t in range(I.shape[0]):
        r = oracle_tile(I[t], N)
        out.append(np.concatenate([r.field.ravel(), r.c15.astype(np.complex128)]))
    return np.stack(out) if out else np.zeros((0, 4 * N * N + 15), np.complex128)


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    I = _tiles()
    a, b = tile_range(rank, world, N_TILES)
    mine = _reconstruct(I[a:b])
    parts = [None] * world
    dist.all_gather_object(parts, (a, b, mine))
    if rank == 0:
        q.put(parts)
    dist.destroy_process_group()


def test_tile_range_partitions():
    for n in (0, 1, 5, 512, 1023):
        for w in (1, 2, 3, 8):
            rs = [tile_range(r, w, n) for r in range(w)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            assert all(rs[i][1] == rs[i + 1][0] for i in range(w - 1))
            assert max(b - a for a, b in rs) - min(b - a for a, b in rs) <= 1


def test_two_rank_sharding_matches_single_process():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    parts = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = _reconstruct(_tiles())
    got = np.concatenate([m for _, _, m in sorted(parts, key=lambda x: x[0])])
    assert got.shape == ref.shape
    assert np.array_equal(got, ref)
