"""World-size-2 gloo tests of the multi-GPU host logic (CPU only): independent subband shards, the
barrier, and the max/sum reductions that bench.py uses around its timed region."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as tmp  # noqa: E402

from paper_1105_0661_gb300 import dist  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    r, w = dist.init("gloo")
    assert (r, w) == (rank, world)
    lo, hi = dist.shard_range(244, r, w)
    dist.barrier()
    mx = dist.reduce_scalar(10.0 + r, "max")
    total = dist.reduce_scalar(hi - lo, "sum")
    q.put((r, lo, hi, mx, total))
    dist.finalize()


def test_shard_range_partitions():
    for n in (1, 7, 244):
        for world in (1, 2, 3, 8):
            parts = [dist.shard_range(n, r, world) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(parts[i][1] == parts[i + 1][0] for i in range(world - 1))
            sizes = [hi - lo for lo, hi in parts]
            assert max(sizes) - min(sizes) <= 1


def test_two_rank_gloo_reductions():
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1:3] for r in res] == [(0, 122), (122, 244)]
    assert all(r[3] == 11.0 for r in res)      # max over ranks
    assert all(r[4] == 244.0 for r in res)     # every subband owned exactly once


def test_single_process_is_identity():
    for k in ("RANK", "LOCAL_RANK", "WORLD_SIZE"):
        os.environ.pop(k, None)
    assert dist.env_rank() == (0, 0, 1)
    assert dist.reduce_scalar(3.5, "max") == 3.5
