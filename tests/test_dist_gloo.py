"""Multi-process host logic of the benchmark, world size 2 on CPU (gloo).

The GPU path needs no collective (each rank solves its own right-hand sides
against its own replica of the factors), so what is tested here is the part
that runs on the host: the column shares and the max-over-ranks timing that
sets a step's time and the whole-job rate."""

import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2203_13283_gb300 import dist as wdist


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world_size, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world_size), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world_size)
    try:
        r, w, lr = wdist.world()
        c0, c1 = wdist.shard_columns(1024, r, w)
        # rank-dependent "timings": the slowest rank must set both entries
        mx = wdist.max_over_ranks([1.0 + r, 10.0 - r])
        rate = wdist.job_throughput(c1 - c0, w, mx[0])
        out.put((r, w, lr, c0, c1, mx, rate))
    finally:
        dist.destroy_process_group()


def test_two_rank_shares_and_max_timing():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, l0, a0, b0, m0, q0), (r1, w1, l1, a1, b1, m1, q1) = res
    assert (r0, r1, w0, w1, l0, l1) == (0, 1, 2, 2, 0, 1)
    assert (a0, b0, a1, b1) == (0, 512, 512, 1024)
    assert m0 == m1 == [2.0, 10.0]
    assert q0 == q1 == pytest.approx(512 * 2 / 2.0)


@pytest.mark.parametrize("B,w", [(0, 3), (7, 3), (1024, 8), (5, 8)])
def test_shards_cover_columns_once(B, w):
    seen = []
    for r in range(w):
        c0, c1 = wdist.shard_columns(B, r, w)
        assert 0 <= c0 <= c1 <= B
        seen.extend(range(c0, c1))
    assert seen == list(range(B))
    sizes = [wdist.shard_columns(B, r, w)[1] - wdist.shard_columns(B, r, w)[0] for r in range(w)]
    assert max(sizes) - min(sizes) <= 1


def test_single_process_max_is_identity():
    assert wdist.max_over_ranks([3.0, 4.0]) == [3.0, 4.0]
    with pytest.raises(ValueError):
        wdist.shard_columns(4, 2, 2)


def _gather_main(rank, world_size, port, n, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world_size)
    try:
        c0, c1 = wdist.shard_columns(n, rank, world_size)
        local = [float(i * i) + 0.5 for i in range(c0, c1)]      # a rank's share of a gradient
        out.put((rank, wdist.gather_shards(local, n)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("n", [32, 7, 1])
def test_two_rank_gather_of_parameter_shares(n):
    # the shape gradient's parameters split over two ranks and gathered back:
    # each rank ends with the whole vector in parameter order
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gather_main, args=(r, 2, port, n, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = [float(i * i) + 0.5 for i in range(n)]
    assert res[0] == want and res[1] == want


def test_gather_shards_single_process():
    assert wdist.gather_shards([1.0, 2.0], 2) == [1.0, 2.0]
