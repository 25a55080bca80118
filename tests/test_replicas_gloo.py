"""Multi-rank path on CPU: two gloo ranks share the serving stream and reduce their times the way
bench.py does on N GPUs (replicas, no data-path collective)."""
import multiprocessing as mp
import os
import socket

import pytest

from paper_0904_4504_gb300 import replicas as R


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    from paper_0904_4504_gb300 import inputs as I
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, _ = R.env_rank()
        mine = R.rank_slice(I.serving_requests(n=40), r, 8)
        R.barrier(w)
        t = R.max_over_ranks(1.0 + r, w, device="cpu")
        rate = R.whole_job_rate(len(mine), w, t)
        q.put((r, [x.arrival_s for x in mine], t, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_share_requests_and_take_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    from paper_0904_4504_gb300 import inputs as I
    stream = [x.arrival_s for x in I.serving_requests(n=40)]
    assert res[0][1] == stream[0:8] and res[1][1] == stream[8:16]
    assert all(t == 2.0 for _, _, t, _ in res)          # max over ranks
    assert all(rate == 8 * 2 / 2.0 for _, _, _, rate in res)


def test_rank_slice_blocks_are_disjoint_and_cover():
    items = list(range(37))
    blocks = [R.rank_slice(items, r, 5) for r in range(4)]
    assert sum(blocks, []) == items[:20]
    with pytest.raises(ValueError):
        R.rank_slice(items, -1, 5)
    assert R.max_over_ranks(3.5, 1) == 3.5
