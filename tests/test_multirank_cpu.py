"""The multi-process host logic on CPU: two gloo ranks.

Ranks share nothing on the data path; they only meet at a barrier and take
the maximum of their step times.  The ROI split covers every ROI once.
"""
import os
import socket

import pytest

from paper_2009_00735_gb300.ranks import max_over_ranks, roi_shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2009_00735_gb300.ranks import barrier, rank_info
    r, w, _ = rank_info()
    barrier()
    m = max_over_ranks(10.0 + 5.0 * r)
    lo, hi = roi_shard(8192 + 3, r, w)
    q.put((r, w, m, lo, hi))
    dist.destroy_process_group()


def test_two_gloo_ranks_max_and_split():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[0] for x in res] == [0, 1] and all(x[1] == 2 for x in res)
    assert all(x[2] == 15.0 for x in res)
    assert res[0][3] == 0 and res[0][4] == res[1][3] and res[1][4] == 8195


@pytest.mark.parametrize("n,w", [(0, 3), (5, 8), (8192, 2), (100003, 7)])
def test_roi_shard_partition(n, w):
    spans = [roi_shard(n, r, w) for r in range(w)]
    assert spans[0][0] == 0 and spans[-1][1] == n
    assert all(spans[i][1] == spans[i + 1][0] for i in range(w - 1))
    sizes = [b - a for a, b in spans]
    assert max(sizes) - min(sizes) <= 1
