"""The N > 1 bench path on CPU: two gloo ranks.  Every rank steps its own
replica melt (distinct seeds, no exchange between ranks), the timed region is
the slowest rank's, and the whole-job value counts all ranks' atom-steps."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        got_ws, got_rank, _ = bench._dist()
        t = bench.max_over_ranks(10.0 + 7.5 * rank, ws)       # this rank's "elapsed time"
        m = bench.make_workload(rank, chains=3)
        q.put((rank, got_ws, got_rank, t, bench.replica_seed(rank), float(m["pos"][0, 0])))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_time_the_slowest_and_step_distinct_replicas():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [2, 2] and [o[2] for o in out] == [0, 1]
    assert all(o[3] == 17.5 for o in out)                      # max over ranks on every rank
    assert out[0][4] != out[1][4] and out[0][5] != out[1][5]   # independent replicas


def test_aggregate_rate_counts_every_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_rate(4, 1000, 10, 2.0) == 4 * 1000 * 10 / 2.0
    assert bench.max_over_ranks(3.25, 1) == 3.25
