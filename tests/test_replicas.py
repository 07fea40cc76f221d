"""Multi-rank bench path on CPU: two gloo ranks stand for two GPUs.

The path does not shard (each rank runs an independent replica of the job),
so the only cross-rank step is the aggregation: the slowest rank's time and
the updates of all ranks.  The reference arm runs on rank 0 only.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r timed (r + 1) * 10 ms on the device and (r + 1) * 15 ms end to end,
    # and applied (r + 1) million updates
    res = bench.replica_throughput(dist, 10.0 * (rank + 1), 15.0 * (rank + 1), 1e6 * (rank + 1),
                                   "cpu")
    dist.destroy_process_group()
    out.put((rank, res))


@pytest.mark.timeout(120)
def test_two_rank_aggregation_takes_slowest_time_and_all_updates():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    results = dict(out.get(timeout=100) for _ in range(world))
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    for rank in range(world):
        value, e2e, ms_max, e2e_max, total = results[rank]
        assert ms_max == 20.0 and e2e_max == 30.0
        assert total == 3e6
        assert value == pytest.approx(3e6 / 0.020)
        assert e2e == pytest.approx(3e6 / 0.030)


def test_one_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    value, e2e, ms_max, e2e_max, total = bench.replica_throughput(None, 50.0, 0.0, 2e6, "cpu")
    assert value == pytest.approx(2e6 / 0.05) and e2e is None and total == 2e6


def test_reference_arm_runs_on_rank_zero_only(capsys, monkeypatch):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup = 1, 0

    bench.bench_reference(Args())
    assert capsys.readouterr().out == ""
