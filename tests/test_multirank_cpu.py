"""The N > 1 path of bench.py on CPU: two gloo ranks run independent replicas
and exchange only their timing, the job's time is the slowest rank's and the
value counts every rank's units.  Also: the reference arm prints on rank 0
only."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = [1.5, 2.25][rank]
    t = bench.max_over_ranks(local, dist, "cpu")
    v = bench.job_throughput(1000, world, t)
    out.put((rank, t, v, bench.dist_env()))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
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
    for rank, t, v, env in res:
        assert t == 2.25                      # max over ranks
        assert v == pytest.approx(2 * 1000 / 2.25)
        assert env[0] == rank and env[1] == 2


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.0, None, "cpu") == 3.0
    assert bench.job_throughput(10, 1, 2.0) == 5.0


def test_reference_arm_prints_on_rank_zero_only(capsys, monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        pass
    a = A()
    a.seed, a.scale, a.steps, a.warmup, a.gpus = 1, 1.0, 1, 1, 2
    bench.run_reference(a)  # a non-zero rank returns without work
    assert capsys.readouterr().out == ""
