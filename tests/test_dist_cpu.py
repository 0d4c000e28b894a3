"""The multi-rank path of bench.py on CPU: two gloo ranks (127.0.0.1) run the
host-side coordination - barrier, max over ranks of the step time, whole-job
throughput - exactly as the GPU ranks do (each rank filters its own search
block; there is no data-path collective)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, results):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank), CHEBFD_BENCH_BACKEND="gloo")
    w, r, local = bench.dist_setup(None)
    assert (w, r, local) == (world, rank, rank)
    bench.barrier(w)
    t_local = 1.0 + rank          # rank 1 is the slow one
    value, t_max = bench.aggregate(w, 1000.0, t_local)
    results[rank] = (value, t_max)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_two_gloo_ranks_aggregate_like_the_gpu_job(world):
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    results = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, results)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    # both ranks see the slowest time; value = all units / that time
    for r in range(world):
        value, t_max = results[r]
        assert t_max == pytest.approx(float(world))
        assert value == pytest.approx(world * 1000.0 / world)


def test_reference_arm_of_other_ranks_exits_quietly(monkeypatch, capsys):
    """Under torchrun the oracle reference runs on rank 0 only."""
    import bench
    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setenv("RANK", "1")

    class A:
        pass
    a = A()
    a.gpus, a.steps, a.warmup, a.Np = 2, 1, 1, 0
    assert bench.run_reference(a) == 0
    assert capsys.readouterr().out == ""
