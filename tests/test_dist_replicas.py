"""Multi-process (replicas) path of bench.py on CPU: two gloo ranks.

The solver is single-GPU; with N ranks bench.py runs N independent replicas,
times them between barriers, takes the slowest rank's time and reports the
whole-job throughput.  These tests run that host logic with world size 2.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        local_s = 1.0 + rank                              # rank 1 is the slowest
        dist.barrier()
        slowest = bench.max_over_ranks(local_s)
        value = bench.replica_mlups(1000, 10, world, slowest)
        q.put((rank, slowest, value, bench.dist_env()))
    finally:
        dist.destroy_process_group()


def test_two_rank_max_over_ranks_and_whole_job_value():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, value, env in out:
        assert slowest == 2.0                            # both ranks see the slowest time
        assert value == pytest.approx(1000 * 10 * 2 / 2.0 / 1e6)
        assert env == (rank, 2, rank)


def test_single_process_is_its_own_max():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.replica_mlups(100, 4, 1, 2.0) == pytest.approx(100 * 4 / 2.0 / 1e6)


def test_reference_arm_is_rank0_only(monkeypatch, capsys):
    """Under torchrun the oracle arm runs on rank 0 alone; other ranks exit 0 silently."""
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        workload, steps, warmup, gpus = "riemann", 1, 3, 2
    assert bench.run_reference(A()) == 0
    assert capsys.readouterr().out == ""
