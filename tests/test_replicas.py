"""The N > 1 benchmark path on CPU: replicas only (each rank solves its own system; no
collective on the data path).  Two gloo ranks check the whole-job aggregation -- slowest
rank's time, all ranks' steps -- and that the reference arm runs on rank 0 only."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, e2e, steps = bench.reduce_replicas(10.0 + rank, 20.0 - rank, 100 * (rank + 1), dist, "cpu")
    q.put((rank, ms, e2e, steps, bench.dist_env()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, e2e, steps, env in out:
        assert ms == 11.0 and e2e == 20.0 and steps == 300  # max, max, sum
        assert env == (2, rank, rank)


def test_reference_arm_other_ranks_do_nothing(capsys, monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")

    class Args:
        steps, warmup, gs = 1, 3, 2

    bench.run_reference(Args())
    assert capsys.readouterr().out == ""


def test_local_aggregation_without_group():
    import bench
    assert bench.reduce_replicas(5.0, 6.0, 100) == (5.0, 6.0, 100)
