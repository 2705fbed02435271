"""Multi-rank plumbing of bench.py on CPU (gloo, world size 2).

The path has no exchange step, so N GPUs run N replicas; what needs checking
is the host logic around them: the rendezvous, the barrier, the max over ranks
of the timed region and the whole-job value computed from it, and that only
rank 0 runs the reference arm.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, q) -> None:
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import bench

    d = bench.Dist()
    d.init("gloo")
    d.barrier()
    # rank r "took" 100 (r + 1) ms for 3 steps of 20 solves
    mx = d.max(100.0 * (rank + 1), torch.device("cpu"))
    value = bench.aggregate_value(d.world, 20, 3, mx)
    ref = bench.run_reference(type("A", (), {"delta": 1e-4})(), d) if rank else "rank0-skipped"
    d.barrier()
    d.done()
    q.put((rank, d.world, mx, value, ref))


def test_replicas_time_is_max_over_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, world, mx, value, ref in out:
        assert world == 2
        assert mx == pytest.approx(200.0)
        # 2 replicas x 20 solves x 3 steps in 0.2 s
        assert value == pytest.approx(600.0)
    # the reference arm runs on rank 0 only; rank 1 returns nothing
    assert out[1][4] is None


def test_single_process_defaults():
    import bench

    d = bench.Dist()
    assert (d.world, d.rank) == (1, 0) or "WORLD_SIZE" in os.environ
    assert bench.aggregate_value(1, 20, 5, 1000.0) == pytest.approx(100.0)
