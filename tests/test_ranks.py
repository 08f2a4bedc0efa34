"""The multi-rank path of bench.py on CPU: two gloo ranks, each standing for a
GPU replica, reduce their timings and particle-step counts the way the
benchmark does (whole-job time = the slowest rank, work = the sum)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, ps = bench.reduce_over_ranks(10.0 + 5.0 * rank, 1000.0 * (rank + 1))
        out.put((rank, ms, ps))
    finally:
        torch.distributed.destroy_process_group()


def test_two_rank_reduction_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 15.0, 3000.0), (1, 15.0, 3000.0)]


def test_single_process_reduction_is_identity():
    import bench
    assert bench.reduce_over_ranks(7.5, 123.0) == (7.5, 123.0)


def test_step_work_count_per_step():
    """The particle-step kernel's Philox calls per step over one two-step
    launch: a quarter call per survivor-step (offsets) and a quarter per
    survivor of a reach cell (pair-creation words); the pair draws belong to
    the pair kernel."""
    import bench
    c0 = {"particle_steps": 1000, "pairs": 10}
    c1 = {"particle_steps": 1000 + 2 * 400, "pairs": 10 + 6}
    got = bench.philox_calls(c0, c1, 40.0, 48.0)
    assert got == (800 / 4 + (40 + 48) / 4) / 2
    assert bench.philox_calls(c0, c0, 0.0, 0.0) == 0.0
