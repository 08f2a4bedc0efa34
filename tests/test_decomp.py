"""Domain decomposition over cell ranges (paper_1806_00082_gb300.decomp) on
CPU ranks: each rank steps its own cells with the CPU oracle (its particles
numbered after those of the cells before it), the ranks exchange the rows
their particles drifted into, and the joined state equals the one-rank run bit
for bit, with pairs created and particles crossing every rank boundary in both
directions.  Once emulated in one process (three ranks), once as two gloo
processes."""
import os
import socket

import numpy as np
import pytest

import oracle
import wmc_inputs as wi
from paper_1806_00082_gb300 import decomp

# the packet straddles the middle of the 100-cell domain and the barrier
WL = wi.BARRIER_100.replace(packet=wi.Packet(50e-9, 5e-9, 0.1, 60_000))
STEPS = 6


def _oracle_step_fn(w):
    po = oracle.params(w)
    V = wi.potential(w)

    def step(hist, t, id_base):
        out, st = oracle.simulate_subdomain(po, hist, t, id_base, V=V)
        return out, {"pairs": int(st[oracle.ST_PAIRS]), "absorbed": int(st[oracle.ST_ABSORBED]),
                     "dropped": int(st[oracle.ST_DROPPED]), "particle_steps": int(st[oracle.ST_PARTICLE_STEPS])}

    return step


def _one_rank():
    return oracle.simulate(oracle.params(WL), wi.initial_histogram(WL), 1, STEPS, V=wi.potential(WL))


def test_ranges_prefix_and_halo_rows():
    r = decomp.CellRanges(10, 3)
    assert [r.range(k) for k in range(3)] == [(0, 3), (3, 6), (6, 10)]
    assert decomp.exclusive_prefix([5, 0, 7]) == [0, 5, 5]
    h = np.arange(40, dtype=np.int32).reshape(10, 4)
    left, right = decomp.split_halo(h, 3, 6, 10)
    assert left.tolist() == [8, 9, 10, 11] and right.tolist() == [24, 25, 26, 27]
    assert not h[2].any() and not h[6].any()
    decomp.merge_halo(h, 3, 6, np.ones(4, np.int32), 2 * np.ones(4, np.int32))
    assert h[3].tolist() == [13, 14, 15, 16] and h[5].tolist() == [22, 23, 24, 25]
    with pytest.raises(ValueError):
        decomp.CellRanges(2, 3)


def test_three_emulated_ranks_equal_one_rank():
    ref, st = _one_rank()
    ranges = decomp.CellRanges(WL.n_x, 3)
    states = decomp.scatter_ranges(wi.initial_histogram(WL), ranges)
    step = _oracle_step_fn(WL)
    tot = {"pairs": 0, "absorbed": 0, "dropped": 0, "particle_steps": 0}
    crossed = 0
    for t in range(1, STEPS + 1):
        before = [decomp.population(h, *ranges.range(r)) for r, h in enumerate(states)]
        states, counters = decomp.emulate_ranks(states, ranges, t, step)
        for c in counters:
            for k in tot:
                tot[k] += c[k]
        crossed += sum(abs(decomp.population(h, *ranges.range(r)) - b) for r, (h, b) in enumerate(zip(states, before)))
    np.testing.assert_array_equal(decomp.gather_ranges(states, ranges), ref)
    assert tot["pairs"] == st[oracle.ST_PAIRS] > 1000
    assert tot["particle_steps"] == st[oracle.ST_PARTICLE_STEPS]
    assert tot["dropped"] == st[oracle.ST_DROPPED] and tot["absorbed"] == st[oracle.ST_ABSORBED]
    assert crossed > 0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        comm = decomp.TorchComm()
        ranges = decomp.CellRanges(WL.n_x, world)
        lo, hi = ranges.range(rank)
        h = decomp.scatter_ranges(wi.initial_histogram(WL), ranges)[rank]
        step = _oracle_step_fn(WL)
        pairs = 0
        for t in range(1, STEPS + 1):
            h, c = decomp.decomposed_step(comm, ranges, h, t, step)
            pairs += c["pairs"]
        pairs_all = comm.allreduce_ints([pairs])[0]
        q.put((rank, lo, hi, h[lo:hi].copy(), pairs_all))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_equal_one_rank():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref, st = _one_rank()
    joined = np.zeros_like(ref)
    for _, lo, hi, rows, _ in res:
        joined[lo:hi] = rows
    np.testing.assert_array_equal(joined, ref)
    assert res[0][4] == res[1][4] == st[oracle.ST_PAIRS] > 1000
