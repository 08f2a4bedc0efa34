"""The domain decomposition through libwmc: ranks emulated one after another
on one GPU (no rank waits on another inside a kernel; rows are exchanged
between steps), each numbering its particles after those of the cells before
its range (wmc_set_id_base).  The joined state equals the one-rank wmc_run
bit for bit, and the CPU oracle."""
import numpy as np
import pytest

import oracle
import wmc_inputs as wi
from paper_1806_00082_gb300 import decomp
from tests._util import gpu_run

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wmc():
    from paper_1806_00082_gb300 import build, wmc as w
    build.build()
    w.load()
    return w


@pytest.mark.parametrize("wl,world,steps", [
    (wi.BARRIER_100.replace(packet=wi.Packet(50e-9, 5e-9, 0.1, 60_000)), 3, 6),
    (wi.DOUBLE_BARRIER_16384.replace(packet=wi.Packet(819.2e-9, 5e-9, 0.1, 400_000)), 2, 3),
])
def test_emulated_ranks_equal_one_rank(wmc, wl, world, steps):
    p = wmc.Params.of(wl)
    V = torch.from_numpy(wi.potential(wl)).cuda()
    h0 = wi.initial_histogram(wl)
    ref, c_ref = gpu_run(wmc, torch, p, wi.potential(wl), h0, 1, steps, use_graph=False)
    ranges = decomp.CellRanges(wl.n_x, world)
    ws = wmc.workspace(p)
    wmc.init(p, ws)
    step = decomp.gpu_step_fn(wmc, p, V, ws)
    states = decomp.scatter_ranges(torch.from_numpy(h0).cuda(), ranges)
    pairs = 0
    for t in range(1, steps + 1):
        states, counters = decomp.emulate_ranks(states, ranges, t, step)
        pairs += sum(c["pairs"] for c in counters)
    got = decomp.gather_ranges(states, ranges).cpu().numpy()
    np.testing.assert_array_equal(got, ref)
    assert pairs == c_ref["pairs"] > 1000
    if wl.n_x <= 100:
        o, st = oracle.simulate(oracle.params(wl), h0, 1, steps, V=wi.potential(wl))
        assert np.abs(got.sum(1) - o.sum(1)).sum() / wl.packet.n0 <= 1e-3


def test_id_base_numbering_and_materialize(wmc):
    """Survivors enumerated from id_base draw the Philox words of their global
    numbers and are written at id - id_base."""
    wl = wi.BARRIER_100
    p = wmc.Params.of(wl)
    h = wi.random_histogram(wl, 5_000, seed=3, cells=(60, 80))
    ws = wmc.workspace(p)
    wmc.init(p, ws)
    hd = torch.from_numpy(h).cuda()
    base = 123_457
    wmc.set_id_base(p, ws, base)
    wmc.annihilate(p, hd, ws)
    P = int(np.abs(h).sum())
    cell, f, M, s = (x.cpu().numpy() for x in wmc.materialize(p, hd, 9, ws, P))
    # the oracle's global numbering: the same particles after `base` others
    rc, rf, rM, rs = oracle.materialize(oracle.params(wl), h, 9)
    np.testing.assert_array_equal(cell, rc)
    np.testing.assert_array_equal(M, rM)
    po = oracle.params(wl)
    for j in (0, 1, 2, 3, 17, P - 1):
        gid = base + j
        w = oracle.philox((gid >> 2, 9, 2, po.sim), (po.seed & 0xFFFFFFFF, po.seed >> 32))
        assert f[j] == oracle.u24(int(w[gid & 3]))
    with pytest.raises(wmc.WmcError):
        wmc.set_id_base(p, ws, 1 << 32)
