"""The batched form (many simulations, one launch per phase) against each
simulation run alone through wmc_run, which the parity suite pins to the
oracle; plus the oracle directly where the kernel values do not enter."""
import numpy as np
import pytest

import oracle
import wmc_inputs as wi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wmc():
    from paper_1806_00082_gb300 import build, wmc as w
    build.build()
    w.load()
    return w


def _batch(wmc, wls):
    ps = wmc.params_array([wmc.Params.of(w) for w in wls])
    co, ho = wmc.batch_layout(ps)
    V = np.concatenate([wi.potential(w) for w in wls]).astype(np.float32)
    H = np.concatenate([wi.initial_histogram(w).reshape(-1) for w in wls]).astype(np.int32)
    return ps, co, ho, V, H


def _run_batch(wmc, ps, V, H, t_first, n_steps, per=0, use_graph=True):
    ws = wmc.batch_workspace(ps)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        wmc.batch_init(ps, ws)
        Vd = torch.from_numpy(V).cuda()
        a = torch.from_numpy(H).cuda()
        b = torch.empty_like(a)
        wmc.batch_run(ps, Vd, a, b, t_first, n_steps, ws, per_thread=per, use_graph=use_graph)
        c = wmc.batch_get_counters(ps, ws)
    s.synchronize()
    return a.cpu().numpy(), c


def _run_alone(wmc, w, t_first, n_steps):
    from tests._util import gpu_run
    return gpu_run(wmc, torch, wmc.Params.of(w), wi.potential(w), wi.initial_histogram(w), t_first, n_steps)


def test_batch_equals_each_simulation_alone(wmc):
    wls = wi.batch_workloads(12, seed=7, n_x_range=(120, 700), n0_range=(5_000, 60_000))
    # two packets next to their barriers, so that pairs are created
    wls[3] = wls[3].replace(packet=wi.Packet(wls[3].length_m / 2 - 12e-9, 4e-9, 0.1, 40_000))
    wls[8] = wls[8].replace(packet=wi.Packet(wls[8].length_m / 2 + 10e-9, 4e-9, 0.2, 30_000))
    ps, co, ho, V, H = _batch(wmc, wls)
    got, c = _run_batch(wmc, ps, V, H, 1, 9)
    total_pairs = 0
    for s, w in enumerate(wls):
        alone, ca = _run_alone(wmc, w, 1, 9)
        np.testing.assert_array_equal(got[ho[s]:ho[s + 1]].reshape(w.n_x, w.n_M), alone)
        total_pairs += ca["pairs"]
    assert c["pairs"] == total_pairs and total_pairs > 1000
    assert c["flags"] == 0


def test_batch_work_item_sizes_and_graph(wmc):
    """Every autotuner candidate and graph / direct launches give the same bits."""
    wls = wi.batch_workloads(6, seed=11, n_x_range=(100, 400), n0_range=(5_000, 40_000))
    wls[2] = wls[2].replace(packet=wi.Packet(wls[2].length_m / 2 - 8e-9, 4e-9, 0.1, 20_000))
    ps, co, ho, V, H = _batch(wmc, wls)
    ref, _ = _run_batch(wmc, ps, V, H, 3, 5, per=16)
    for per in (4, 8, 32, 64, 128, 256):
        got, _ = _run_batch(wmc, ps, V, H, 3, 5, per=per)
        np.testing.assert_array_equal(got, ref)
    got, _ = _run_batch(wmc, ps, V, H, 3, 5, per=16, use_graph=False)
    np.testing.assert_array_equal(got, ref)
    ws = wmc.batch_workspace(ps)
    wmc.batch_init(ps, ws)
    a = torch.from_numpy(H).cuda()
    scratch = torch.empty_like(a)
    best = wmc.batch_autotune(ps, torch.from_numpy(V).cuda(), a, scratch, 1, ws)
    assert best in (16, 32, 64, 128, 256)
    np.testing.assert_array_equal(a.cpu().numpy(), H)


def test_batch_matches_oracle_where_kernel_is_zero(wmc):
    """Packets farther than L_C/2 from the barrier: no pairs, so the FP32
    kernel does not enter and every simulation equals the FP64 oracle."""
    wls = wi.batch_workloads(5, seed=3, n_x_range=(800, 1200), n0_range=(20_000, 50_000))
    wls = [w.replace(packet=wi.Packet(w.length_m / 8, w.length_m / 60, w.packet.energy_ev, w.packet.n0))
           for w in wls]
    ps, co, ho, V, H = _batch(wmc, wls)
    got, c = _run_batch(wmc, ps, V, H, 1, 4)
    assert c["pairs"] == 0
    for s, w in enumerate(wls):
        ref, _ = oracle.simulate(oracle.params(w), wi.initial_histogram(w), 1, 4, V=wi.potential(w))
        np.testing.assert_array_equal(got[ho[s]:ho[s + 1]].reshape(w.n_x, w.n_M), ref)


def test_batch_with_pairs_matches_oracle_bit_exact(wmc):
    """A batch whose simulations create pairs (n_M 128 and 256, packets next to
    their barriers), every simulation compared bit for bit with the CPU oracle
    fed the FP32 kernel values of that simulation (wmc_kernel_eval, the values
    the solo and batched steps use) and the same Philox streams; the batch's
    counters equal the sums of the oracle's."""
    from tests._util import full_from_half
    wls = wi.batch_workloads(8, seed=21, n_x_range=(150, 600), n0_range=(20_000, 80_000))
    for s in range(len(wls)):
        w = wls[s]
        side = -1 if s % 2 else 1
        wls[s] = w.replace(packet=wi.Packet(w.length_m / 2 + side * 9e-9, 4e-9, 0.05 + 0.02 * (s % 3),
                                            w.packet.n0))
    assert {w.n_M for w in wls} == {128, 256}
    ps, co, ho, V, H = _batch(wmc, wls)
    steps = 6
    got, c = _run_batch(wmc, ps, V, H, 1, steps)
    tot = {"pairs": 0, "absorbed": 0, "dropped": 0, "particle_steps": 0}
    for s, w in enumerate(wls):
        p = wmc.Params.of(w)
        ws = wmc.workspace(p)
        wmc.init(p, ws)
        occ = torch.arange(w.n_x, dtype=torch.int32, device="cuda")
        half = wmc.kernel_eval(p, torch.from_numpy(wi.potential(w)).cuda(), occ, ws).cpu().numpy()
        ref, st = oracle.simulate(oracle.params(w), wi.initial_histogram(w), 1, steps,
                                  table=full_from_half(half, w.Q, w.n_M))
        np.testing.assert_array_equal(got[ho[s]:ho[s + 1]].reshape(w.n_x, w.n_M), ref)
        tot["pairs"] += int(st[oracle.ST_PAIRS])
        tot["absorbed"] += int(st[oracle.ST_ABSORBED])
        tot["dropped"] += int(st[oracle.ST_DROPPED])
        tot["particle_steps"] += int(st[oracle.ST_PARTICLE_STEPS])
    for k, v in tot.items():
        assert c[k] == v, k
    assert tot["pairs"] > 1000
