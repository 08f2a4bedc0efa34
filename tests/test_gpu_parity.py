"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bars: bit-exact for Philox words, CDFs built from the same FP32 kernel values,
histograms, counters and survivors (same kernel table, same Philox streams);
kernel values within 1e-6 normwise of the FP64 oracle (FP32 form); densities of
the full production loop (FP32 kernel in the loop) within 1e-3 L1 of the
oracle's FP64 run under common random numbers.
"""
import numpy as np
import pytest

import oracle
import wmc_inputs as wi
from tests._util import gpu_run, gpu_run_table, normwise, oracle_tables

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KERNEL_TOL = 1e-6       # normwise, FP32 form vs FP64 oracle
DENSITY_L1_TOL = 1e-3   # sum_i |rho_gpu - rho_oracle| / N0


@pytest.fixture(scope="module")
def wmc():
    from paper_1806_00082_gb300 import build, wmc as w
    build.build()
    w.load()
    return w


# --------------------------------------------------------------------------- Philox
def test_philox_matches_oracle(wmc):
    rng = np.random.default_rng(0)
    n = 100_000
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = (0x9E3779B9, 0xDEADBEEF)
    out = wmc.philox4x32_10(torch.from_numpy(ctr.view(np.int32)).cuda(), *key).cpu().numpy().view(np.uint32)
    for q in list(range(0, n, 997)) + [n - 1]:
        assert out[q].tolist() == oracle.philox(ctr[q], key).tolist()
    # published known-answer vector
    z = wmc.philox4x32_10(torch.zeros((1, 4), dtype=torch.int32, device="cuda"), 0, 0).cpu().numpy().view(np.uint32)
    assert z[0].tolist() == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]


# --------------------------------------------------------------------------- kernel
def _half_from_full(w, full64):
    h = w.Q // 2
    return full64[:, w.n_M // 2: w.n_M // 2 + h] if w.n_M >= w.Q else None


@pytest.mark.parametrize("wl", [wi.BARRIER_100, wi.BARRIER_2000])
def test_kernel_eval_fp32_all_cells(wmc, wl):
    p = wmc.Params.of(wl)
    V = wi.potential(wl)
    ws = wmc.workspace(p)
    wmc.init(p, ws)
    occ = torch.arange(wl.n_x, dtype=torch.int32, device="cuda")
    got = wmc.kernel_eval(p, torch.from_numpy(V).cuda(), occ, ws).cpu().numpy()
    ref = oracle.kernel_rows(oracle.params(wl.replace(n_M=wl.Q)), V, np.arange(wl.n_x))[:, wl.Q // 2:]
    assert got.shape == ref.shape
    assert normwise(got, ref) <= KERNEL_TOL
    assert np.all(got[:, 0] == 0)


def test_kernel_eval_fp32_double_barrier_sampled(wmc):
    """Q = 1024 (8 column tiles, a 511-term contraction): a ragged set of 333
    cells spread over the barrier region and the edges, with repeats."""
    wl = wi.DOUBLE_BARRIER_16384
    p = wmc.Params.of(wl)
    V = wi.potential(wl)
    ws = wmc.workspace(p)
    wmc.init(p, ws)
    rng = np.random.default_rng(7)
    cells = np.concatenate([rng.integers(8192 - 700, 8192 + 700, 300), [0, 1, 511, 512, 16383, 16382],
                            rng.integers(0, wl.n_x, 24), [8192, 8192, 8192]]).astype(np.int32)
    assert cells.size == 333
    got = wmc.kernel_eval(p, torch.from_numpy(V).cuda(), torch.from_numpy(cells).cuda(), ws).cpu().numpy()
    ref = oracle.kernel_rows(oracle.params(wl.replace(n_M=wl.Q)), V, cells)[:, wl.Q // 2:]
    e = normwise(got, ref)
    assert e <= KERNEL_TOL, e
    big = np.abs(ref) > 1e-3 * np.abs(ref).max()
    rel = np.abs(got[big] - ref[big]) / np.abs(ref[big])
    assert np.median(rel) < 1e-6


@pytest.mark.parametrize("n_occ", [0, 1, 63, 64, 65, 130])
def test_kernel_eval_ragged_and_empty(wmc, n_occ):
    wl = wi.BARRIER_2000
    p = wmc.Params.of(wl)
    V = wi.potential(wl)
    ws = wmc.workspace(p)
    wmc.init(p, ws)
    cells = (np.arange(n_occ) * 7 + 950) % wl.n_x
    out = torch.full((n_occ, wl.Q // 2), 7.0, device="cuda")
    wmc.kernel_eval(p, torch.from_numpy(V).cuda(), torch.from_numpy(cells.astype(np.int32)).cuda(), ws, out=out)
    got = out.cpu().numpy()
    if n_occ:
        ref = oracle.kernel_rows(oracle.params(wl.replace(n_M=wl.Q)), V, cells)[:, wl.Q // 2:]
        assert normwise(got, ref) <= KERNEL_TOL


def test_kernel_eval_clamp_boundary(wmc):
    """bc 1 (edge value outside the domain) on a rough potential."""
    wl = wi.BARRIER_100.replace(bc_potential=1)
    p = wmc.Params.of(wl)
    V = np.random.default_rng(3).uniform(-0.2, 0.3, wl.n_x).astype(np.float32)
    ws = wmc.workspace(p)
    wmc.init(p, ws)
    occ = torch.arange(wl.n_x, dtype=torch.int32, device="cuda")
    got = wmc.kernel_eval(p, torch.from_numpy(V).cuda(), occ, ws).cpu().numpy()
    ref = oracle.kernel_rows(oracle.params(wl.replace(n_M=wl.Q)), V, np.arange(wl.n_x))[:, wl.Q // 2:]
    assert normwise(got, ref) <= KERNEL_TOL


@pytest.mark.parametrize("wl", [wi.BARRIER_100, wi.BARRIER_2000, wi.DOUBLE_BARRIER_16384])
def test_cdf_bit_exact_on_same_kernel_values(wmc, wl):
    """gamma, the fixed-point CDF and its scale from identical FP32 kernel values
    are identical."""
    p = wmc.Params.of(wl)
    V = wi.potential(wl)
    rows = np.arange(wl.n_x) if wl.n_x <= 2000 else np.arange(8192 - 160, 8192 + 160)
    po = oracle.params(wl)
    full = oracle.kernel_rows(po, V, rows).astype(np.float32)
    half = oracle.kernel_rows(oracle.params(wl.replace(n_M=wl.Q)), V, rows)[:, wl.Q // 2:].astype(np.float32)
    cdf, gamma, scale = wmc.kernel_cdf(p, torch.from_numpy(np.ascontiguousarray(half)).cuda())
    cdf, gamma, scale = cdf.cpu().numpy(), gamma.cpu().numpy(), scale.cpu().numpy()
    npos = 0
    for r in range(rows.size):
        c_ref, g_ref, s_ref = oracle.cdf_row(full[r].astype(np.float64), with_scale=True)
        assert np.array_equal(cdf[r], c_ref)
        assert gamma[r] == g_ref
        assert scale[r] == s_ref
        npos += g_ref > 0
    assert npos > 0


@pytest.mark.parametrize("wl", [wi.BARRIER_100, wi.BARRIER_2000, wi.BARRIER_2000.replace(n_M=48),
                                wi.DOUBLE_BARRIER_16384,
                                wi.DOUBLE_BARRIER_16384.replace(n_M=1536, dt_s=0.5 * wi.DOUBLE_BARRIER_16384.dt_s)])
def test_gamma_only_bit_exact(wmc, wl):
    """gamma and the scale without the CDF (read from the folded row with
    residue multiplicities) equal the oracle's for momentum grids shorter than,
    equal to and longer than the period, including rows that are all zero."""
    p = wmc.Params.of(wl)
    V = wi.potential(wl)
    rows = np.arange(0, wl.n_x, max(1, wl.n_x // 300))
    po = oracle.params(wl)
    full = oracle.kernel_rows(po, V, rows).astype(np.float32)
    half = oracle.kernel_rows(oracle.params(wl.replace(n_M=wl.Q)), V, rows)[:, wl.Q // 2:].astype(np.float32)
    half[3] = 0.0
    full[3] = 0.0
    _, gamma, scale = wmc.kernel_cdf(p, torch.from_numpy(np.ascontiguousarray(half)).cuda(), with_cdf=False)
    gamma, scale = gamma.cpu().numpy(), scale.cpu().numpy()
    for r in range(rows.size):
        _, g_ref, s_ref = oracle.cdf_row(full[r].astype(np.float64), with_scale=True)
        assert gamma[r] == g_ref, r
        assert scale[r] == s_ref, r
    assert gamma[3] == 0.0


# --------------------------------------------------------------------------- steps, bit-exact
def _compare_steps(wmc, wl, hist0, t_first, n_steps, V=None):
    p = wmc.Params.of(wl)
    V = wi.potential(wl) if V is None else V
    full, half = oracle_tables(wl, V)
    ref, st = oracle.simulate(oracle.params(wl), hist0, t_first, n_steps, table=full)
    got, c = gpu_run_table(wmc, torch, p, half, hist0, t_first, n_steps)
    np.testing.assert_array_equal(got, ref)
    assert c["pairs"] == st[oracle.ST_PAIRS]
    assert c["absorbed"] == st[oracle.ST_ABSORBED]
    assert c["absorbed_signed"] == st[oracle.ST_ABSORBED_SIGNED]
    assert c["dropped"] == st[oracle.ST_DROPPED]
    assert c["dropped_signed"] == st[oracle.ST_DROPPED_SIGNED]
    assert c["particle_steps"] == st[oracle.ST_PARTICLE_STEPS]
    return got, c, st


def test_steps_bit_exact_barrier_100_all_steps(wmc):
    """1e5 particles, 100 steps: every histogram count and counter identical."""
    wl = wi.BARRIER_100
    _, c, st = _compare_steps(wmc, wl, wi.initial_histogram(wl), 1, wl.steps)
    assert st[oracle.ST_PAIRS] > 10000 and st[oracle.ST_DROPPED] > 1000


def test_steps_bit_exact_packet_on_barrier(wmc):
    """Packet centred on the barrier: pairs at the maximal rate, annihilation busy."""
    wl = wi.BARRIER_100.replace(packet=wi.Packet(50e-9, 6e-9, 0.1, 200_000))
    _, c, st = _compare_steps(wmc, wl, wi.initial_histogram(wl), 5, 20)
    assert st[oracle.ST_PAIRS] > 50000


def test_steps_bit_exact_pair_queue_overflow(wmc):
    """About 1.6e5 pair events per step in a 6400-bucket histogram: more than
    the step's pair queue holds (2^16 entries at this size), so events are
    completed both by the pair kernel and inside the step kernel."""
    wl = wi.BARRIER_100.replace(packet=wi.Packet(50e-9, 4e-9, 0.1, 3_000_000))
    _, c, st = _compare_steps(wmc, wl, wi.initial_histogram(wl), 1, 2)
    assert st[oracle.ST_PAIRS] > 2 * 70_000


def test_steps_bit_exact_wrap_and_clamp(wmc):
    wl = wi.BARRIER_100.replace(child_wrap=1, bc_potential=1, sim=7, seed=123456789012345,
                                packet=wi.Packet(45e-9, 6e-9, 0.12, 50_000))
    _, c, st = _compare_steps(wmc, wl, wi.initial_histogram(wl), 1, 10)
    assert st[oracle.ST_DROPPED] == 0 and st[oracle.ST_PAIRS] > 1000


def test_steps_bit_exact_signed_random_and_edges(wmc):
    """Random signed counts in every bucket, including the edge cells (absorption)."""
    wl = wi.BARRIER_100
    h0 = wi.random_histogram(wl, 300_000, seed=9)
    _, c, st = _compare_steps(wmc, wl, h0, 3, 4)
    assert st[oracle.ST_ABSORBED] > 0


def test_steps_empty_and_single(wmc):
    wl = wi.BARRIER_100
    _compare_steps(wmc, wl, np.zeros((wl.n_x, wl.n_M), np.int32), 1, 2)
    h = np.zeros((wl.n_x, wl.n_M), np.int32)
    h[49, 40] = -1
    _compare_steps(wmc, wl, h, 1, 5)
    h = np.zeros((wl.n_x, wl.n_M), np.int32)
    h[0, 0] = 5000       # fastest leftward momentum at the left edge
    h[99, 63] = -5000    # fastest rightward momentum at the right edge
    _compare_steps(wmc, wl, h, 1, 3)


def test_steps_bit_exact_large_buckets(wmc):
    """Cells with more particles than one work item: items split a cell."""
    wl = wi.BARRIER_100
    h = np.zeros((wl.n_x, wl.n_M), np.int32)
    h[44, 30:36] = 3000
    h[45, 33] = -20000
    h[46, 60] = 9000
    _compare_steps(wmc, wl, h, 2, 3)


@pytest.mark.parametrize("sizes", [(7167, 7168, 7169, 7171), (8191, 8192, 8193, 3 * 7168 + 3),
                                   (1, 2, 3, 4 * 7168 - 1)])
def test_steps_bit_exact_work_item_boundaries(wmc, sizes):
    """Cell populations around multiples of the work-item size, in cells whose
    first id is not quad-aligned (a leading odd cell), with buckets split
    across momenta and signs."""
    wl = wi.BARRIER_100
    h = np.zeros((wl.n_x, wl.n_M), np.int32)
    h[40, 5] = 3  # shifts the first id of every later cell off a multiple of four
    for j, n in enumerate(sizes):
        c = 44 + 2 * j
        h[c, 20] = n // 2
        h[c, 41] = -(n - n // 2)
    _compare_steps(wmc, wl, h, 2, 3)


def test_steps_bit_exact_barrier_2000_full_size(wmc):
    """The 2000-cell, 1e7-particle workload at full size, 2 steps."""
    wl = wi.BARRIER_2000
    _compare_steps(wmc, wl, wi.initial_histogram(wl), 1, 2)


def test_steps_bit_exact_double_barrier_near(wmc):
    """Q = n_M = 1024 with the noisy double barrier: a packet next to it."""
    wl = wi.DOUBLE_BARRIER_16384.replace(packet=wi.Packet(8192 * 0.1e-9 - 30e-9, 5e-9, 0.1, 100_000))
    V = wi.potential(wl)
    # kernel table only where particles can go (rows far away are never read)
    full = np.zeros((wl.n_x, wl.n_M), np.float32)
    half = np.zeros((wl.n_x, wl.Q // 2), np.float32)
    rows = np.arange(8192 - 600, 8192 + 200)
    full[rows] = oracle.kernel_rows(oracle.params(wl), V, rows).astype(np.float32)
    half[rows] = oracle.kernel_rows(oracle.params(wl.replace(n_M=wl.Q)), V, rows)[:, wl.Q // 2:].astype(np.float32)
    h0 = wi.initial_histogram(wl)
    assert np.all(np.abs(h0).sum(axis=1)[:8192 - 590] == 0) and np.all(np.abs(h0).sum(axis=1)[8192 + 190:] == 0)
    ref, st = oracle.simulate(oracle.params(wl), h0, 1, 3, table=full)
    got, c = gpu_run_table(wmc, torch, wmc.Params.of(wl), half, h0, 1, 3)
    np.testing.assert_array_equal(got, ref)
    assert c["pairs"] == st[oracle.ST_PAIRS] > 1000


# --------------------------------------------------------------------------- production loop
def test_production_loop_density_barrier_100(wmc):
    """wmc_run (FP32 kernel in the loop, CUDA graph) vs the oracle's FP64 run:
    same seeds and counters, so densities agree within 1e-3 L1."""
    wl = wi.BARRIER_100
    p = wmc.Params.of(wl)
    V = wi.potential(wl)
    h0 = wi.initial_histogram(wl)
    ref, st = oracle.simulate(oracle.params(wl), h0, 1, wl.steps, V=V)
    got, c = gpu_run(wmc, torch, p, V, h0, 1, wl.steps, use_graph=True)
    rho_g, rho_o = got.sum(axis=1), ref.sum(axis=1)
    l1 = np.abs(rho_g - rho_o).sum() / wl.packet.n0
    assert l1 <= DENSITY_L1_TOL, l1
    assert c["flags"] == 0
    assert abs(int(c["pairs"]) - int(st[oracle.ST_PAIRS])) <= 0.01 * st[oracle.ST_PAIRS]
    # graph and direct launches give the same bits
    got2, _ = gpu_run(wmc, torch, p, V, h0, 1, wl.steps, use_graph=False)
    np.testing.assert_array_equal(got, got2)


def test_production_loop_equals_table_path_on_its_own_kernel(wmc):
    """wmc_run (kernel rows at the cell index where the reach bits need them,
    the plan on a second stream) and the call-by-call table path (rows at the
    occupied-list index) fed the same FP32 kernel values give the same
    histogram and counters; the packet sits on the barrier so pairs are
    created every step."""
    from tests._util import gpu_run_table
    wl = wi.BARRIER_100.replace(packet=wi.Packet(50e-9, 6e-9, 0.1, 200_000))
    p = wmc.Params.of(wl)
    V = wi.potential(wl)
    h0 = wi.initial_histogram(wl)
    ws = wmc.workspace(p)
    wmc.init(p, ws)
    occ = torch.arange(wl.n_x, dtype=torch.int32, device="cuda")
    tab = wmc.kernel_eval(p, torch.from_numpy(V).cuda(), occ, ws).cpu().numpy()
    got_t, ct = gpu_run_table(wmc, torch, p, tab, h0, 1, 12)
    got_r, cr = gpu_run(wmc, torch, p, V, h0, 1, 12)
    np.testing.assert_array_equal(got_r, got_t)
    for key in ("pairs", "absorbed", "absorbed_signed", "dropped", "dropped_signed", "particle_steps"):
        assert cr[key] == ct[key], key
    assert cr["pairs"] > 1000


def test_production_loop_barrier_2000_matches_oracle(wmc):
    """At the 2000-cell workload the packet is farther than L_C / 2 from the
    barrier, so the occupied cells have a zero kernel in both precisions and the
    production loop matches the oracle bit for bit."""
    wl = wi.BARRIER_2000
    p = wmc.Params.of(wl)
    V = wi.potential(wl)
    h0 = wi.initial_histogram(wl)
    ref, st = oracle.simulate(oracle.params(wl), h0, 1, 3, V=V)
    got, c = gpu_run(wmc, torch, p, V, h0, 1, 3)
    np.testing.assert_array_equal(got, ref)
    assert c["particle_steps"] == st[oracle.ST_PARTICLE_STEPS]


def test_odd_step_count_and_continuation(wmc):
    """7 steps in one call equal 3 + 4 steps (state and Philox counters resume)."""
    wl = wi.BARRIER_100.replace(packet=wi.Packet(45e-9, 5e-9, 0.1, 50_000))
    p = wmc.Params.of(wl)
    V = wi.potential(wl)
    h0 = wi.initial_histogram(wl)
    a, _ = gpu_run(wmc, torch, p, V, h0, 1, 7)
    b1, _ = gpu_run(wmc, torch, p, V, h0, 1, 3)
    b2, _ = gpu_run(wmc, torch, p, V, b1, 4, 4)
    np.testing.assert_array_equal(a, b2)
    a_direct, _ = gpu_run(wmc, torch, p, V, h0, 1, 7, use_graph=False)
    np.testing.assert_array_equal(a, a_direct)
    # seven one-step calls on one workspace (the cached odd-step graph is reused
    # with a new first step each time)
    ws = wmc.workspace(p)
    wmc.init(p, ws)
    Vd = torch.from_numpy(V).cuda()
    x = torch.from_numpy(h0).cuda()
    y = torch.empty_like(x)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for t in range(1, 8):
            wmc.run(p, Vd, x, y, t, 1, ws, wmc.FP32, True)
    s.synchronize()
    np.testing.assert_array_equal(x.cpu().numpy(), a)


def test_graph_cache_alternating_buffer_sets(wmc):
    """Five buffer sets stepped in turn on one workspace and stream (more sets
    than cached graphs per kind, so slots are reused and recaptured): after
    three rounds of three steps every set holds the nine-step state of the
    direct call sequence."""
    wl = wi.BARRIER_100.replace(packet=wi.Packet(45e-9, 5e-9, 0.1, 50_000))
    p = wmc.Params.of(wl)
    V = wi.potential(wl)
    h0 = wi.initial_histogram(wl)
    ref, _ = gpu_run(wmc, torch, p, V, h0, 1, 9, use_graph=False)
    ws = wmc.workspace(p)
    wmc.init(p, ws)
    Vd = torch.from_numpy(np.ascontiguousarray(V, dtype=np.float32)).cuda()
    x0 = torch.from_numpy(np.ascontiguousarray(h0, dtype=np.int32)).cuda()
    sets = [(x0.clone(), torch.empty_like(x0)) for _ in range(5)]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for rnd in range(3):
            for a, b in sets:
                wmc.run(p, Vd, a, b, 1 + 3 * rnd, 3, ws, wmc.FP32, True)
    s.synchronize()
    for a, _ in sets:
        np.testing.assert_array_equal(a.cpu().numpy(), ref)


def test_step_timing_events_change_nothing(wmc):
    """The library's events around the particle-step kernel (graph nodes in the
    cached step graph, plain records on the direct path) leave every result
    bit-identical and bracket a positive duration."""
    wl = wi.BARRIER_100.replace(packet=wi.Packet(45e-9, 5e-9, 0.1, 50_000))
    p = wmc.Params.of(wl)
    V = wi.potential(wl)
    h0 = wi.initial_histogram(wl)
    ref, c_ref = gpu_run(wmc, torch, p, V, h0, 1, 6)
    wmc.step_timing(True)
    try:
        got_graph, c_graph = gpu_run(wmc, torch, p, V, h0, 1, 6)
        ms_graph = wmc.step_timing_read()
        got_direct, _ = gpu_run(wmc, torch, p, V, h0, 1, 5, use_graph=False)
        ms_direct = wmc.step_timing_read()
    finally:
        wmc.step_timing(False)
    np.testing.assert_array_equal(got_graph, ref)
    assert c_graph["pairs"] == c_ref["pairs"] and c_graph["particle_steps"] == c_ref["particle_steps"]
    ref5, _ = gpu_run(wmc, torch, p, V, h0, 1, 5, use_graph=False)
    np.testing.assert_array_equal(got_direct, ref5)
    assert 0.0 < ms_graph < 100.0 and 0.0 < ms_direct < 100.0


# --------------------------------------------------------------------------- rebuild, density, flags
def test_materialize_matches_oracle(wmc):
    wl = wi.BARRIER_100
    p = wmc.Params.of(wl)
    h = wi.random_histogram(wl, 40_000, seed=12)
    ws = wmc.workspace(p)
    wmc.init(p, ws)
    hd = torch.from_numpy(h).cuda()
    rho = torch.empty(wl.n_x, dtype=torch.int64, device="cuda")
    wmc.annihilate(p, hd, ws, rho=rho)
    P = int(np.abs(h).sum())
    cell, f, M, s = (x.cpu().numpy() for x in wmc.materialize(p, hd, 17, ws, P))
    rc, rf, rM, rs = oracle.materialize(oracle.params(wl), h, 17)
    np.testing.assert_array_equal(cell, rc)
    np.testing.assert_array_equal(f, rf)
    np.testing.assert_array_equal(M, rM)
    np.testing.assert_array_equal(s, rs)
    np.testing.assert_array_equal(rho.cpu().numpy(), oracle.density(oracle.params(wl), h))
    np.testing.assert_array_equal(wmc.density(p, hd).cpu().numpy(), h.sum(axis=1))
    assert wmc.get_counters(p, ws)["population"] == P
    # too small a capacity: nothing written, flag set
    wmc.materialize(p, hd, 17, ws, P - 1)
    assert wmc.get_counters(p, ws)["flags"] & wmc.FLAG_CAPACITY


def test_bounded_wait_timeout_is_reported_and_context_survives(wmc):
    """Failure detection without a fault: a device wait on a word nothing sets
    gives up after its cycle budget and raises the timeout flag; the flag is
    cleared by a counter reset, a wait on a set word passes, and the next
    kernel call on the same context is correct."""
    wl = wi.BARRIER_100
    p = wmc.Params.of(wl)
    ws = wmc.workspace(p)
    wmc.init(p, ws)
    sig = torch.zeros(1, dtype=torch.int32, device="cuda")
    wmc.check_wait(p, sig, 2_000_000, ws)  # about a millisecond
    assert wmc.get_counters(p, ws)["flags"] & wmc.FLAG_TIMEOUT
    wmc.reset_counters(p, ws)
    assert wmc.get_counters(p, ws)["flags"] == 0
    sig.fill_(1)
    wmc.check_wait(p, sig, 2_000_000, ws)
    assert wmc.get_counters(p, ws)["flags"] == 0
    V = wi.potential(wl)
    occ = torch.arange(wl.n_x, dtype=torch.int32, device="cuda")
    got = wmc.kernel_eval(p, torch.from_numpy(V).cuda(), occ, ws).cpu().numpy()
    ref = oracle.kernel_rows(oracle.params(wl.replace(n_M=wl.Q)), V, np.arange(wl.n_x))[:, wl.Q // 2:]
    assert normwise(got, ref) <= KERNEL_TOL


def test_rate_flag(wmc):
    """gamma dt >= 1 is flagged, never clamped silently."""
    wl = wi.BARRIER_100.replace(dt_s=2e-15)
    p = wmc.Params.of(wl)
    V = wi.potential(wl) * 50
    h0 = wi.initial_histogram(wl.replace(packet=wi.Packet(50e-9, 3e-9, 0.1, 1000)))
    _, c = gpu_run(wmc, torch, p, V, h0, 1, 1)
    assert c["flags"] & wmc.FLAG_RATE


def test_get_error_maps_device_flags(wmc):
    """wmc_get_error: no condition after a clean run, the rate condition after
    gamma dt >= 1, the timeout condition after a bounded wait gives up (the
    timeout takes precedence), and nothing after a counter reset."""
    wl = wi.BARRIER_100.replace(dt_s=2e-15)
    p = wmc.Params.of(wl)
    ws = wmc.workspace(p)
    wmc.init(p, ws)
    code, msg = wmc.get_error(p, ws)
    assert code == 0 and msg
    V = torch.from_numpy(wi.potential(wl) * 50).cuda()
    a = torch.from_numpy(wi.initial_histogram(wl.replace(packet=wi.Packet(50e-9, 3e-9, 0.1, 1000)))).cuda()
    b = torch.empty_like(a)
    wmc.run(p, V, a, b, 1, 1, ws, wmc.FP32, False)
    code, msg = wmc.get_error(p, ws)
    assert code == 3 and "gamma" in msg          # WMC_ERR_RATE
    sig = torch.zeros(1, dtype=torch.int32, device="cuda")
    wmc.check_wait(p, sig, 1_000_000, ws)
    code, _ = wmc.get_error(p, ws)
    assert code == 5                              # WMC_ERR_TIMEOUT
    wmc.reset_counters(p, ws)
    assert wmc.get_error(p, ws)[0] == 0


def test_philox_throughput_probe_folds_the_generator(wmc):
    """The throughput probe evaluates exactly the calls it claims: thread g
    folds the words of counters (q, 1, 2, 0) and (q, 2, 1, 0), q = g + j G."""
    out = torch.empty(512, dtype=torch.int32, device="cuda")
    wmc.philox_throughput(out, 3, key0=0x1234, key1=0xabcdef)
    got = out.cpu().numpy().view(np.uint32)
    G = out.numel()
    for g in (0, 1, 257, 511):
        acc = 0
        for j in range(3):
            q = g + j * G
            for ctr in ((q, 1, 2, 0), (q, 2, 1, 0)):
                for wv in oracle.philox(ctr, (0x1234, 0xabcdef)):
                    acc ^= int(wv)
        assert int(got[g]) == acc
