"""Pins of the CPU oracle against values fixed by the paper and by mathematics.

Every check here is independent of the oracle's own code: closed forms written
from their own derivation, a library routine (scipy's DST-I), the paper's
network form with its analytic weight w_l (Sec. 2.2), published Philox
known-answer vectors, exact invariants, and statistical laws of the postulate
(Sec. 2.1).  A dropped term, a wrong sign, index or prefactor in the oracle
fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
import scipy.fft

import oracle
import wmc_inputs as wi

HBAR_EVS = 6.582119569e-16
HBAR_JS = 1.054571817e-34
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _p(n_x=100, Q=32, n_M=64, dx=1e-9, bc=0, dt=0.1e-15, seed=0, wrap=0, sim=0):
    w = wi.Workload(name="t", n_x=n_x, dx_m=dx, Q=Q, n_M=n_M, dt_s=dt, steps=1, seed=seed,
                    bc_potential=bc, child_wrap=wrap, sim=sim)
    return oracle.params(w)


def _normwise(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


# --------------------------------------------------------------------------- Philox
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert oracle.philox(v[0:4], v[4:6]).tolist() == v[6:10]


def test_uniform_conversions_exact():
    assert oracle.u53(0, 0) == 0.0
    assert oracle.u53(0xFFFFFFFF, 0xFFFFFFFF) == (2.0 ** 53 - 1) / 2.0 ** 53
    assert oracle.u53(1 << 5, 0) == 2.0 ** 26 / 2.0 ** 53
    assert oracle.u53(0, 1 << 6) == 2.0 ** -53
    assert oracle.u24(0xFFFFFFFF) == np.float32(1 - 2.0 ** -24)
    assert oracle.u24(0x100) == np.float32(2.0 ** -24)
    assert oracle.u24(0xFF) == 0.0
    assert oracle.u32(0) == 0.0 and oracle.u32(1) == 2.0 ** -32
    assert oracle.u32(0xFFFFFFFF) == 1 - 2.0 ** -32


# --------------------------------------------------------------------------- sine table
@pytest.mark.parametrize("Q", [2, 6, 8, 32, 128, 1000, 1024])
def test_sine_table(Q):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    t = np.arange(-3 * Q, 3 * Q)
    s = np.array([oracle.sine(Q, int(x)) for x in t])
    ref = np.array([float(mpmath.sin(2 * mpmath.pi * int(x) / Q)) for x in t])
    # within about one unit in the last place of the correctly rounded value
    assert np.max(np.abs(s - ref)) <= 2.3e-16
    # exact symmetries of the integer-indexed table
    for x in range(-Q, Q):
        assert oracle.sine(Q, -x) == -oracle.sine(Q, x) or oracle.sine(Q, x) == 0.0
        assert oracle.sine(Q, x + Q) == oracle.sine(Q, x)
    assert oracle.sine(Q, 0) == 0.0 and oracle.sine(Q, Q // 2) == 0.0


# --------------------------------------------------------------------------- kernel closed forms
def test_kernel_rows_equal_single_value_sum():
    """The row routine (sine values and differences looked up from per-call
    tables) gives bit-for-bit the single-value sum of Eq. (wigner-1d-discrete)
    term by term, for n_M below, at and above the period, both boundary modes
    and rows at and beyond the window edges."""
    rng = np.random.default_rng(11)
    for n_x, Q, n_M, bc in [(40, 8, 8, 0), (60, 16, 48, 1), (90, 32, 64, 0), (70, 30, 20, 1)]:
        p = _p(n_x=n_x, Q=Q, n_M=n_M, bc=bc)
        V = rng.uniform(-0.3, 0.3, n_x)
        rows = np.array([0, 1, Q // 2 - 1, Q // 2, n_x // 2, n_x - 2, n_x - 1])
        got = oracle.kernel_rows(p, V, rows)
        for r, i in enumerate(rows):
            for k in range(n_M):
                assert got[r, k] == oracle.kernel_value(p, V, int(i), k - n_M // 2), (n_x, Q, n_M, bc, i, k)


def _dirichlet_sine_sum(p, q, phi):
    """sum_{m=p}^{q} sin(m phi) in closed form."""
    if p > q:
        return 0.0
    return (math.cos((p - 0.5) * phi) - math.cos((q + 0.5) * phi)) / (2.0 * math.sin(phi / 2.0))


def test_kernel_rectangular_barrier_closed_form():
    """Barrier of height V0 on cells [a, b], zero outside: the window sum of the
    kernel reduces to two finite sine sums with a closed form."""
    w = wi.BARRIER_100
    p = oracle.params(w)
    V = wi.potential(w)
    a, b = 47, 52
    V0 = float(np.float32(0.2))
    assert np.all(V[a:b + 1] == np.float32(0.2)) and np.count_nonzero(V) == 6
    h = w.Q // 2
    rows = np.arange(w.n_x)
    got = oracle.kernel_rows(p, V, rows)
    ref = np.zeros_like(got)
    c = -2.0 / (HBAR_EVS * w.Q)
    for i in rows:
        for k in range(w.n_M):
            M = k - w.n_M // 2
            if M % w.Q == 0:
                continue
            phi = 2 * math.pi * M / w.Q
            s1 = _dirichlet_sine_sum(max(a - i, 1), min(b - i, h - 1), phi)
            s2 = _dirichlet_sine_sum(max(i - b, 1), min(i - a, h - 1), phi)
            ref[i, k] = c * V0 * (s1 - s2)
    assert _normwise(got, ref) < 1e-12


def test_kernel_gaussian_bump_closed_form():
    """A Gaussian bump V0 exp(-(x - xc)^2 / s^2) far inside the window has the
    continuous transform (2 / (hbar L_C)) V0 s sqrt(pi) exp(-k^2 s^2) sin(2 k (x - xc)),
    k = M pi / L_C; the window sum is the trapezoidal rule of that integral and
    is spectrally accurate for |M| < Q/2."""
    n_x, dx, Q = 256, 1e-9, 128
    p = _p(n_x=n_x, Q=Q, n_M=Q, dx=dx)
    s, V0, xc = 4e-9, 0.3, 128.3e-9
    x = (np.arange(n_x) + 0.5) * dx
    V = V0 * np.exp(-((x - xc) / s) ** 2)
    L_C = Q * dx
    rows = [i for i in range(n_x) if abs(x[i] - xc) + 5 * s < L_C / 2]
    assert len(rows) > 50
    got = oracle.kernel_rows(p, V, rows)
    Ms = np.arange(Q) - Q // 2
    k = Ms * math.pi / L_C
    ref = (2.0 / (HBAR_EVS * L_C)) * V0 * s * math.sqrt(math.pi) * np.exp(-(k * s) ** 2) \
        * np.sin(2 * np.outer(x[rows] - xc, k))
    inside = np.abs(Ms) < Q // 2
    assert _normwise(got[:, inside], ref[:, inside]) < 1e-9


def test_kernel_linear_potential_closed_form():
    """V = a x: V(i+m) - V(i-m) = 2 a m dx, so interior rows all equal
    c 2 a dx sum_{m=1}^{h-1} m sin(m phi), whose closed form is
    [h sin((h-1) phi) - (h-1) sin(h phi)] / (4 sin^2(phi/2))."""
    n_x, dx, Q = 200, 0.5e-9, 64
    p = _p(n_x=n_x, Q=Q, n_M=2 * Q, dx=dx)
    h = Q // 2
    slope = 1e7  # eV/m
    x = (np.arange(n_x) + 0.5) * dx
    V = slope * x
    rows = list(range(h, n_x - h))
    got = oracle.kernel_rows(p, V, rows)
    c = -2.0 / (HBAR_EVS * Q)
    ref = np.zeros(2 * Q)
    for kk in range(2 * Q):
        M = kk - Q
        if M % Q == 0:
            continue
        phi = 2 * math.pi * M / Q
        n = h - 1
        ref[kk] = c * 2 * slope * dx * ((n + 1) * math.sin(n * phi) - n * math.sin((n + 1) * phi)) \
            / (4 * math.sin(phi / 2) ** 2)
    assert _normwise(got, np.broadcast_to(ref, got.shape)) < 1e-11


def test_kernel_is_dst1_of_potential_differences():
    """For 0 < M < Q/2 a kernel row is a type-I discrete sine transform of
    dV(m) = V(i+m) - V(i-m), m = 1..h-1 (scipy.fft.dst, type 1)."""
    rng = np.random.default_rng(5)
    n_x, Q = 300, 64
    h = Q // 2
    p = _p(n_x=n_x, Q=Q, n_M=Q, dx=1e-9, bc=1)
    V = rng.normal(size=n_x).astype(np.float32).astype(np.float64)
    rows = rng.integers(0, n_x, size=25)
    got = oracle.kernel_rows(p, V, rows)
    Vp = np.concatenate([np.full(h, V[0]), V, np.full(h, V[-1])])   # clamp outside
    for r, i in enumerate(rows):
        m = np.arange(1, h)
        dV = Vp[i + h + m] - Vp[i + h - m]
        y = scipy.fft.dst(dV, type=1) / 2.0
        ref = (-2.0 / (HBAR_EVS * Q)) * y
        # columns k = M + Q/2 for M = 1 .. h-1
        assert _normwise(got[r, Q // 2 + 1: Q // 2 + h], ref) < 1e-12


def test_kernel_equals_analytic_network():
    """Sec. 2.2: the N = 1 network with angles theta_l(i, j) = 2 (l - i) dx j dp / hbar,
    dp = pi hbar / L_C, hidden units V_l sin(theta_l) and output weights
    w_l = -2 dx / (hbar L_C) gives the same kernel as the discrete sum."""
    rng = np.random.default_rng(11)
    n_x, Q, dx = 16, 8, 2e-9
    L_C = Q * dx
    h = Q // 2
    p = _p(n_x=n_x, Q=Q, n_M=2 * Q, dx=dx, bc=0)
    V = rng.uniform(-0.3, 0.3, size=n_x)
    dp = math.pi * HBAR_JS / L_C
    w_l = -2 * dx / (HBAR_EVS * L_C)
    got = oracle.kernel_rows(p, V, np.arange(n_x))
    ref = np.zeros_like(got)
    for i in range(n_x):
        for kk in range(2 * Q):
            j = kk - Q
            acc = 0.0
            for l in range(i - h, i + h + 1):
                Vl = V[l] if 0 <= l < n_x else 0.0
                theta = 2 * (l - i) * dx * j * dp / HBAR_JS
                acc += w_l * Vl * math.sin(theta)
            ref[i, kk] = acc
    assert _normwise(got, ref) < 1e-12


# --------------------------------------------------------------------------- kernel invariants
def test_kernel_invariants():
    rng = np.random.default_rng(2)
    n_x, Q = 120, 32
    h = Q // 2
    p = _p(n_x=n_x, Q=Q, n_M=4 * Q, bc=0)
    V1 = rng.uniform(0, 0.3, n_x)
    V2 = rng.uniform(-0.1, 0.1, n_x)
    K1 = oracle.kernel_rows(p, V1, np.arange(n_x))
    Ms = np.arange(4 * Q) - 2 * Q
    col = {M: k for k, M in enumerate(Ms)}
    for M in range(-2 * Q + 1, 2 * Q):
        assert np.array_equal(K1[:, col[M]], -K1[:, col[-M]]) or M == 0   # antisymmetry
    for M in range(-2 * Q, Q):
        assert np.array_equal(K1[:, col[M]], K1[:, col[M + Q]])           # period Q
    assert np.all(K1[:, col[0]] == 0) and np.all(K1[:, col[h]] == 0)
    # linearity
    K2 = oracle.kernel_rows(p, V2, np.arange(n_x))
    K12 = oracle.kernel_rows(p, 2.0 * V1 - 3.0 * V2, np.arange(n_x))
    assert _normwise(K12, 2.0 * K1 - 3.0 * K2) < 1e-13
    # V -> -V flips the kernel exactly
    assert np.array_equal(oracle.kernel_rows(p, -V1, np.arange(n_x)), -K1)
    # translation by s cells shifts interior rows
    s = 7
    Vs = np.roll(V1, s)
    Vs[:s] = 0
    V1z = V1.copy()
    V1z[n_x - s:] = 0
    Ka = oracle.kernel_rows(p, V1z, np.arange(n_x))
    Kb = oracle.kernel_rows(p, Vs, np.arange(n_x))
    assert _normwise(Kb[s:], Ka[:n_x - s]) < 1e-14
    # a constant potential has a zero kernel everywhere under the clamp
    # condition, and on interior cells when V = 0 outside
    pc = _p(n_x=n_x, Q=Q, n_M=2 * Q, bc=1)
    assert np.all(oracle.kernel_rows(pc, np.full(n_x, 0.17), np.arange(n_x)) == 0)
    Kz = oracle.kernel_rows(_p(n_x=n_x, Q=Q, n_M=2 * Q, bc=0), np.full(n_x, 0.17), np.arange(n_x))
    assert np.all(Kz[h - 1:n_x - h + 1] == 0) and np.any(Kz[0] != 0)


def test_gamma_even_in_potential_and_cdf():
    w = wi.BARRIER_100
    p = oracle.params(w)
    V = wi.potential(w).astype(np.float64)
    K = oracle.kernel_rows(p, V, np.arange(w.n_x))
    Kn = oracle.kernel_rows(p, -V, np.arange(w.n_x))
    for i in range(0, w.n_x, 3):
        cdf, g, sc = oracle.cdf_row(K[i], with_scale=True)
        _, gn = oracle.cdf_row(Kn[i])
        assert np.all(np.diff(cdf) >= 0)
        assert cdf[-1] < 2 ** 62
        assert g == math.ldexp(float(cdf[-1]), -sc)
        # gamma is the sum of V_W^+ to within the fixed-point resolution
        assert abs(g - math.fsum(np.maximum(K[i], 0))) <= 1e-14 * max(g, 1)
        # each CDF increment is the positive part in units of 2^-s
        inc = np.diff(np.concatenate([[0], cdf])).astype(np.float64)
        pos = np.maximum(K[i], 0)
        if g > 0:
            assert np.all(np.abs(np.ldexp(inc, -sc) - pos) <= np.ldexp(0.5, -sc))
        # V -> -V mirrors the positive parts in M: the exact sums are equal
        assert g == gn
    # far from the barrier (beyond L_C / 2 from it) the kernel and gamma vanish
    _, g0 = oracle.cdf_row(K[5])
    assert g0 == 0.0


def test_momentum_sampling_law():
    """p' is drawn with probability V_W^+(p') / gamma (postulate): chi-square."""
    w = wi.BARRIER_100
    p = oracle.params(w)
    V = wi.potential(w)
    row = oracle.kernel_rows(p, V, [44])[0]
    cdf, g = oracle.cdf_row(row)
    rng = np.random.default_rng(3)
    n = 40000
    counts = np.zeros(w.n_M)
    for U2 in rng.integers(0, 2 ** 53, size=n, dtype=np.uint64):
        counts[oracle.sample_row(cdf, int(U2))] += 1
    prob = np.maximum(row, 0) / g
    assert np.all(counts[prob == 0] == 0)
    sel = prob * n > 5
    chi2 = np.sum((counts[sel] - n * prob[sel]) ** 2 / (n * prob[sel]))
    dof = sel.sum() - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof)
    # the extreme uniforms land on the first and last positive entries
    pos = np.nonzero(row > 0)[0]
    assert oracle.sample_row(cdf, 0) == pos[0]
    assert oracle.sample_row(cdf, 2 ** 53 - 1) == pos[-1]


def test_drift_is_free_flight():
    """D[M] dx / dt is the free-particle velocity hbar M dk / m, dk = pi / L_C."""
    w = wi.BARRIER_2000
    p = oracle.params(w)
    D = oracle.drift_table(p)
    Ms = np.arange(w.n_M) - w.n_M // 2
    v = HBAR_JS * Ms * (math.pi / (w.Q * w.dx_m)) / w.mass_kg
    ref = v * w.dt_s / w.dx_m
    assert np.all(np.abs(D - ref) <= 2 ** -23 * np.abs(ref))
    assert D[w.n_M // 2] == 0.0


# --------------------------------------------------------------------------- ensemble
def test_materialize_order_and_offsets():
    w = wi.BARRIER_100
    p = oracle.params(w)
    h = wi.random_histogram(w, 3000, seed=4)
    cell, f, M, s = oracle.materialize(p, h, step=9)
    assert cell.size == np.abs(h).sum()
    key = cell.astype(np.int64) * w.n_M + (M.astype(np.int64) + w.n_M // 2)
    assert np.all(np.diff(key) >= 0)
    np.testing.assert_array_equal(np.bincount(key, weights=s, minlength=w.n_x * w.n_M).reshape(h.shape), h)
    assert np.all((f >= 0) & (f < 1)) and np.all(f * 2 ** 24 == np.floor(f * 2 ** 24))
    # offsets: word id mod 4 of the REPOS draw of counter id / 4 at this step
    for i in [0, 1, 2, 3, 17, cell.size - 1]:
        wds = oracle.philox([i >> 2, 9, 2, 0], [w.seed & 0xFFFFFFFF, w.seed >> 32])
        assert f[i] == oracle.u24(int(wds[i & 3]))


def test_density_is_signed_row_sum():
    w = wi.BARRIER_100
    p = oracle.params(w)
    h = wi.random_histogram(w, 5000, seed=8)
    rho = oracle.density(p, h)
    np.testing.assert_array_equal(rho, h.sum(axis=1))


def test_net_sign_conservation():
    """Pairs carry +s and -s, annihilation keeps the net count per cell, so the
    net sign changes only by what leaves the domain or the momentum grid."""
    w = wi.BARRIER_100.replace(packet=wi.Packet(40e-9, 5e-9, 0.1, 20000))
    p = oracle.params(w)
    h0 = wi.initial_histogram(w)
    out, st = oracle.simulate(p, h0, 1, 30, V=wi.potential(w))
    assert st[oracle.ST_PAIRS] > 1000
    assert out.sum() == h0.sum() - st[oracle.ST_ABSORBED_SIGNED] - st[oracle.ST_DROPPED_SIGNED]
    assert st[oracle.ST_NET] == out.sum() and st[oracle.ST_POP] == np.abs(out).sum()


def test_free_drift_crossing_law():
    """V = 0: no pairs; a particle crosses to the next cell with probability |D[M]|."""
    n_x, Q, n_M = 40, 16, 32
    p = _p(n_x=n_x, Q=Q, n_M=n_M, dt=2e-15)
    D = oracle.drift_table(p)
    h0 = np.zeros((n_x, n_M), np.int32)
    kp, km = n_M // 2 + 5, n_M // 2 - 9
    n = 200000
    h0[20, kp] = n
    h0[10, km] = -n
    out, st = oracle.simulate(p, h0, 1, 1, V=np.zeros(n_x))
    assert st[oracle.ST_PAIRS] == 0
    for (i, k, sgn, dirn) in [(20, kp, 1, 1), (10, km, -1, -1)]:
        moved = sgn * out[i + dirn, k]
        stay = sgn * out[i, k]
        assert moved + stay == n
        q = abs(float(D[k]))
        z = (moved - n * q) / math.sqrt(n * q * (1 - q))
        assert abs(z) < 5, (moved, n * q)


def test_absorbing_boundary():
    n_x, Q, n_M = 30, 16, 32
    p = _p(n_x=n_x, Q=Q, n_M=n_M, dt=2e-15)
    D = oracle.drift_table(p)
    h0 = np.zeros((n_x, n_M), np.int32)
    k = 3
    n = 100000
    h0[0, k] = n
    out, st = oracle.simulate(p, h0, 1, 1, V=np.zeros(n_x))
    q = abs(float(D[k]))
    z = (st[oracle.ST_ABSORBED] - n * q) / math.sqrt(n * q * (1 - q))
    assert abs(z) < 5
    assert out.sum() == n - st[oracle.ST_ABSORBED]


def test_pair_creation_rate_and_momentum_law():
    """Particles with M = 0 do not drift; at a cell with rate gamma the number of
    pairs in one step is Binomial(n, gamma dt) and each pair puts +s at M' and
    -s at -M' with M' drawn from V_W^+ / gamma."""
    w = wi.BARRIER_100
    p = oracle.params(w)
    V = wi.potential(w)
    i = 45
    row = oracle.kernel_rows(p, V, [i])[0]
    _, g = oracle.cdf_row(row)
    q = g * w.dt_s
    assert 0.01 < q < 1
    n = 200000
    h0 = np.zeros((w.n_x, w.n_M), np.int32)
    h0[i, w.n_M // 2] = n
    out, st = oracle.simulate(p, h0, 1, 1, V=V)
    pairs = st[oracle.ST_PAIRS]
    z = (pairs - n * q) / math.sqrt(n * q * (1 - q))
    assert abs(z) < 5
    assert st[oracle.ST_DROPPED] == 0      # |M'| < n_M / 2 when the parent has M = 0
    prob = np.maximum(row, 0) / g
    plus = np.where(prob > 0, out[i], 0)
    assert plus.sum() == pairs
    # the -s children sit at -M', exactly mirrored
    for kk in np.nonzero(prob > 0)[0]:
        assert out[i, w.n_M - kk] == -out[i, kk]
    sel = prob * pairs > 5
    chi2 = np.sum((plus[sel] - pairs * prob[sel]) ** 2 / (pairs * prob[sel]))
    dof = sel.sum() - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof)


def test_single_particle_hand_trace():
    """One particle traced by hand through the counter layout: REPOS draw of
    step t-1 for the offset, GEN draw of step t for the event, PICK draw for p'."""
    w = wi.BARRIER_100
    p = oracle.params(w)
    V = wi.potential(w)
    D = oracle.drift_table(p)
    key = [w.seed & 0xFFFFFFFF, w.seed >> 32]
    for (i, k, t) in [(44, 60, 1), (46, 20, 7), (53, 40, 3)]:
        h0 = np.zeros((w.n_x, w.n_M), np.int32)
        h0[i, k] = 1
        f = np.float32(oracle.u24(int(oracle.philox([0, t - 1, 2, 0], key)[0])))
        fn = np.float32(f + D[k])
        c = i + (1 if fn >= 1 else (-1 if fn < 0 else 0))
        row = oracle.kernel_rows(p, V, [c])[0]
        cdf, g = oracle.cdf_row(row)
        wd = oracle.philox([0, t, 1, 0], key)
        expect = np.zeros_like(h0)
        expect[c, k] += 1
        if oracle.u32(int(wd[0])) < g * w.dt_s:
            wp = oracle.philox([0, t, 3, 0], key)
            kp = oracle.sample_row(cdf, oracle.u53_bits(int(wp[0]), int(wp[1])))
            for (kc, sg) in [(k + kp - w.n_M // 2, 1), (k - (kp - w.n_M // 2), -1)]:
                if 0 <= kc < w.n_M:
                    expect[c, kc] += sg
        out, _ = oracle.simulate(p, h0, t, 1, V=V)
        np.testing.assert_array_equal(out, expect)


def test_table_mode_matches_fp64_kernel_when_table_is_exact():
    """Feeding the FP64 kernel rounded to FP32 changes only rare sampling edges:
    with the rounded table the run is reproducible bit for bit."""
    w = wi.scaled(wi.BARRIER_100, 20000)
    p = oracle.params(w)
    V = wi.potential(w)
    h0 = wi.initial_histogram(w)
    table = oracle.kernel_rows(p, V, np.arange(w.n_x)).astype(np.float32)
    a, sa = oracle.simulate(p, h0, 1, 5, table=table)
    b, sb = oracle.simulate(p, h0, 1, 5, table=table)
    np.testing.assert_array_equal(a, b)
    c, _ = oracle.simulate(p, h0, 1, 5, V=V)
    assert np.abs(a - c).sum() <= 0.01 * np.abs(c).sum()
