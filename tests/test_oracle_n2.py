"""Pins of the oracle's N = 2 network (Eq. kernel_ML with N = 2 and the
barycentric weights of Sec. 2.3) against facts that do not use its code path:
the un-combined pair sum of the N = 1 network's terms (before the
sin a + sin b product identity), exact equality with the N = 1 kernel where the
potential is constant on every pair of cells, convergence to the N = 1 kernel
as dx -> 0 for a smooth potential, and exact symmetries."""
import math

import numpy as np
import pytest

import oracle
import wmc_inputs as wi

HBAR_EVS = 6.582119569e-16


def _p(n_x=64, Q=16, n_M=32, dx=1e-9, bc=0):
    return oracle.params(wi.Workload(name="t", n_x=n_x, dx_m=dx, Q=Q, n_M=n_M, dt_s=1e-16, steps=1,
                                     bc_potential=bc))


def _nw(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.mark.parametrize("bc", [0, 1])
def test_n2_equals_pairwise_averaged_network_terms(bc):
    """Brute force on a tiny grid: for each pair of cells (2q, 2q+1) inside the
    window, the pair's average potential times sin(theta_2q) + sin(theta_2q+1)
    (the network's own angles theta_l = (l - i) 2 pi M / Q), times the weight
    w = -2 / (hbar Q)."""
    n_x, Q, n_M = 14, 8, 16
    p = _p(n_x=n_x, Q=Q, n_M=n_M, bc=bc)
    V = np.random.default_rng(4).uniform(-0.3, 0.4, n_x)
    h = Q // 2

    def pot(l):
        if 0 <= l < n_x:
            return V[l]
        return 0.0 if bc == 0 else V[0 if l < 0 else n_x - 1]

    got = oracle.kernel_rows_n2(p, V, np.arange(n_x))
    w = -2.0 / (HBAR_EVS * Q)
    for i in range(n_x):
        for k in range(n_M):
            M = k - n_M // 2
            acc = 0.0
            for l in range(i - h - 1, i + h + 1):
                if l % 2 == 0 and l >= i - h and l + 1 <= i + h:
                    th0, th1 = (l - i) * 2 * math.pi * M / Q, (l + 1 - i) * 2 * math.pi * M / Q
                    acc += 0.5 * (pot(l) + pot(l + 1)) * (math.sin(th0) + math.sin(th1))
            assert abs(got[i, k] - w * acc) <= 1e-12 * abs(w) * 8, (i, k)


def test_n2_equals_n1_for_pairwise_constant_potential():
    """V(2q) = V(2q+1) for every q: the barycentric replacement changes
    nothing, so the N = 2 kernel equals the exact N = 1 kernel."""
    n_x, Q = 120, 32
    p = _p(n_x=n_x, Q=Q, n_M=2 * Q)
    V = np.repeat(np.random.default_rng(9).uniform(-0.2, 0.3, n_x // 2), 2)
    a = oracle.kernel_rows(p, V, np.arange(n_x))
    b = oracle.kernel_rows_n2(p, V, np.arange(n_x))
    assert _nw(b, a) < 1e-12
    # and generically it does not (a rough potential)
    V2 = np.random.default_rng(10).uniform(-0.2, 0.3, n_x)
    assert _nw(oracle.kernel_rows_n2(p, V2, np.arange(n_x)), oracle.kernel_rows(p, V2, np.arange(n_x))) > 0.05


def test_n2_converges_to_n1_as_dx_shrinks():
    """A Gaussian bump at a fixed coherence length L_C = 32 nm: halving dx
    (doubling Q) halves the N = 2 / N = 1 difference (first order: a pair's
    error is half the potential step across it times the difference of its two
    sines)."""
    errs = []
    for dx_nm, Q in ((1.0, 32), (0.5, 64), (0.25, 128)):
        n_x = int(round(160 / dx_nm))
        x = (np.arange(n_x) + 0.5) * dx_nm
        V = 0.25 * np.exp(-((x - 80.3) / 6.0) ** 2)
        p = _p(n_x=n_x, Q=Q, n_M=Q, dx=dx_nm * 1e-9)
        rows = np.arange(n_x // 2 - Q, n_x // 2 + Q)
        errs.append(_nw(oracle.kernel_rows_n2(p, V, rows), oracle.kernel_rows(p, V, rows)))
    assert errs[0] < 0.1
    for e0, e1 in zip(errs, errs[1:]):
        assert 1.8 < e0 / e1 < 2.2, errs


def test_n2_symmetries():
    """Odd in M, Q-periodic in M, zero at M = 0 and M = Q/2; linear in V; a
    shift of the potential by an even number of cells shifts the rows (the
    pairing is by absolute cell index)."""
    n_x, Q = 80, 16
    p = _p(n_x=n_x, Q=Q, n_M=4 * Q)
    rng = np.random.default_rng(2)
    V1, V2 = rng.uniform(-0.2, 0.2, n_x), rng.uniform(-0.2, 0.2, n_x)
    K = oracle.kernel_rows_n2(p, V1, np.arange(n_x))
    Ms = np.arange(4 * Q) - 2 * Q
    for k, M in enumerate(Ms):
        kn = np.flatnonzero(Ms == -M)
        if kn.size:
            np.testing.assert_allclose(K[:, kn[0]], -K[:, k], rtol=0, atol=1e-12 * np.abs(K).max())
        kp = np.flatnonzero(Ms == M + Q)
        if kp.size:
            np.testing.assert_allclose(K[:, kp[0]], K[:, k], rtol=0, atol=1e-12 * np.abs(K).max())
        if M % Q == 0 or M % Q == Q // 2:
            assert np.all(np.abs(K[:, k]) <= 1e-12 * np.abs(K).max())
    K2 = oracle.kernel_rows_n2(p, V2, np.arange(n_x))
    K12 = oracle.kernel_rows_n2(p, 2.0 * V1 - 3.0 * V2, np.arange(n_x))
    assert _nw(K12, 2.0 * K - 3.0 * K2) < 1e-13
    Vz = np.zeros(n_x)
    Vz[20:40] = V1[20:40]
    Vs = np.zeros(n_x)
    Vs[22:42] = V1[20:40]
    Ka = oracle.kernel_rows_n2(p, Vz, np.arange(n_x))
    Kb = oracle.kernel_rows_n2(p, Vs, np.arange(n_x))
    np.testing.assert_allclose(Kb[2:], Ka[:-2], rtol=0, atol=1e-12 * np.abs(Ka).max())


def test_n2_folded_contraction_identity():
    """The folded form the GPU contraction evaluates: with pair sums
    P(i, u) = V(i+u) + V(i+u+1), column r of the half period is
    w cos(pi r / Q) sum_{u=0}^{h-1} A(i, u) sin(pi (2u+1) r / Q), where
    A(i, u) = P(i, u) if i + u is even, else -P(i, -u-1) (a pair at offset u
    and its mirror at -u-1 have opposite sines and exactly one of them starts
    at an even cell)."""
    n_x, Q = 50, 20
    h = Q // 2
    p = _p(n_x=n_x, Q=Q, n_M=Q)
    V = np.random.default_rng(3).uniform(-0.3, 0.3, n_x)
    pot = lambda l: V[l] if 0 <= l < n_x else 0.0
    ref = oracle.kernel_rows_n2(p, V, np.arange(n_x))[:, Q // 2:]   # columns M = 0 .. h-1
    w = -2.0 / (HBAR_EVS * Q)
    for i in range(n_x):
        A = np.array([(pot(i + u) + pot(i + u + 1)) if (i + u) % 2 == 0 else -(pot(i - u - 1) + pot(i - u))
                      for u in range(h)])
        for r in range(h):
            B = np.array([math.sin(math.pi * (2 * u + 1) * r / Q) for u in range(h)])
            assert abs(w * math.cos(math.pi * r / Q) * (A @ B) - ref[i, r]) <= 1e-12 * np.abs(ref).max()
