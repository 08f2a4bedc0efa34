"""Pins of the FP64 adjoint oracle by central finite differences of the oracle
forward (the potential builder, the kernel of Eq. (wigner-1d-discrete) and
gamma of Eq. (momentum_integral))."""
import numpy as np

import oracle
from oracle import adjoint as adj
import wmc_inputs as wi


def test_potential_vjp_matches_finite_differences():
    nb, ns, eps = 4, 3, 0.5
    n_x, dx = 200, 0.25
    th = wi.tanh_parameters(1, n_x=n_x, dx_nm=dx, n_barriers=nb, n_segments=ns, seed=5)[0].astype(np.float64)
    vb = np.random.default_rng(1).normal(size=n_x)
    got = adj.potential_tanh_vjp(th, vb, n_x, dx, nb, ns, eps)
    for j in range(th.size):
        hstep = 1e-6 * max(1.0, abs(th[j]))
        tp, tm = th.copy(), th.copy()
        tp[j] += hstep
        tm[j] -= hstep
        fd = (vb @ adj.potential_tanh(tp, n_x, dx, nb, ns, eps) - vb @ adj.potential_tanh(tm, n_x, dx, nb, ns, eps)) / (2 * hstep)
        assert abs(fd - got[j]) <= 1e-6 * max(1.0, abs(fd)), (j, fd, got[j])


def test_kernel_vjp_matches_finite_differences():
    """L = sum gVW V_W(i; r) + sum g_gamma gamma(i) on a small random potential."""
    w = wi.Workload(name="t", n_x=60, dx_m=1e-9, Q=16, n_M=32, dt_s=1e-16, steps=1)
    p = oracle.params(w)
    h = w.Q // 2
    rng = np.random.default_rng(2)
    V = rng.uniform(-0.2, 0.3, w.n_x)
    gv = rng.normal(size=(w.n_x, h)) * 1e-14
    gg = rng.normal(size=w.n_x) * 1e-14
    ph = oracle.params(w.replace(n_M=w.Q))

    def loss(Vx):
        half = oracle.kernel_rows(ph, Vx, np.arange(w.n_x))[:, h:]
        full = oracle.kernel_rows(p, Vx, np.arange(w.n_x))
        gam = np.maximum(full, 0).sum(axis=1)
        return np.sum(gv * half) + np.sum(gg * gam), full

    got = adj.kernel_vjp(p, V, gv, gg)
    _, full = loss(V)
    step = 1e-7
    checked = 0
    for l in range(w.n_x):
        Vp, Vm = V.copy(), V.copy()
        Vp[l] += step
        Vm[l] -= step
        # skip probes whose perturbation moves a kernel value across zero (gamma's kink)
        dfull = np.abs(oracle.kernel_rows(p, Vp, np.arange(w.n_x)) - full)
        if np.any((np.abs(full) < 10 * dfull) & (full != 0)):
            continue
        fd = (loss(Vp)[0] - loss(Vm)[0]) / (2 * step)
        assert abs(fd - got[l]) <= 1e-6 * np.max(np.abs(got)), (l, fd, got[l])
        checked += 1
    assert checked > w.n_x // 2
