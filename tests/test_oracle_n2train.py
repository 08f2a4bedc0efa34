"""Pins of the trained N = 2 network's oracle (oracle/n2train.py, Eq. kernel_ML
with N = 2, Sec. 2.3): at its initial weights the model is the analytic N = 2
network (itself pinned in test_oracle_n2.py); its loss vanishes where N = 2 is
exact (pairwise-constant potentials against the exact kernel); its gradient
equals central differences of its loss; SGD lowers the loss on the
Gaussian-bump set."""
import numpy as np
import pytest

import oracle
import wmc_inputs as wi
from oracle import n2train as nt

N_X, Q = 64, 16


def _p(n_x=N_X, q=Q, bc=0):
    return oracle.params(wi.N2_TRAIN.replace(n_x=n_x, Q=q, n_M=q, bc_potential=bc))


def _targets(p, V, q):
    return oracle.kernel_rows(p, V, np.arange(V.shape[0]))[:, q // 2:] * nt.target_scale(q)


@pytest.mark.parametrize("bc", [0, 1])
def test_initial_model_is_the_analytic_n2_network(bc):
    V = np.random.default_rng(1).uniform(-0.2, 0.3, N_X).astype(np.float32)
    y = nt.model(nt.initial_params(Q), V, Q, bc)
    ref = oracle.kernel_rows_n2(_p(bc=bc), V, np.arange(N_X))[:, Q // 2:] * nt.target_scale(Q)
    assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max()
    assert np.all(y[:, 0] == 0.0)


def test_zero_loss_where_n2_is_exact():
    # V constant on every absolute pair (2q, 2q + 1) and zero near the edges
    V = np.zeros(N_X, np.float32)
    V[20:44] = np.repeat(np.random.default_rng(2).uniform(0.05, 0.3, 12), 2)
    p = _p()
    loss, g = nt.loss_and_grad(nt.initial_params(Q), V, _targets(p, V, Q), Q)
    T = _targets(p, V, Q)
    assert loss <= 1e-26 * (T ** 2).mean() + 1e-300
    assert np.abs(g).max() <= 1e-12 * np.abs(T).max() * np.abs(V).max()


@pytest.mark.parametrize("bc", [0, 1])
def test_gradient_equals_central_differences(bc):
    rng = np.random.default_rng(3)
    Vs = wi.gaussian_bumps(2, n_x=N_X, seed=7)
    p = _p(bc=bc)
    T = _targets(p, Vs[1], Q) * 1.01 + 0.001
    params = nt.initial_params(Q) + rng.normal(0.0, 0.05, Q + 4)
    _, g = nt.loss_and_grad(params, Vs[0], T, Q, bc)
    fd = np.empty_like(params)
    for k in range(params.size):
        e = np.zeros_like(params)
        e[k] = 1e-6
        fd[k] = (nt.loss_and_grad(params + e, Vs[0], T, Q, bc)[0] - nt.loss_and_grad(params - e, Vs[0], T, Q, bc)[0]) / 2e-6
    assert np.abs(fd - g).max() <= 1e-7 * np.abs(g).max()


def test_sgd_lowers_the_loss_on_gaussian_bumps():
    p = _p()
    Vs = wi.gaussian_bumps(8, n_x=N_X, dx_nm=0.5, seed=4)
    Ts = np.stack([_targets(p, V, Q) for V in Vs])
    order = wi.sgd_order(12, 8)
    p0 = nt.initial_params(Q)
    pf, hist = nt.train(p0, Vs, Ts, order, 3e-2, Q)
    assert hist[-1] < hist[0]
    full = lambda q: np.mean([nt.loss_and_grad(q, Vs[e], Ts[e], Q)[0] for e in range(8)])
    assert full(pf) < full(p0)
    # one step is a step along the negative gradient of the example's loss
    l0, g0 = nt.loss_and_grad(p0, Vs[order[0, 0]], Ts[order[0, 0]], Q)
    l1, _ = nt.loss_and_grad(p0 - 1e-3 * g0, Vs[order[0, 0]], Ts[order[0, 0]], Q)
    assert l1 < l0
