"""The trained N = 2 network on the GPU (wmc_n2_train / wmc_n2_eval) against
the FP64 oracle (oracle/n2train.py): the model's rows at the analytic weights
and at perturbed weights, SGD trajectories of several learning rates in one
launch fed the oracle's targets (trained weights and per-epoch losses), zero
loss where N = 2 is exact, determinism."""
import numpy as np
import pytest

import oracle
import wmc_inputs as wi
from oracle import n2train as nt
from tests._util import normwise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_X, Q = 64, 16


@pytest.fixture(scope="module")
def wmc():
    from paper_1806_00082_gb300 import build, wmc as w
    build.build()
    w.load()
    return w


def _wl(n_x=N_X, q=Q, bc=0):
    return wi.N2_TRAIN.replace(n_x=n_x, Q=q, n_M=q, bc_potential=bc)


def _targets(w, Vs):
    p = oracle.params(w)
    return np.stack([oracle.kernel_rows(p, V, np.arange(w.n_x))[:, w.Q // 2:] for V in Vs]).astype(np.float32)


@pytest.mark.parametrize("bc", [0, 1])
def test_eval_at_analytic_weights_is_the_n2_network(wmc, bc):
    w = _wl(n_x=256, q=64, bc=bc)
    V = np.random.default_rng(1).uniform(-0.2, 0.3, w.n_x).astype(np.float32)
    p = wmc.Params.of(w)
    prm = torch.from_numpy(nt.initial_params(w.Q).astype(np.float32)).cuda()
    got = wmc.n2_eval(p, prm, torch.from_numpy(V).cuda()).cpu().numpy()
    ref = oracle.kernel_rows_n2(oracle.params(w), V, np.arange(w.n_x))[:, w.Q // 2:]
    assert normwise(got, ref) <= 1e-6


def test_eval_at_perturbed_weights_matches_oracle_model(wmc):
    w = _wl(n_x=256, q=64)
    rng = np.random.default_rng(2)
    Vs = wi.gaussian_bumps(3, n_x=w.n_x)
    prm = nt.initial_params(w.Q) + rng.normal(0.0, 0.05, w.Q + 4)
    got = wmc.n2_eval(wmc.Params.of(w), torch.from_numpy(prm.astype(np.float32)).cuda(),
                      torch.from_numpy(Vs).cuda()).cpu().numpy()
    ref = np.concatenate([nt.model(prm.astype(np.float32).astype(np.float64), V, w.Q) for V in Vs]) / nt.target_scale(w.Q)
    assert normwise(got, ref) <= 2e-6


def test_sgd_trajectories_match_oracle(wmc):
    w = _wl()
    n_ex, epochs = 8, 10
    lrs = np.array([3e-2, 1e-2, 3e-3], np.float32)
    Vs = wi.gaussian_bumps(n_ex, n_x=w.n_x, seed=4)
    T = _targets(w, Vs)
    order = wi.sgd_order(epochs, n_ex)
    p0 = nt.initial_params(w.Q)
    prm = torch.from_numpy(np.tile(p0.astype(np.float32), (lrs.size, 1))).cuda()
    loss = torch.zeros((lrs.size, epochs), device="cuda")
    wmc.n2_train(wmc.Params.of(w), torch.from_numpy(Vs).cuda(), torch.from_numpy(T).cuda(),
                 torch.from_numpy(order).cuda(), torch.from_numpy(lrs).cuda(), prm, loss)
    got, got_loss = prm.cpu().numpy().astype(np.float64), loss.cpu().numpy()
    Ts = T.astype(np.float64) * nt.target_scale(w.Q)
    for r, lr in enumerate(lrs):
        pf, hist = nt.train(p0, Vs, Ts, order, float(lr), w.Q)
        delta_ref = pf - p0
        assert np.linalg.norm(got[r] - pf) <= 1e-2 * np.linalg.norm(delta_ref), (r, lr)
        assert np.all(np.abs(got_loss[r] - hist) <= 1e-4 * hist), (r, got_loss[r], hist)
        assert hist[-1] < hist[0]


def test_zero_loss_where_n2_is_exact_and_determinism(wmc):
    w = _wl()
    V = np.zeros(w.n_x, np.float32)
    V[20:44] = np.repeat(np.random.default_rng(3).uniform(0.05, 0.3, 12), 2).astype(np.float32)
    Vs = np.stack([V, V])
    T = _targets(w, Vs)
    order = np.array([[0, 1]], np.int32)
    p0 = nt.initial_params(w.Q).astype(np.float32)
    prm = torch.from_numpy(np.tile(p0, (2, 1))).cuda()
    loss = torch.zeros((2, 1), device="cuda")
    wmc.n2_train(wmc.Params.of(w), torch.from_numpy(Vs).cuda(), torch.from_numpy(T).cuda(),
                 torch.from_numpy(order).cuda(), torch.tensor([1e-2, 1e-2], device="cuda"), prm, loss)
    scale2 = float(((T.astype(np.float64) * nt.target_scale(w.Q)) ** 2).mean())
    assert float(loss[0, 0]) <= 1e-10 * scale2
    out = prm.cpu().numpy()
    assert np.array_equal(out[0], out[1])
    assert np.abs(out[0] - p0).max() <= 1e-5
