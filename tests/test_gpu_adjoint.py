"""The differentiation form on the GPU (autograd.Function over libwmc) against
the FP64 adjoint oracle, at the 4096-cell, Q = 256, n_M = 512 shape with the
64-parameter tanh-barrier potentials (a few of the batch)."""
import numpy as np
import pytest

import oracle
from oracle import adjoint as adj
import wmc_inputs as wi
from tests._util import normwise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NB, NS, EPS = 16, 16, 0.5
GRAD_TOL = 1e-4   # normwise, FP32 path vs FP64 oracle on the same active set
POT_TOL = 1e-6    # normwise, FP32 potential


@pytest.fixture(scope="module")
def wmc():
    from paper_1806_00082_gb300 import build, wmc as w
    build.build()
    w.load()
    return w


def _setup(wmc, n_pot, seed=3):
    wl = wi.TANH_BARRIERS_4096
    p = wmc.Params.of(wl)
    ws = wmc.workspace(p)
    wmc.init(p, ws)
    th = wi.tanh_parameters(n_pot, n_x=wl.n_x, dx_nm=wl.dx_m * 1e9, n_barriers=NB, n_segments=NS, seed=seed)
    return wl, p, ws, th


def test_potential_forward_and_vjp(wmc):
    wl, p, ws, th = _setup(wmc, 3)
    dx = wl.dx_m * 1e9
    V = wmc.potential_tanh(p, torch.from_numpy(th).cuda(), NB, NS, EPS).cpu().numpy()
    vb = np.random.default_rng(4).normal(size=(3, wl.n_x)).astype(np.float32)
    tb = wmc.potential_tanh_vjp(p, torch.from_numpy(th).cuda(), NB, NS, EPS, torch.from_numpy(vb).cuda()).cpu().numpy()
    for b in range(3):
        ref = adj.potential_tanh(th[b].astype(np.float64), wl.n_x, dx, NB, NS, EPS)
        assert normwise(V[b], ref) <= POT_TOL
        tref = adj.potential_tanh_vjp(th[b].astype(np.float64), vb[b].astype(np.float64), wl.n_x, dx, NB, NS, EPS)
        assert normwise(tb[b], tref) <= 1e-4


def test_kernel_rows_of_potentials(wmc):
    wl, p, ws, th = _setup(wmc, 2)
    V = wmc.potential_tanh(p, torch.from_numpy(th).cuda(), NB, NS, EPS)
    VWh = wmc.kernel_eval_rows(p, V, ws).cpu().numpy()
    Vn = V.cpu().numpy()
    rows = np.arange(0, wl.n_x, 37)
    ph = oracle.params(wl.replace(n_M=wl.Q))
    for b in range(2):
        ref = oracle.kernel_rows(ph, Vn[b], rows)[:, wl.Q // 2:]
        assert normwise(VWh[b * wl.n_x + rows], ref) <= 1e-6
    # tensor-core split form on the same implicit rows
    VWs = wmc.kernel_eval_rows(p, V, ws, prec=wmc.FP16_SPLIT).cpu().numpy()
    ref = oracle.kernel_rows(ph, Vn[1], rows)[:, wl.Q // 2:]
    assert normwise(VWs[wl.n_x + rows], ref) <= 1e-6


def _active_full(VWh_rows, Q, n_M):
    """[V_W(i; M_k) > 0] on the full momentum grid from half-period rows."""
    h = Q // 2
    r = (np.arange(n_M) - n_M // 2) % Q
    full = np.zeros((VWh_rows.shape[0], n_M))
    lo = (r > 0) & (r < h)
    hi = r > h
    full[:, lo] = VWh_rows[:, r[lo]]
    full[:, hi] = -VWh_rows[:, Q - r[hi]]
    return full > 0


def test_active_set_agrees_where_well_determined(wmc):
    """The FP32 rows give the FP64 sign of V_W wherever |V_W| exceeds the FP32
    error bound (1e-6 of the row block maximum)."""
    wl, p, ws, th = _setup(wmc, 1, seed=8)
    V = wmc.potential_tanh(p, torch.from_numpy(th).cuda(), NB, NS, EPS)
    VWh = wmc.kernel_eval_rows(p, V, ws).cpu().numpy()
    rows = np.arange(0, wl.n_x, 13)
    full64 = oracle.kernel_rows(oracle.params(wl), V.cpu().numpy()[0].astype(np.float64), rows)
    act = _active_full(VWh[rows], wl.Q, wl.n_M)
    sure = np.abs(full64) > 1e-6 * np.abs(full64).max()
    assert np.array_equal(act[sure], full64[sure] > 0)


def test_kernel_vjp_vs_oracle(wmc):
    """dL/dV for L = sum gVW VWh + sum g_gamma gamma, same FP32 potential on both sides."""
    wl, p, ws, th = _setup(wmc, 2, seed=8)
    V = wmc.potential_tanh(p, torch.from_numpy(th).cuda(), NB, NS, EPS)
    VWh = wmc.kernel_eval_rows(p, V, ws)
    rng = np.random.default_rng(6)
    h = wl.Q // 2
    gv = (rng.normal(size=(2 * wl.n_x, h)) * 1e-15).astype(np.float32)
    gg = (rng.normal(size=2 * wl.n_x) * 1e-16).astype(np.float32)
    Vbar = wmc.kernel_vjp(p, VWh, torch.from_numpy(gv).cuda(), torch.from_numpy(gg).cuda(), 2, ws).cpu().numpy()
    Vn = V.cpu().numpy().astype(np.float64)
    po = oracle.params(wl)
    VWn = VWh.cpu().numpy()
    for b in range(2):
        sl = slice(b * wl.n_x, (b + 1) * wl.n_x)
        ref = adj.kernel_vjp(po, Vn[b], gv[sl], gg[sl], active=_active_full(VWn[sl], wl.Q, wl.n_M))
        assert normwise(Vbar[b], ref) <= GRAD_TOL, (b, normwise(Vbar[b], ref))


def test_autograd_theta_gradient_vs_oracle(wmc):
    from paper_1806_00082_gb300.adjoint import kernel_of_potential
    wl, p, ws, th = _setup(wmc, 2, seed=9)
    rng = np.random.default_rng(7)
    h = wl.Q // 2
    gv = torch.from_numpy((rng.normal(size=(2 * wl.n_x, h)) * 1e-15).astype(np.float32)).cuda()
    gg = torch.from_numpy((rng.normal(size=2 * wl.n_x) * 1e-16).astype(np.float32)).cuda()
    theta = torch.from_numpy(th).cuda().requires_grad_(True)
    VWh, gamma = kernel_of_potential(theta, p, NB, NS, EPS, ws)
    loss = (VWh * gv).sum() + (gamma * gg).sum()
    loss.backward()
    got = theta.grad.cpu().numpy()
    po = oracle.params(wl)
    dx = wl.dx_m * 1e9
    VWn = VWh.detach().cpu().numpy()
    for b in range(2):
        sl = slice(b * wl.n_x, (b + 1) * wl.n_x)
        V64 = adj.potential_tanh(th[b].astype(np.float64), wl.n_x, dx, NB, NS, EPS)
        vb = adj.kernel_vjp(po, V64, gv[sl].cpu().numpy(), gg[sl].cpu().numpy(),
                            active=_active_full(VWn[sl], wl.Q, wl.n_M))
        ref = adj.potential_tanh_vjp(th[b].astype(np.float64), vb, wl.n_x, dx, NB, NS, EPS)
        assert normwise(got[b], ref) <= GRAD_TOL, (b, normwise(got[b], ref))


def test_autograd_smooth_loss_central_differences(wmc):
    """Central differences of the GPU forward (h = 1e-4 eV for heights and
    offsets, 1e-4 nm for widths and centres) on the smooth loss sum gVW VWh."""
    from paper_1806_00082_gb300.adjoint import kernel_of_potential
    wl, p, ws, th = _setup(wmc, 1, seed=10)
    h = wl.Q // 2
    gv = torch.from_numpy((np.random.default_rng(8).normal(size=(wl.n_x, h)) * 1e-15).astype(np.float32)).cuda()
    theta = torch.from_numpy(th).cuda().requires_grad_(True)
    VWh, _ = kernel_of_potential(theta, p, NB, NS, EPS, ws)
    (VWh * gv).sum().backward()
    got = theta.grad.cpu().numpy()[0]
    po = oracle.params(wl.replace(n_M=wl.Q))
    dx = wl.dx_m * 1e9
    gvn = gv.cpu().numpy().astype(np.float64)

    def L(t):  # FP64 forward of the same loss
        V = adj.potential_tanh(t, wl.n_x, dx, NB, NS, EPS)
        return np.sum(gvn * oracle.kernel_rows(po, V, np.arange(wl.n_x))[:, h:])

    t0 = th[0].astype(np.float64)
    for j in [0, 5, 16, 21, 32, 40, 48, 63]:
        tp, tm = t0.copy(), t0.copy()
        tp[j] += 1e-4
        tm[j] -= 1e-4
        fd = (L(tp) - L(tm)) / 2e-4
        assert abs(fd - got[j]) <= 2e-3 * max(np.max(np.abs(got)), 1e-30), (j, fd, got[j])
