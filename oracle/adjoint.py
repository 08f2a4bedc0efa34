"""FP64 oracle of the differentiation form (test infrastructure only).

- potential_tanh / potential_tanh_vjp: the smooth multi-barrier potential
  (tanh-edged barriers and segment offsets) and its exact derivatives.
- kernel_vjp: dL/dV for L = sum gVW[i][r] V_W(i; r) + sum g_gamma[i] gamma(i),
  written from the unfolded Eq. (wigner-1d-discrete): for |l - i| < h,
  d V_W(i; M) / d V(l) = -(2 / (hbar Q)) sin(2 pi (l - i) M / Q), and
  d gamma(i) / d V_W(i; M) = [V_W(i; M) > 0] (Eq. momentum_integral), with V = 0
  outside the domain.  A matrix product (numpy) is the only library step.
"""
from __future__ import annotations

import numpy as np

from . import kernel_rows, params as _params, sine  # noqa: F401

HBAR_EVS = 6.582119569e-16


def _window(x, a, b, eps):
    return 0.5 * (np.tanh((x - a) / eps) - np.tanh((x - b) / eps))


def _sech2(u):
    e = np.exp(-2.0 * np.abs(u))
    return 4.0 * e / (1.0 + e) ** 2


def potential_tanh(theta, n_x, dx_nm, nb, ns, eps):
    """V [n_x] in eV (FP64) of one parameter vector (lengths in nm)."""
    th = np.asarray(theta, np.float64)
    x = (np.arange(n_x) + 0.5) * dx_nm
    L = n_x * dx_nm
    V = np.zeros(n_x)
    for k in range(nb):
        h, w, c = th[k], th[nb + k], th[2 * nb + k]
        V += h * _window(x, c - w / 2, c + w / 2, eps)
    for s in range(ns):
        V += th[3 * nb + s] * _window(x, L * s / ns, L * (s + 1) / ns, eps)
    return V


def potential_tanh_vjp(theta, Vbar, n_x, dx_nm, nb, ns, eps):
    """sum_i Vbar[i] dV(x_i) / d theta (FP64)."""
    th = np.asarray(theta, np.float64)
    vb = np.asarray(Vbar, np.float64)
    x = (np.arange(n_x) + 0.5) * dx_nm
    L = n_x * dx_nm
    out = np.zeros(3 * nb + ns)
    for k in range(nb):
        h, w, c = th[k], th[nb + k], th[2 * nb + k]
        up, um = (x - c + w / 2) / eps, (x - c - w / 2) / eps
        sech2p, sech2m = _sech2(up), _sech2(um)
        out[k] = np.dot(vb, 0.5 * (np.tanh(up) - np.tanh(um)))
        out[nb + k] = np.dot(vb, h * 0.5 * (sech2p + sech2m) * 0.5 / eps)
        out[2 * nb + k] = np.dot(vb, h * 0.5 * (-sech2p + sech2m) / eps)
    for s in range(ns):
        out[3 * nb + s] = np.dot(vb, _window(x, L * s / ns, L * (s + 1) / ns, eps))
    return out


def kernel_vjp(p, V, gVW=None, g_gamma=None, active=None):
    """dL/dV [n_x] for one potential (bc 0): gVW [n_x, Q/2] weights V_W(i; r),
    r = 0 .. h-1, g_gamma [n_x] weights gamma(i).  gamma is piecewise linear in
    V; its gradient is that of the active set, active[i][k] = [V_W(i; M_k) > 0]
    (from this oracle's FP64 kernel unless given)."""
    n_x, Q, n_M = p.n_x, p.Q, p.n_M
    h = Q // 2
    Ms = np.arange(n_M) - n_M // 2
    G = np.zeros((n_x, n_M))
    if g_gamma is not None:
        if active is None:
            active = kernel_rows(p, np.asarray(V, np.float64), np.arange(n_x)) > 0
        G += np.asarray(g_gamma, np.float64)[:, None] * active
    if gVW is not None:
        gv = np.asarray(gVW, np.float64)
        for r in range(h):
            k = np.nonzero(Ms == r)[0]
            if k.size:
                G[:, k[0]] += gv[:, r]
    ds = np.arange(-(h - 1), h)
    Sd = np.array([[sine(Q, int(d) * int(M)) for d in ds] for M in Ms])  # [n_M, 2h-1]
    Y = G @ Sd                                                             # [n_x, 2h-1]
    coef = -2.0 / (HBAR_EVS * Q)
    Vbar = np.zeros(n_x)
    for q, d in enumerate(ds):
        i = np.arange(n_x)
        l = i + d
        ok = (l >= 0) & (l < n_x)
        np.add.at(Vbar, l[ok], coef * Y[i[ok], q])
    return Vbar
