"""FP64 oracle of the trained N = 2 network (test infrastructure only).

Eq. (kernel_ML) of Sec. 2.3 with N = 2 (one cosine factor), its weights learnt
by stochastic gradient descent on a mean-squared-error loss against exact
kernels, as the paper trains it.  Reduced units: kernels are scaled by
hbar Q / 2 (V in eV), so the model reads

  y(i, j) = cos(pi j / Q) sum_{d in D(i)} W[d] (wv1 V(i + d) + wv2 V(i + d + 1))
                                          sin(2 pi j / Q (wt1 d + wt2 (d + 1))),

with D(i) = {d in [-h, h - 1] : i + d even}: the absolute cell pairs
(2q, 2q + 1), 2q = i + d, that lie inside the window [i - h, i + h], the pair
offset d indexing the weight W (Q of them, W[d + h]).  At W = -1,
(wv1, wv2) = (1, 1), (wt1, wt2) = (1/2, 1/2) this is the analytic N = 2 network
(the oracle's kernel_rows_n2) times hbar Q / 2.  V is 0 outside the domain
(bc = 0) or the edge value (bc = 1).

Parameters are one vector [W[0..Q-1], wv1, wv2, wt1, wt2].  The loss of one
example is the mean over the cells i in [0, n_x) and the distinct columns
j in [1, h) of (y - t)^2; one SGD step takes one example and sets
p <- p - lr dL/dp; an epoch visits the examples in the order given.

All arrays are numpy FP64; the only library steps are elementwise numpy
functions and sums.
"""
from __future__ import annotations

import numpy as np

HBAR_EVS = 6.582119569e-16


def initial_params(Q: int) -> np.ndarray:
    """The analytic N = 2 network's weights (the training's starting point)."""
    p = np.empty(Q + 4)
    p[:Q] = -1.0
    p[Q:] = (1.0, 1.0, 0.5, 0.5)
    return p


def target_scale(Q: int) -> float:
    """Factor from kernels in 1/s to the model's reduced units."""
    return HBAR_EVS * Q / 2.0


def _offsets(n_x: int, Q: int) -> np.ndarray:
    """D[i, k] = the k-th pair offset of row i (h of them, ascending)."""
    h = Q // 2
    i = np.arange(n_x)[:, None]
    d0 = np.where((i - h) % 2 == 0, -h, -h + 1)
    return d0 + 2 * np.arange(h)[None, :]


def _pot(V: np.ndarray, idx: np.ndarray, bc: int) -> np.ndarray:
    n_x = V.shape[0]
    inside = (idx >= 0) & (idx < n_x)
    out = np.where(inside, V[np.clip(idx, 0, n_x - 1)], 0.0)
    if bc:
        out = np.where(idx < 0, V[0], np.where(idx >= n_x, V[n_x - 1], out))
    return out


def _parts(params: np.ndarray, V: np.ndarray, Q: int, bc: int):
    n_x = V.shape[0]
    h = Q // 2
    W = params[:Q]
    wv1, wv2, wt1, wt2 = params[Q:]
    D = _offsets(n_x, Q)                                   # [n_x, h]
    i = np.arange(n_x)[:, None]
    Va = _pot(np.asarray(V, np.float64), i + D, bc)        # V(2q)
    Vb = _pot(np.asarray(V, np.float64), i + D + 1, bc)    # V(2q + 1)
    P = wv1 * Va + wv2 * Vb
    Wd = W[D + h]
    j = np.arange(h)
    phi = 2.0 * np.pi * j / Q                               # [h]
    arg = phi[None, None, :] * (wt1 * D + wt2 * (D + 1))[:, :, None]   # [n_x, h(k), h(j)]
    cj = np.cos(np.pi * j / Q)
    return D, Va, Vb, P, Wd, phi, np.sin(arg), np.cos(arg), cj


def model(params: np.ndarray, V: np.ndarray, Q: int, bc: int = 0) -> np.ndarray:
    """y [n_x, h] (columns j = 0 .. h - 1 of the half period; column 0 is zero)."""
    _, _, _, P, Wd, _, S, _, cj = _parts(params, V, Q, bc)
    return cj[None, :] * np.einsum("ik,ikj->ij", Wd * P, S)


def loss_and_grad(params: np.ndarray, V: np.ndarray, T: np.ndarray, Q: int, bc: int = 0):
    """(loss, dloss/dparams) of one example; T [n_x, h] targets in reduced units."""
    n_x = V.shape[0]
    h = Q // 2
    D, Va, Vb, P, Wd, phi, S, C, cj = _parts(params, V, Q, bc)
    y = cj[None, :] * np.einsum("ik,ikj->ij", Wd * P, S)
    r = y - T
    r[:, 0] = 0.0
    n_out = n_x * (h - 1)
    loss = float((r * r).sum() / n_out)
    rc = (2.0 / n_out) * r * cj[None, :]                    # dL/dy times cos(pi j / Q)
    G = np.einsum("ij,ikj->ik", rc, S)                      # sum_j dL/dy c_j sin
    H = np.einsum("ij,ikj->ik", rc * phi[None, :], C)       # sum_j dL/dy c_j phi_j cos
    grad = np.zeros_like(params)
    np.add.at(grad, D + h, P * G)                           # dW[d]
    wt1_part = Wd * P * H
    grad[Q + 0] = (Wd * Va * G).sum()
    grad[Q + 1] = (Wd * Vb * G).sum()
    grad[Q + 2] = (wt1_part * D).sum()
    grad[Q + 3] = (wt1_part * (D + 1)).sum()
    return loss, grad


def train(params0: np.ndarray, Vs: np.ndarray, Ts: np.ndarray, order: np.ndarray, lr: float, Q: int,
          bc: int = 0):
    """SGD over epochs: order [epochs, n_examples] gives the examples of each
    epoch in turn.  Returns (final params, mean loss of each epoch, measured at
    each step before its update)."""
    p = np.array(params0, np.float64)
    epochs = order.shape[0]
    hist = np.empty(epochs)
    for e in range(epochs):
        tot = 0.0
        for ex in order[e]:
            loss, g = loss_and_grad(p, Vs[ex], Ts[ex], Q, bc)
            tot += loss
            p = p - lr * g
        hist[e] = tot / order.shape[1]
    return p, hist
