"""Training of the N = 2 network of Sec. 2.3 (Eq. kernel_ML, N = 2) on the GPU:
the exact kernels of the example potentials from wmc_kernel_eval_rows (the
FP32-accuracy form), then stochastic gradient descent in wmc_n2_train, one
thread block per learning rate.  The trained weights give kernel rows through
wmc_n2_eval."""
from __future__ import annotations

import torch

from . import wmc


def initial_params(Q: int, n_runs: int = 1, device="cuda") -> torch.Tensor:
    """[n_runs, Q + 4]: the analytic N = 2 network's weights (W = -1,
    (wv1, wv2) = (1, 1), (wt1, wt2) = (1/2, 1/2)), the starting point."""
    p = torch.full((n_runs, Q + 4), -1.0, dtype=torch.float32, device=device)
    p[:, Q:] = torch.tensor([1.0, 1.0, 0.5, 0.5], device=device)
    return p


def train(p: wmc.Params, V: torch.Tensor, order: torch.Tensor, lrs: torch.Tensor, ws: torch.Tensor,
          params: torch.Tensor | None = None):
    """Trains from params (default: the analytic weights) on the potentials
    V [n_examples, n_x]; order [epochs, n_examples] int32; lrs [n_runs].
    Returns (params [n_runs, Q + 4], loss [n_runs, epochs])."""
    n_runs, epochs = lrs.numel(), order.shape[0]
    if params is None:
        params = initial_params(p.Q, n_runs, V.device)
    VW = wmc.kernel_eval_rows(p, V, ws)
    loss = torch.empty((n_runs, epochs), dtype=torch.float32, device=V.device)
    wmc.n2_train(p, V, VW, order, lrs, params, loss)
    return params, loss
