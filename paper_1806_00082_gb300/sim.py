"""A simulation's device buffers and the libwmc calls that advance it.

The state is the net signed histogram hist[n_x, n_M] left by annihilation
(rule 2 of the signed particle formulation, Sec. 2.1); ``run`` advances it by
whole steps of the postulate through ``wmc_run`` (one CUDA graph per step pair).
"""
from __future__ import annotations

import numpy as np
import torch

from . import wmc


class Simulation:
    def __init__(self, params: wmc.Params, V, hist0, t_first: int = 1, device="cuda", prec: int = wmc.FP32):
        self.p = params
        self.prec = prec
        self.device = torch.device(device)
        self.V = torch.as_tensor(np.asarray(V, dtype=np.float32)).to(self.device)
        h0 = torch.as_tensor(np.asarray(hist0, dtype=np.int32)).reshape(params.n_x, params.n_M)
        self.hist = h0.to(self.device).contiguous()
        self.hist_b = torch.empty_like(self.hist)
        self.ws = wmc.workspace(params, self.device)
        wmc.init(params, self.ws)
        self.t = t_first

    def run(self, n_steps: int, use_graph: bool = True) -> None:
        wmc.run(self.p, self.V, self.hist, self.hist_b, self.t, n_steps, self.ws, self.prec, use_graph)
        self.t += n_steps

    def density(self) -> torch.Tensor:
        return wmc.density(self.p, self.hist)

    def counters(self) -> dict:
        return wmc.get_counters(self.p, self.ws)
