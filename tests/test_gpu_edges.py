"""Degenerate and extreme inputs of the kernel evaluation through the C ABI:
every form gives exact zeros where Eq. (wigner-1d-discrete) is exactly zero (a
constant potential in clamp mode: every difference V(i+m) - V(i-m) vanishes),
and the widest window the tensor-core kernels hold (Q = 4096, K = 2047 terms)
stays within the FP32-accuracy bar against the FP64 oracle and the FP64
sliding window."""
import numpy as np
import pytest

import oracle
import wmc_inputs as wi
from tests._util import normwise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wmc():
    from paper_1806_00082_gb300 import build, wmc as w
    build.build()
    w.load()
    return w


@pytest.mark.parametrize("Q", [128, 1024])
@pytest.mark.parametrize("form", ["fp32", "fp32_simt", "bf16", "fp16", "fp16_split", "tf32x3"])
def test_constant_potential_in_clamp_mode_gives_exact_zeros(wmc, Q, form):
    wl = wi.DOUBLE_BARRIER_16384.replace(n_x=4096, Q=Q, n_M=Q, bc_potential=1)
    p = wmc.Params.of(wl)
    V = torch.full((wl.n_x,), 0.2371, dtype=torch.float32, device="cuda")
    ws = wmc.workspace(p)
    wmc.init(p, ws)
    occ = torch.arange(wl.n_x, dtype=torch.int32, device="cuda")
    out = wmc.kernel_eval(p, V, occ, ws, prec=wmc.PRECISIONS[form])
    assert torch.count_nonzero(out) == 0
    if form != "tf32x3":
        # the N = 2 form contracts pair sums 2V (not differences) against sines
        # whose sum over the window vanishes: what is left is rounding, below the
        # form's precision times the sum of the terms' magnitudes, 2 |V| h |c|
        n2 = wmc.kernel_eval_n2(p, V, occ, ws, prec=wmc.PRECISIONS["fp32" if form == "fp32_simt" else form])
        bound = {"fp32": 1e-6, "fp32_simt": 1e-6, "bf16": 1e-2, "fp16": 2e-3, "fp16_split": 1e-6}[form]
        terms = 2.0 / (6.582119569e-16 * Q) * 2 * 0.2371 * (Q // 2)
        assert float(n2.abs().max()) <= bound * terms


_REF = {}


@pytest.mark.parametrize("form,tol", [("fp32", 1.5e-6), ("fp16_split", 1.5e-6), ("fp32_simt", 1e-6),
                                      ("bf16", 1.5e-2)])
def test_widest_window(wmc, form, tol):
    wl = wi.DOUBLE_BARRIER_16384.replace(Q=4096, n_M=4096)
    p = wmc.Params.of(wl)
    V = wi.potential(wl)
    ws = wmc.workspace(p)
    wmc.init(p, ws)
    cells = np.concatenate([np.arange(8192 - 24, 8192 + 24), [0, 1, 2047, 2048, 14000, wl.n_x - 1]]).astype(np.int32)
    got = wmc.kernel_eval(p, torch.from_numpy(V).cuda(), torch.from_numpy(cells).cuda(), ws,
                          prec=wmc.PRECISIONS[form]).cpu().numpy()
    if "ref" not in _REF:
        _REF["ref"] = oracle.kernel_rows(oracle.params(wl.replace(n_M=wl.Q)), V, cells)[:, wl.Q // 2:]
    assert np.all(np.isfinite(got))
    assert normwise(got, _REF["ref"]) <= tol, (form, normwise(got, _REF["ref"]))
    assert wmc.get_counters(p, ws)["flags"] == 0


def test_widest_window_sliding_window(wmc):
    wl = wi.DOUBLE_BARRIER_16384.replace(Q=4096, n_M=4096)
    p = wmc.Params.of(wl)
    V = wi.potential(wl)
    ws = wmc.workspace(p)
    wmc.init(p, ws)
    got = wmc.kernel_eval_dft(p, torch.from_numpy(V).cuda(), ws).cpu().numpy()
    cells = np.array([0, 100, 8000, 8192, 8300, wl.n_x - 1])
    ref = oracle.kernel_rows(oracle.params(wl.replace(n_M=wl.Q)), V, cells)[:, wl.Q // 2:]
    assert normwise(got[cells], ref) <= 2e-7
