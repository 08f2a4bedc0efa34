"""The FP64 sliding-window evaluation on the GPU (wmc_kernel_eval_dft) against
the oracle's, and every contraction form on all 16384 cells of the double
barrier against the oracle's FP64 rows (the full-size parity of the kernel)."""
import numpy as np
import pytest

import oracle
import wmc_inputs as wi
from tests._util import normwise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32": 5e-7, "fp32_simt": 5e-7, "bf16": 1.5e-2, "fp16": 1e-3, "fp16_split": 5e-7, "tf32x3": 5e-7}
_ref = {}


@pytest.fixture(scope="module")
def wmc():
    from paper_1806_00082_gb300 import build, wmc as w
    build.build()
    w.load()
    return w


def _half_ref(wl, V):
    key = (wl.name, wl.bc_potential, V.tobytes())
    if key not in _ref:
        _ref[key] = oracle.kernel_all_dft(oracle.params(wl.replace(n_M=wl.Q)), V)[:, wl.Q // 2:]
    return _ref[key]


@pytest.mark.parametrize("wl", [wi.BARRIER_100, wi.BARRIER_100.replace(bc_potential=1), wi.BARRIER_2000,
                                wi.DOUBLE_BARRIER_16384])
def test_dft_matches_oracle(wmc, wl):
    p = wmc.Params.of(wl)
    V = wi.potential(wl)
    if wl.bc_potential:
        V = np.random.default_rng(5).uniform(-0.2, 0.3, wl.n_x).astype(np.float32)
    ws = wmc.workspace(p)
    wmc.init(p, ws)
    got = wmc.kernel_eval_dft(p, torch.from_numpy(V).cuda(), ws).cpu().numpy()
    assert normwise(got, _half_ref(wl, V)) <= 2e-7


@pytest.mark.parametrize("form", ["fp32", "fp32_simt", "bf16", "fp16", "fp16_split", "tf32x3"])
def test_forms_on_every_cell_of_the_double_barrier(wmc, form):
    wl = wi.DOUBLE_BARRIER_16384
    p = wmc.Params.of(wl)
    V = wi.potential(wl)
    ws = wmc.workspace(p)
    wmc.init(p, ws)
    occ = torch.arange(wl.n_x, dtype=torch.int32, device="cuda")
    got = wmc.kernel_eval(p, torch.from_numpy(V).cuda(), occ, ws, prec=wmc.PRECISIONS[form]).cpu().numpy()
    assert normwise(got, _half_ref(wl, V)) <= TOL[form]
