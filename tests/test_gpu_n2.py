"""The N = 2 barycentric network (Sec. 2.3, Eq. kernel_ML with N = 2) on the
GPU through the C ABI, against the CPU oracle's FP64 evaluation of the same
network: FP32 within 1e-6 normwise, the tensor-core forms within the bounds of
the N = 1 forms; its rows driving the simulation bit for bit against the oracle
fed the same table."""
import numpy as np
import pytest

import oracle
import wmc_inputs as wi
from tests._util import full_from_half, gpu_run_table, normwise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-6, "bf16": 1.5e-2, "fp16": 1e-3, "fp16_split": 1e-6}


@pytest.fixture(scope="module")
def wmc():
    from paper_1806_00082_gb300 import build, wmc as w
    build.build()
    w.load()
    return w


def _ref_half(wl, V, cells):
    return oracle.kernel_rows_n2(oracle.params(wl.replace(n_M=wl.Q)), V, cells)[:, wl.Q // 2:]


def _cells(wl, n, seed):
    if wl.n_x <= 2000:
        return np.arange(wl.n_x, dtype=np.int32)
    rng = np.random.default_rng(seed)
    c = np.concatenate([np.arange(8192 - 100, 8192 + 100), rng.integers(0, wl.n_x, n - 206),
                        [0, 1, 2, wl.n_x - 1, wl.n_x - 2, 8191]])
    return c.astype(np.int32)


@pytest.mark.parametrize("form", ["fp32", "bf16", "fp16", "fp16_split"])
@pytest.mark.parametrize("wl", [wi.BARRIER_100, wi.BARRIER_2000, wi.DOUBLE_BARRIER_16384])
def test_n2_forms_vs_oracle(wmc, form, wl):
    p = wmc.Params.of(wl)
    V = wi.potential(wl)
    ws = wmc.workspace(p)
    wmc.init(p, ws)
    cells = _cells(wl, 333, 5)
    got = wmc.kernel_eval_n2(p, torch.from_numpy(V).cuda(), torch.from_numpy(cells).cuda(), ws,
                             prec=wmc.PRECISIONS[form]).cpu().numpy()
    ref = _ref_half(wl, V, cells)
    assert np.all(np.isfinite(got))
    assert np.all(got[:, 0] == 0)
    err = normwise(got, ref)
    assert err <= TOL[form], (form, wl.name, err)
    exact = oracle.kernel_rows(oracle.params(wl.replace(n_M=wl.Q)), V, cells)[:, wl.Q // 2:]
    if wl is wi.BARRIER_2000:
        # its barrier covers cells 990-1009, whole pairs (2q, 2q+1): the network is exact
        assert normwise(ref, exact) < 1e-12
    else:
        # an odd-aligned barrier (cells 47-52) and per-cell noise: the network differs
        assert normwise(ref, exact) > 10 * TOL["fp32"]


def test_n2_clamp_boundary_and_pairwise_constant(wmc):
    """Edge-value potential outside the domain; and a pairwise-constant
    potential, where the N = 2 rows equal the N = 1 rows."""
    wl = wi.BARRIER_100.replace(bc_potential=1)
    p = wmc.Params.of(wl)
    ws = wmc.workspace(p)
    wmc.init(p, ws)
    occ = torch.arange(wl.n_x, dtype=torch.int32, device="cuda")
    V = np.random.default_rng(3).uniform(-0.2, 0.3, wl.n_x).astype(np.float32)
    got = wmc.kernel_eval_n2(p, torch.from_numpy(V).cuda(), occ, ws).cpu().numpy()
    assert normwise(got, _ref_half(wl, V, np.arange(wl.n_x))) <= TOL["fp32"]
    Vp = np.repeat(V[::2], 2).astype(np.float32)
    a = wmc.kernel_eval_n2(p, torch.from_numpy(Vp).cuda(), occ, ws).cpu().numpy()
    b = wmc.kernel_eval(p, torch.from_numpy(Vp).cuda(), occ, ws).cpu().numpy()
    assert normwise(a, b.astype(np.float64)) <= 2e-6


@pytest.mark.parametrize("n_occ", [0, 1, 127, 128, 129, 333])
def test_n2_ragged_row_counts(wmc, n_occ):
    wl = wi.DOUBLE_BARRIER_16384
    p = wmc.Params.of(wl)
    V = wi.potential(wl)
    ws = wmc.workspace(p)
    wmc.init(p, ws)
    cells = ((np.arange(n_occ) * 37 + 8000) % wl.n_x).astype(np.int32)
    for form in ("fp32", "fp16_split"):
        out = torch.full((n_occ, wl.Q // 2), 7.0, device="cuda")
        wmc.kernel_eval_n2(p, torch.from_numpy(V).cuda(), torch.from_numpy(cells).cuda(), ws,
                           prec=wmc.PRECISIONS[form], out=out)
        if n_occ:
            assert normwise(out.cpu().numpy(), _ref_half(wl, V, cells)) <= TOL[form]


def test_n2_unsupported_form(wmc):
    wl = wi.BARRIER_100
    p = wmc.Params.of(wl)
    ws = wmc.workspace(p)
    wmc.init(p, ws)
    occ = torch.arange(4, dtype=torch.int32, device="cuda")
    with pytest.raises(wmc.WmcError):
        wmc.kernel_eval_n2(p, torch.from_numpy(wi.potential(wl)).cuda(), occ, ws, prec=wmc.TF32X3)


def test_n2_rows_drive_the_simulation_bit_exact(wmc):
    """The N = 2 network's FP32 rows of every cell as the kernel table of the
    step (wmc_kernel_table_occupied): histograms and counters equal the oracle's
    run fed the same table and Philox streams; pairs are created every step."""
    wl = wi.BARRIER_100.replace(packet=wi.Packet(48e-9, 5e-9, 0.1, 150_000))
    p = wmc.Params.of(wl)
    V = wi.potential(wl)
    ws = wmc.workspace(p)
    wmc.init(p, ws)
    occ = torch.arange(wl.n_x, dtype=torch.int32, device="cuda")
    half = wmc.kernel_eval_n2(p, torch.from_numpy(V).cuda(), occ, ws).cpu().numpy()
    h0 = wi.initial_histogram(wl)
    ref, st = oracle.simulate(oracle.params(wl), h0, 1, 8, table=full_from_half(half, wl.Q, wl.n_M))
    got, c = gpu_run_table(wmc, torch, p, half, h0, 1, 8)
    np.testing.assert_array_equal(got, ref)
    assert c["pairs"] == st[oracle.ST_PAIRS] > 5000
