"""Precision forms of the kernel contraction on the tcgen05 tensor cores
(BF16, FP16, FP16 hi/lo split, 3xTF32), against the FP64 oracle (normwise
error, reading 13), and the FP32 form.

Expected input-rounding errors (numpy estimates at Q = 1024): BF16 about 3-6e-3,
FP16 about 2e-4.  The split forms keep each K block's hi x hi product in its
own tensor-memory accumulator and sum the blocks in FP32 registers: measured
3.6e-7 at Q = 1024 and 4.9e-7 at Q = 2048 on every cell of the double barrier
(the CUDA-core FP32 form: 2.9e-7), against 9.3e-7 and 2.1e-6 with the K halves
in two accumulators.  WMC_FP32 runs the 3xTF32 form for Q > 256."""
import numpy as np
import pytest

import oracle
import wmc_inputs as wi
from tests._util import normwise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"bf16": 1.5e-2, "fp16": 1e-3, "fp16_split": 5e-7, "tf32x3": 5e-7, "fp32": 5e-7, "fp32_simt": 5e-7}


@pytest.fixture(scope="module")
def wmc():
    from paper_1806_00082_gb300 import build, wmc as w
    build.build()
    w.load()
    return w


def _cells(wl, n, seed):
    rng = np.random.default_rng(seed)
    c = np.concatenate([rng.integers(0, wl.n_x, n - 8), [0, wl.n_x - 1, wl.n_x // 2, wl.n_x // 2,
                                                         1, 2, wl.n_x - 2, wl.n_x // 3]])
    return c.astype(np.int32)


@pytest.mark.parametrize("form", ["bf16", "fp16", "fp16_split", "tf32x3", "fp32", "fp32_simt"])
@pytest.mark.parametrize("wl,n", [(wi.BARRIER_100, 100), (wi.BARRIER_2000, 333), (wi.DOUBLE_BARRIER_16384, 333)])
def test_tensorcore_forms_vs_fp64(wmc, form, wl, n):
    p = wmc.Params.of(wl)
    V = wi.potential(wl)
    ws = wmc.workspace(p)
    wmc.init(p, ws)
    cells = _cells(wl, n, 17) if wl.n_x > 100 else np.arange(wl.n_x, dtype=np.int32)
    if wl.n_x > 2000:  # concentrate on the barrier region
        cells[:200] = np.arange(8192 - 100, 8192 + 100)
    occ = torch.from_numpy(cells).cuda()
    got = wmc.kernel_eval(p, torch.from_numpy(V).cuda(), occ, ws, prec=wmc.PRECISIONS[form]).cpu().numpy()
    ref = oracle.kernel_rows(oracle.params(wl.replace(n_M=wl.Q)), V, cells)[:, wl.Q // 2:]
    err = normwise(got, ref)
    assert np.all(np.isfinite(got))
    assert err <= TOL[form], (form, wl.name, err)
    assert wmc.get_counters(p, ws)["flags"] == 0


@pytest.mark.parametrize("form", ["fp16_split", "bf16", "fp16"])
def test_tensorcore_ragged_rows_and_tiles(wmc, form):
    """Row counts below, at and around the 128-row tile (1, 15, 17, 127-129,
    300) and an empty list, for scattered and for consecutive cells (the
    potential-window path of the builders, with a ragged last tile)."""
    wl = wi.DOUBLE_BARRIER_16384
    p = wmc.Params.of(wl)
    V = torch.from_numpy(wi.potential(wl)).cuda()
    ws = wmc.workspace(p)
    wmc.init(p, ws)
    for n in (0, 1, 15, 17, 127, 128, 129, 300):
        for stride in (37, 1):
            cells = (np.arange(n) * stride + 8000) % wl.n_x
            occ = torch.from_numpy(cells.astype(np.int32)).cuda()
            out = torch.full((n, wl.Q // 2), 3.0, device="cuda")
            wmc.kernel_eval(p, V, occ, ws, prec=wmc.PRECISIONS[form], out=out)
            if n:
                ref = oracle.kernel_rows(oracle.params(wl.replace(n_M=wl.Q)), wi.potential(wl), cells)[:, wl.Q // 2:]
                assert normwise(out.cpu().numpy(), ref) <= TOL[form], (form, n, stride)
    assert wmc.get_counters(p, ws)["flags"] == 0


@pytest.mark.parametrize("form", ["bf16", "fp16"])
def test_tensorcore_consecutive_rows_window_not_multiple_of_4(wmc, form):
    """Consecutive cells with h = Q/2 not a multiple of 4 (Q = n_M = 1020):
    the potential window is staged but read element by element; the whole
    domain (sampled) and a ragged run of 300 cells."""
    wl = wi.DOUBLE_BARRIER_16384.replace(Q=1020, n_M=1020)
    p = wmc.Params.of(wl)
    V = wi.potential(wl)
    ws = wmc.workspace(p)
    wmc.init(p, ws)
    for cells in (np.arange(wl.n_x, dtype=np.int32), np.arange(8000, 8300, dtype=np.int32)):
        got = wmc.kernel_eval(p, torch.from_numpy(V).cuda(), torch.from_numpy(cells).cuda(), ws,
                              prec=wmc.PRECISIONS[form]).cpu().numpy()
        assert np.all(np.isfinite(got))
        assert _sampled_err(got, wl, V, cells, 120, 3) <= TOL[form], (form, cells.size)
    assert wmc.get_counters(p, ws)["flags"] == 0


def test_tensorcore_in_production_loop(wmc):
    """wmc_run with the BF16 and split kernels: the CDF and the step consume
    the tensor-core rows; densities stay close to the FP64 oracle under common
    random numbers (BF16 within its kernel error, split within the FP32 bar)."""
    from tests._util import gpu_run
    wl = wi.BARRIER_100
    p = wmc.Params.of(wl)
    V = wi.potential(wl)
    h0 = wi.initial_histogram(wl)
    ref, _ = oracle.simulate(oracle.params(wl), h0, 1, 50, V=V)
    for form, tol in (("fp16_split", 1e-3), ("tf32x3", 1e-3), ("bf16", 2e-2)):
        ws = wmc.workspace(p)
        wmc.init(p, ws)
        Vd = torch.from_numpy(V).cuda()
        a = torch.from_numpy(h0).cuda()
        b = torch.empty_like(a)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            wmc.run(p, Vd, a, b, 1, 50, ws, prec=wmc.PRECISIONS[form])
            c = wmc.get_counters(p, ws)
        s.synchronize()
        got = a.cpu().numpy()
        l1 = np.abs(got.sum(axis=1) - ref.sum(axis=1)).sum() / wl.packet.n0
        assert l1 <= tol, (form, l1)
        assert c["flags"] == 0


def _sampled_err(got, wl, V, cells, n_sample, seed):
    rng = np.random.default_rng(seed)
    pick = np.unique(np.concatenate([rng.integers(0, cells.size, n_sample), [0, cells.size - 1]]))
    ref = oracle.kernel_rows(oracle.params(wl.replace(n_M=wl.Q)), V, cells[pick])[:, wl.Q // 2:]
    return normwise(got[pick], ref)


@pytest.mark.parametrize("form", ["bf16", "fp16", "fp16_split", "tf32x3"])
@pytest.mark.parametrize("wl,n", [(wi.DOUBLE_BARRIER_16384, 16384 - 77), (wi.DOUBLE_BARRIER_16384, 16384),
                                  (wi.BARRIER_2000, 40_000 + 45)])
def test_tensorcore_whole_row_form(wmc, form, wl, n):
    """Row counts that fill the GPU (the warp-specialised contractions):
    every cell of the domain (contiguous windows), a permutation with a ragged
    last tile, and a list longer than the domain with repeated cells; sampled
    rows against the FP64 oracle, every row finite, and each repeated cell
    bit-identical."""
    p = wmc.Params.of(wl)
    V = wi.potential(wl)
    ws = wmc.workspace(p)
    wmc.init(p, ws)
    if n == wl.n_x:
        cells = np.arange(n, dtype=np.int32)
    elif n < wl.n_x:
        cells = np.random.default_rng(5).permutation(wl.n_x)[:n].astype(np.int32)
    else:
        cells = (np.arange(n) % wl.n_x).astype(np.int32)
    got = wmc.kernel_eval(p, torch.from_numpy(V).cuda(), torch.from_numpy(cells).cuda(), ws,
                          prec=wmc.PRECISIONS[form]).cpu().numpy()
    assert np.all(np.isfinite(got))
    assert _sampled_err(got, wl, V, cells, 160, 9) <= TOL[form], (form, wl.name, n)
    if n > wl.n_x:
        assert np.array_equal(got[:wl.n_x], got[wl.n_x:2 * wl.n_x])
    assert wmc.get_counters(p, ws)["flags"] == 0


@pytest.mark.parametrize("form", ["bf16", "fp16", "fp16_split", "tf32x3"])
def test_tensorcore_implicit_rows_many_potentials(wmc, form):
    """Implicit rows (row r = cell r mod n_x of potential r / n_x) over several
    potentials, with n_x not a multiple of the 128-row tile, so that tiles
    straddle two potentials."""
    wl = wi.BARRIER_2000.replace(n_x=2000 + 13)
    p = wmc.Params.of(wl)
    rng = np.random.default_rng(4)
    n_pot = 24
    Vs = np.stack([wi.potential(wl) * np.float32(rng.uniform(0.5, 1.5)) for _ in range(n_pot)]).astype(np.float32)
    ws = wmc.workspace(p)
    wmc.init(p, ws)
    got = wmc.kernel_eval_rows(p, torch.from_numpy(Vs).cuda(), ws, prec=wmc.PRECISIONS[form]).cpu().numpy()
    assert np.all(np.isfinite(got))
    for b in (0, 7, n_pot - 1):
        cells = np.arange(wl.n_x, dtype=np.int32)
        err = _sampled_err(got[b * wl.n_x:(b + 1) * wl.n_x], wl, Vs[b], cells, 120, b)
        assert err <= TOL[form], (form, b, err)
    assert wmc.get_counters(p, ws)["flags"] == 0


_REF = {}  # FP64 reference rows shared by the parametrised forms


@pytest.mark.parametrize("form", ["bf16", "fp16", "fp16_split", "tf32x3"])
def test_tensorcore_wide_window(wmc, form):
    """A window wider than the resident-A forms hold (Q = n_M = 2048): the
    per-tile kernel with streamed A, on a ragged list of cells around the
    barriers, against the FP64 oracle."""
    wl = wi.DOUBLE_BARRIER_16384.replace(Q=2048, n_M=2048)
    p = wmc.Params.of(wl)
    V = wi.potential(wl)
    ws = wmc.workspace(p)
    wmc.init(p, ws)
    cells = np.concatenate([np.arange(8192 - 40, 8192 + 40), [0, 1, wl.n_x - 1, 4000, 12000]]).astype(np.int32)
    got = wmc.kernel_eval(p, torch.from_numpy(V).cuda(), torch.from_numpy(cells).cuda(), ws,
                          prec=wmc.PRECISIONS[form]).cpu().numpy()
    if "wide" not in _REF:
        _REF["wide"] = oracle.kernel_rows(oracle.params(wl.replace(n_M=wl.Q)), V, cells)[:, wl.Q // 2:]
    ref = _REF["wide"]
    assert np.all(np.isfinite(got))
    # the split forms over the 1023-term window: 16 K blocks drained one by one
    # (measured 4.9e-7 on every cell)
    tol = {"fp16_split": 1e-6, "tf32x3": 1e-6}.get(form, TOL[form])
    assert normwise(got, ref) <= tol, (form, normwise(got, ref))
    assert wmc.get_counters(p, ws)["flags"] == 0


@pytest.mark.parametrize("wl,form", [(wi.DOUBLE_BARRIER_16384, "tf32x3"), (wi.BARRIER_2000, "fp32_simt"),
                                     (wi.BARRIER_100, "fp32_simt")])
def test_fp32_request_runs_the_stated_form(wmc, wl, form):
    """WMC_FP32 is the 3xTF32 tensor-core form for Q > 256 and the CUDA-core
    form otherwise: bit-identical rows to the form asked for by name."""
    p = wmc.Params.of(wl)
    V = torch.from_numpy(wi.potential(wl)).cuda()
    ws = wmc.workspace(p)
    wmc.init(p, ws)
    cells = np.concatenate([np.arange(wl.n_x // 2 - 70, wl.n_x // 2 + 70), [0, wl.n_x - 1]]).astype(np.int32)
    occ = torch.from_numpy(cells % wl.n_x).cuda()
    a = wmc.kernel_eval(p, V, occ, ws, prec=wmc.FP32).cpu().numpy()
    b = wmc.kernel_eval(p, V, occ, ws, prec=wmc.PRECISIONS[form]).cpu().numpy()
    assert np.array_equal(a, b)
