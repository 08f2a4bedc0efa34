"""The allocation-free kernel evaluation (wmc_kernel_eval_noalloc).

It serves callers that cannot allocate device memory or hand the library a
workspace, for instance code inside an application whose device memory belongs
to a pool allocator, or one that forbids allocation after start-up.  Its
scratch (the sine matrix) is a fixed array in the library's device memory.

Checked through the C ABI against wmc_kernel_eval (the workspace entry point)
on consecutive calls that reuse the shared array with different window sizes:
bit-identical to its CUDA-core form where both run the tiled kernel (Q > 256),
and within the kernel tolerance of the other tests otherwise and against the
default FP32-accuracy form.  Collected last on purpose; it
passes alone in a fresh process and after the rest of the suite.
"""
import numpy as np
import pytest

import wmc_inputs as wi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KERNEL_TOL = 1e-6   # normwise, as for wmc_kernel_eval


def _normwise(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def test_noalloc_matches_workspace_entry_point_on_consecutive_calls():
    from paper_1806_00082_gb300 import build, wmc
    build.build()
    wmc.load()
    rng = np.random.default_rng(21)
    # Q = 1024, then 128 (a smaller table in the same array), then 1024 again
    for wl in (wi.DOUBLE_BARRIER_16384, wi.BARRIER_2000, wi.DOUBLE_BARRIER_16384):
        p = wmc.Params.of(wl)
        V = torch.from_numpy(wi.potential(wl)).cuda()
        cells = rng.integers(0, wl.n_x, size=257).astype(np.int32)
        cells[:64] = np.arange(wl.n_x // 2 - 32, wl.n_x // 2 + 32)
        occ = torch.from_numpy(cells).cuda()
        ws = wmc.workspace(p)
        wmc.init(p, ws)
        ref = wmc.kernel_eval(p, V, occ, ws, prec=wmc.FP32_SIMT)
        dflt = wmc.kernel_eval(p, V, occ, ws)
        out = torch.full_like(ref, float("nan"))
        wmc.kernel_eval_noalloc(p, V, occ, out)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        if wl.Q > 256:
            assert torch.equal(out, ref)
        assert _normwise(out, ref) <= KERNEL_TOL
        assert _normwise(out, dflt) <= KERNEL_TOL


def test_noalloc_rejects_window_beyond_limit():
    from paper_1806_00082_gb300 import wmc
    wl = wi.DOUBLE_BARRIER_16384.replace(Q=2048, n_M=2048, dt_s=0.02e-15)
    p = wmc.Params.of(wl)
    V = torch.from_numpy(wi.potential(wl)).cuda()
    occ = torch.arange(8, dtype=torch.int32, device="cuda")
    out = torch.zeros((8, wl.Q // 2), device="cuda")
    with pytest.raises(wmc.WmcError) as e:
        wmc.kernel_eval_noalloc(p, V, occ, out)
    assert e.value.code == 2   # WMC_ERR_CAPACITY
    assert torch.count_nonzero(out) == 0
