"""The 16384-cell double barrier with per-cell noise (Q = n_M = 1024, 1e8
particles, dt = 0.05 fs) stepped at full size on the GPU against the CPU
oracle.  The noise gives every cell gamma > 0, so every step creates pairs
(about 4e5 of them): drift, pair creation at rate gamma (Eq. momentum_integral)
with p' ~ V_W^+ / gamma, and the signed histogram (rule 2) all run at scale.

Bars: with the oracle's FP64 kernel table fed to both sides (same Philox
streams) histograms and counters are bit-exact over the first five steps; with
the kernel evaluated in the loop by the GPU (FP32 accuracy: the 3xTF32
tensor-core form at this Q; the CUDA-core FP32 form; the FP16 hi/lo split)
the density stays within 1e-3 L1 of the oracle's FP64 run under common random
numbers.
"""
import numpy as np
import pytest

import oracle
import wmc_inputs as wi
from tests._util import gpu_run, gpu_run_table, reach_rows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

WL = wi.DOUBLE_BARRIER_16384
STEPS = 5
DENSITY_L1_TOL = 1e-3
_cache = {}


@pytest.fixture(scope="module")
def wmc():
    from paper_1806_00082_gb300 import build, wmc as w
    build.build()
    w.load()
    return w


def _h0():
    if "h0" not in _cache:
        _cache["h0"] = wi.initial_histogram(WL)
    return _cache["h0"]


def _oracle_fp64_run():
    """The oracle's own run: FP64 kernel evaluated on the occupied cells."""
    if "fp64" not in _cache:
        _cache["fp64"] = oracle.simulate(oracle.params(WL), _h0(), 1, STEPS, V=wi.potential(WL))
    return _cache["fp64"]


def test_c3_full_size_bit_exact_with_oracle_table(wmc):
    h0 = _h0()
    assert int(np.abs(h0).sum()) == WL.packet.n0
    V = wi.potential(WL)
    rows = reach_rows(h0, STEPS, WL.n_x)
    full = np.zeros((WL.n_x, WL.n_M), np.float32)
    full[rows] = oracle.kernel_rows(oracle.params(WL), V, rows).astype(np.float32)
    # n_M = Q: the half period is columns M = 0 .. Q/2 - 1 of the full rows
    half = np.ascontiguousarray(full[:, WL.n_M // 2: WL.n_M // 2 + WL.Q // 2])
    ref, st = oracle.simulate(oracle.params(WL), h0, 1, STEPS, table=full)
    got, c = gpu_run_table(wmc, torch, wmc.Params.of(WL), half, h0, 1, STEPS)
    np.testing.assert_array_equal(got, ref)
    for key, idx in (("pairs", oracle.ST_PAIRS), ("absorbed", oracle.ST_ABSORBED),
                     ("absorbed_signed", oracle.ST_ABSORBED_SIGNED), ("dropped", oracle.ST_DROPPED),
                     ("dropped_signed", oracle.ST_DROPPED_SIGNED), ("particle_steps", oracle.ST_PARTICLE_STEPS)):
        assert c[key] == st[idx], key
    assert st[oracle.ST_PAIRS] > 100_000 * STEPS
    assert c["flags"] == 0
    # net sign: pairs add +s and -s, so the change is the absorbed and dropped signs
    assert int(ref.sum()) == int(h0.sum()) - st[oracle.ST_ABSORBED_SIGNED] - st[oracle.ST_DROPPED_SIGNED]


@pytest.mark.parametrize("form", ["fp32", "fp32_simt", "fp16_split"])
def test_c3_production_loop_density(wmc, form):
    """wmc_run with the kernel computed in the loop (CUDA graph) against the
    oracle's FP64 run over the first five steps."""
    h0 = _h0()
    ref, st = _oracle_fp64_run()
    got, c = gpu_run(wmc, torch, wmc.Params.of(WL), wi.potential(WL), h0, 1, STEPS, prec=wmc.PRECISIONS[form])
    l1 = np.abs(got.sum(axis=1).astype(np.int64) - ref.sum(axis=1)).sum() / WL.packet.n0
    assert l1 <= DENSITY_L1_TOL, (form, l1)
    assert c["flags"] == 0
    assert c["pairs"] > 100_000 * STEPS
    assert abs(int(c["pairs"]) - int(st[oracle.ST_PAIRS])) <= 1e-3 * st[oracle.ST_PAIRS]
