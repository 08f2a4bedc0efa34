"""CPU oracle for the signed-particle Wigner Monte Carlo hot path (arXiv:1806.00082).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the benchmark's
CPU-baseline leg are the only callers.  The oracle is plain, sequential FP64 C
(``wmc_oracle.c``) behind ctypes; it shares no code, header or table with the
CUDA path and never imports it.

Functions and the passages they follow:

- :func:`kernel_rows` -- Eq. (wigner-1d-discrete): the finite-window discrete
  Wigner kernel, summed over m = -h..h (h = L_C / (2 dx)) in FP64.
- :func:`kernel_all_dft` -- the same sum for every cell by a sliding window
  over exp(i 2 pi l M / Q)-weighted potentials, O(n_x n_M), FP64.
- :func:`kernel_rows_n2` -- Eq. (kernel_ML) with N = 2 and the barycentric
  weights of Sec. 2.3: consecutive cells grouped in pairs, FP64.
- :func:`cdf_row` -- Eq. (momentum_integral): gamma as the sum of V_W^+ over M
  and the CDF for drawing p' ~ V_W^+ / gamma, as exact sums of V_W^+ quantised
  to 62-bit fixed point relative to the row maximum.
- :func:`philox` -- Philox4x32-10 from Salmon et al., SC'11.
- :func:`materialize` -- rule 2 survivors re-emitted in (cell, M) order.
- :func:`simulate` -- the postulate of Sec. 2.1 (free drift, pair creation with
  probability gamma dt, momenta p +- p') with rules 1 and 2, step by step;
  :func:`simulate_subdomain` one step of a range of cells whose particles are
  numbered after those of the cells before it.
- :func:`density` -- rule 1: signed counts summed over M.

``oracle/adjoint.py`` holds the differentiation form's FP64 adjoint and
``oracle/n2train.py`` the trained N = 2 network of Sec. 2.3 (model, MSE loss,
gradients and SGD), both in numpy.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wmc_oracle.c")
_LIB = os.path.join(_HERE, "lib", "libwmc_oracle.so")
_lock = threading.Lock()
_lib = None

# indices into the statistics vector returned by simulate()
ST_PAIRS, ST_ABSORBED, ST_ABSORBED_SIGNED, ST_DROPPED, ST_DROPPED_SIGNED = 0, 1, 2, 3, 4
ST_RATE, ST_POP, ST_NET, ST_PARTICLE_STEPS, ST_ERR, ST_N = 5, 6, 7, 8, 9, 10


class Params(ctypes.Structure):
    """The oracle's own copy of the run parameters (same meaning as the library's)."""

    _fields_ = [
        ("dx_m", ctypes.c_double),
        ("mass_kg", ctypes.c_double),
        ("dt_s", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("n_x", ctypes.c_int32),
        ("Q", ctypes.c_int32),
        ("n_M", ctypes.c_int32),
        ("bc_potential", ctypes.c_int32),
        ("child_wrap", ctypes.c_int32),
        ("sim", ctypes.c_uint32),
    ]


def params(w, sim: int | None = None) -> Params:
    """Oracle parameters from a workload description (see ``wmc_inputs.Workload``)."""
    return Params(
        dx_m=w.dx_m, mass_kg=w.mass_kg, dt_s=w.dt_s, seed=w.seed, n_x=w.n_x, Q=w.Q, n_M=w.n_M,
        bc_potential=w.bc_potential, child_wrap=w.child_wrap, sim=w.sim if sim is None else sim,
    )


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction) into oracle/lib/."""
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
            return _LIB
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
             "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        u32p, i32p, i64p = P(ctypes.c_uint32), P(ctypes.c_int32), P(ctypes.c_int64)
        f32p, f64p, i16p, i8p = P(ctypes.c_float), P(ctypes.c_double), P(ctypes.c_int16), P(ctypes.c_int8)
        pp = P(Params)
        lib.wmco_philox4x32_10.argtypes = [u32p, u32p, u32p]
        lib.wmco_u53.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
        lib.wmco_u53.restype = ctypes.c_double
        lib.wmco_u24.argtypes = [ctypes.c_uint32]
        lib.wmco_u24.restype = ctypes.c_float
        lib.wmco_u32.argtypes = [ctypes.c_uint32]
        lib.wmco_u32.restype = ctypes.c_double
        lib.wmco_sine.argtypes = [ctypes.c_int32, ctypes.c_int64]
        lib.wmco_sine.restype = ctypes.c_double
        lib.wmco_kernel_value.argtypes = [pp, f64p, ctypes.c_int32, ctypes.c_int32]
        lib.wmco_kernel_value.restype = ctypes.c_double
        lib.wmco_kernel_rows.argtypes = [pp, f64p, ctypes.c_int32, i32p, f64p]
        lib.wmco_kernel_rows_n2.argtypes = [pp, f64p, ctypes.c_int32, i32p, f64p]
        lib.wmco_kernel_all_dft.argtypes = [pp, f64p, f64p]
        lib.wmco_cdf_row.argtypes = [ctypes.c_int32, f64p, i64p, i32p]
        lib.wmco_cdf_row.restype = ctypes.c_double
        lib.wmco_sample_row.argtypes = [ctypes.c_int32, i64p, ctypes.c_uint64]
        lib.wmco_sample_row.restype = ctypes.c_int32
        lib.wmco_u53_bits.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
        lib.wmco_u53_bits.restype = ctypes.c_uint64
        lib.wmco_drift_table.argtypes = [pp, f32p]
        lib.wmco_population.argtypes = [pp, i32p]
        lib.wmco_population.restype = ctypes.c_int64
        lib.wmco_materialize.argtypes = [pp, i32p, ctypes.c_uint32, ctypes.c_int64, i32p, f32p, i16p, i8p]
        lib.wmco_materialize.restype = ctypes.c_int64
        lib.wmco_density.argtypes = [pp, i32p, i64p]
        lib.wmco_simulate.argtypes = [pp, f64p, f32p, i32p, ctypes.c_uint32, ctypes.c_int32, i32p, i64p]
        lib.wmco_simulate.restype = ctypes.c_int32
        lib.wmco_simulate_subdomain.argtypes = [pp, f64p, f32p, i32p, ctypes.c_uint32, ctypes.c_uint64, i32p, i64p]
        lib.wmco_simulate_subdomain.restype = ctypes.c_int32
        _lib = lib
    return _lib


def _ptr(a: np.ndarray, ctype):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 of one 4-word counter under a 2-word key."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.wmco_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32), _ptr(out, ctypes.c_uint32))
    return out


def u53(a: int, b: int) -> float:
    return _load().wmco_u53(a, b)


def u24(a: int) -> float:
    return _load().wmco_u24(a)


def u32(a: int) -> float:
    return _load().wmco_u32(a)


def sine(Q: int, t: int) -> float:
    """sin(2 pi t / Q) with exact integer reduction."""
    return _load().wmco_sine(Q, t)


def kernel_value(p: Params, V: np.ndarray, i: int, M: int) -> float:
    V64 = np.ascontiguousarray(V, dtype=np.float64)
    return _load().wmco_kernel_value(ctypes.byref(p), _ptr(V64, ctypes.c_double), i, M)


def kernel_rows(p: Params, V: np.ndarray, rows) -> np.ndarray:
    """V_W(rows[r]; k - n_M/2) for k in [0, n_M): array [len(rows), n_M] in 1/s."""
    V64 = np.ascontiguousarray(V, dtype=np.float64)
    r = np.ascontiguousarray(rows, dtype=np.int32)
    out = np.zeros((r.size, p.n_M), dtype=np.float64)
    _load().wmco_kernel_rows(ctypes.byref(p), _ptr(V64, ctypes.c_double), r.size, _ptr(r, ctypes.c_int32),
                             _ptr(out, ctypes.c_double))
    return out


def kernel_all_dft(p: Params, V: np.ndarray) -> np.ndarray:
    """Eq. (wigner-1d-discrete) on every cell by the sliding window of
    exp(i 2 pi l M / Q)-weighted potentials: [n_x, n_M] in 1/s, FP64."""
    V64 = np.ascontiguousarray(V, dtype=np.float64)
    out = np.zeros((p.n_x, p.n_M), dtype=np.float64)
    _load().wmco_kernel_all_dft(ctypes.byref(p), _ptr(V64, ctypes.c_double), _ptr(out, ctypes.c_double))
    return out


def kernel_rows_n2(p: Params, V: np.ndarray, rows) -> np.ndarray:
    """The N = 2 barycentric network of Eq. (kernel_ML) (Sec. 2.3):
    V_W2(rows[r]; k - n_M/2) for k in [0, n_M), array [len(rows), n_M] in 1/s."""
    V64 = np.ascontiguousarray(V, dtype=np.float64)
    r = np.ascontiguousarray(rows, dtype=np.int32)
    out = np.zeros((r.size, p.n_M), dtype=np.float64)
    _load().wmco_kernel_rows_n2(ctypes.byref(p), _ptr(V64, ctypes.c_double), r.size, _ptr(r, ctypes.c_int32),
                                _ptr(out, ctypes.c_double))
    return out


def cdf_row(vw_row: np.ndarray, with_scale: bool = False):
    """(cdf, gamma) of one kernel row: the exact running sum of V_W^+ quantised
    to 62-bit fixed point (int64 array) and gamma; with_scale adds the scale s."""
    v = np.ascontiguousarray(vw_row, dtype=np.float64)
    cdf = np.zeros(v.size, dtype=np.int64)
    s = ctypes.c_int32(0)
    g = _load().wmco_cdf_row(v.size, _ptr(v, ctypes.c_double), _ptr(cdf, ctypes.c_int64), ctypes.byref(s))
    return (cdf, g, s.value) if with_scale else (cdf, g)


def sample_row(cdf: np.ndarray, U2: int) -> int:
    """Index of p' for the 53-bit uniform integer U2."""
    c = np.ascontiguousarray(cdf, dtype=np.int64)
    return _load().wmco_sample_row(c.size, _ptr(c, ctypes.c_int64), U2)


def u53_bits(a: int, b: int) -> int:
    return _load().wmco_u53_bits(a, b)


def drift_table(p: Params) -> np.ndarray:
    D = np.zeros(p.n_M, dtype=np.float32)
    _load().wmco_drift_table(ctypes.byref(p), _ptr(D, ctypes.c_float))
    return D


def population(p: Params, hist: np.ndarray) -> int:
    h = np.ascontiguousarray(hist, dtype=np.int32)
    return _load().wmco_population(ctypes.byref(p), _ptr(h, ctypes.c_int32))


def materialize(p: Params, hist: np.ndarray, step: int):
    """Survivors of a net histogram as (cell, f, M, s) arrays in id order."""
    h = np.ascontiguousarray(hist, dtype=np.int32)
    P = population(p, h)
    cell = np.zeros(P, np.int32)
    f = np.zeros(P, np.float32)
    M = np.zeros(P, np.int16)
    s = np.zeros(P, np.int8)
    n = _load().wmco_materialize(ctypes.byref(p), _ptr(h, ctypes.c_int32), step & 0xFFFFFFFF, P,
                                 _ptr(cell, ctypes.c_int32), _ptr(f, ctypes.c_float),
                                 _ptr(M, ctypes.c_int16), _ptr(s, ctypes.c_int8))
    if n < 0:
        raise ValueError("population exceeds 2^32")
    return cell, f, M, s


def density(p: Params, hist: np.ndarray) -> np.ndarray:
    h = np.ascontiguousarray(hist, dtype=np.int32)
    rho = np.zeros(p.n_x, np.int64)
    _load().wmco_density(ctypes.byref(p), _ptr(h, ctypes.c_int32), _ptr(rho, ctypes.c_int64))
    return rho


def simulate(p: Params, hist0: np.ndarray, t_first: int, n_steps: int, V=None, table=None):
    """Run n_steps steps from the net histogram hist0 (state after the rebuild of
    step t_first - 1).  Either V (potential [n_x] in eV: the kernel is evaluated
    in FP64 on occupied cells) or table (FP32 [n_x, n_M] kernel values used as
    given).  Returns (hist, stats)."""
    lib = _load()
    h0 = np.ascontiguousarray(hist0, dtype=np.int32).reshape(-1)
    out = np.zeros_like(h0)
    stats = np.zeros(ST_N, np.int64)
    if table is not None:
        tab = np.ascontiguousarray(table, dtype=np.float32).reshape(-1)
        assert tab.size == p.n_x * p.n_M
        vptr = ctypes.POINTER(ctypes.c_double)()
        tptr = _ptr(tab, ctypes.c_float)
    else:
        V64 = np.ascontiguousarray(V, dtype=np.float64)
        vptr = _ptr(V64, ctypes.c_double)
        tptr = ctypes.POINTER(ctypes.c_float)()
    err = lib.wmco_simulate(ctypes.byref(p), vptr, tptr, _ptr(h0, ctypes.c_int32), t_first & 0xFFFFFFFF,
                            n_steps, _ptr(out, ctypes.c_int32), _ptr(stats, ctypes.c_int64))
    if err:
        raise RuntimeError(f"oracle simulate failed with code {err}")
    return out.reshape(p.n_x, p.n_M), stats


def simulate_subdomain(p: Params, hist: np.ndarray, t: int, id_base: int, V=None, table=None):
    """One step t of a sub-domain (its particles only in hist, full [n_x, n_M]
    layout) whose particles are numbered from id_base; particles leaving it
    land in the neighbouring rows of the result.  Returns (hist, stats)."""
    lib = _load()
    h0 = np.ascontiguousarray(hist, dtype=np.int32).reshape(-1)
    out = np.zeros_like(h0)
    stats = np.zeros(ST_N, np.int64)
    if table is not None:
        tab = np.ascontiguousarray(table, dtype=np.float32).reshape(-1)
        vptr = ctypes.POINTER(ctypes.c_double)()
        tptr = _ptr(tab, ctypes.c_float)
    else:
        V64 = np.ascontiguousarray(V, dtype=np.float64)
        vptr = _ptr(V64, ctypes.c_double)
        tptr = ctypes.POINTER(ctypes.c_float)()
    err = lib.wmco_simulate_subdomain(ctypes.byref(p), vptr, tptr, _ptr(h0, ctypes.c_int32), t & 0xFFFFFFFF,
                                      int(id_base), _ptr(out, ctypes.c_int32), _ptr(stats, ctypes.c_int64))
    if err:
        raise RuntimeError(f"oracle subdomain step failed with code {err}")
    return out.reshape(p.n_x, p.n_M), stats
