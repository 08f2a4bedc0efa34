"""Thin Python binding of libwmc (include/wmc.h): argument marshalling only.

Every function here has the name of the C entry point without the ``wmc_``
prefix, takes torch CUDA tensors for device buffers and passes their data
pointers, with the current torch stream, to the library.  All the work runs in
libwmc's kernels; if the library is missing this module raises at import of
the first call, there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libwmc.so")

FP32, BF16, FP16, FP16_SPLIT, TF32X3, FP32_SIMT = 0, 1, 2, 3, 4, 5
PRECISIONS = {"fp32": FP32, "bf16": BF16, "fp16": FP16, "fp16_split": FP16_SPLIT, "tf32x3": TF32X3,
              "fp32_simt": FP32_SIMT}

FLAG_RATE, FLAG_CAPACITY, FLAG_TIMEOUT = 1, 2, 4
STATUS = {0: "ok", 1: "invalid argument", 2: "capacity exceeded", 3: "gamma dt >= 1", 4: "CUDA error",
          5: "device wait timed out", 6: "unsupported"}

# Every entry point include/wmc.h declares (checked by the tests).
EXPORTS = (
    "wmc_version", "wmc_status_string", "wmc_workspace_size", "wmc_init", "wmc_reset_counters",
    "wmc_get_counters", "wmc_kernel_eval", "wmc_kernel_cdf", "wmc_annihilate", "wmc_kernel_eval_occupied",
    "wmc_kernel_table_occupied", "wmc_step", "wmc_run", "wmc_density", "wmc_materialize", "wmc_philox4x32_10",
    "wmc_kernel_eval_noalloc", "wmc_batch_workspace_size", "wmc_batch_layout", "wmc_batch_init", "wmc_batch_run",
    "wmc_batch_autotune", "wmc_batch_get_counters", "wmc_potential_tanh", "wmc_potential_tanh_vjp",
    "wmc_kernel_eval_rows", "wmc_kernel_vjp", "wmc_check_wait", "wmc_step_timing", "wmc_step_timing_read",
    "wmc_get_error", "wmc_philox_throughput", "wmc_kernel_eval_n2", "wmc_set_id_base",
    "wmc_kernel_eval_dft",
    "wmc_n2_train",
    "wmc_n2_eval",
)


class WmcError(RuntimeError):
    def __init__(self, fn: str, code: int):
        super().__init__(f"{fn}: {STATUS.get(code, code)} (status {code})")
        self.code = code


class Params(ctypes.Structure):
    """wmc_params (include/wmc.h)."""

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

    @classmethod
    def of(cls, obj, **override) -> "Params":
        """From any object (or dict) with the same attribute names."""
        get = (lambda k: obj[k]) if isinstance(obj, dict) else (lambda k: getattr(obj, k))
        vals = {}
        for name, _ in cls._fields_:
            vals[name] = override[name] if name in override else get(name)
        return cls(**vals)

    @property
    def h(self) -> int:
        return self.Q // 2


class Counters(ctypes.Structure):
    _fields_ = [
        ("population", ctypes.c_uint64),
        ("particle_steps", ctypes.c_uint64),
        ("pairs", ctypes.c_uint64),
        ("absorbed", ctypes.c_uint64),
        ("absorbed_signed", ctypes.c_int64),
        ("dropped", ctypes.c_uint64),
        ("dropped_signed", ctypes.c_int64),
        ("n_occ", ctypes.c_int32),
        ("n_items", ctypes.c_int32),
        ("flags", ctypes.c_uint32),
        ("step", ctypes.c_uint32),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


_lib = None
_lock = threading.Lock()


def load(path: str | None = None):
    """Loads libwmc.so (built by ``paper_1806_00082_gb300.build``); raises if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libwmc is not built ({p} missing): run paper_1806_00082_gb300.build.build()")
        lib = ctypes.CDLL(p)
        vp, i32, u32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_int64
        pp = ctypes.POINTER(Params)
        sig = {
            "wmc_version": ([], ctypes.c_char_p),
            "wmc_status_string": ([i32], ctypes.c_char_p),
            "wmc_workspace_size": ([pp], ctypes.c_size_t),
            "wmc_init": ([pp, vp, ctypes.c_size_t, vp], i32),
            "wmc_reset_counters": ([pp, vp, vp], i32),
            "wmc_get_counters": ([pp, vp, ctypes.POINTER(Counters), vp], i32),
            "wmc_kernel_eval": ([pp, vp, vp, i32, i32, vp, vp, vp], i32),
            "wmc_kernel_cdf": ([pp, vp, i32, vp, vp, vp, vp], i32),
            "wmc_annihilate": ([pp, vp, vp, vp, vp], i32),
            "wmc_kernel_eval_occupied": ([pp, vp, i32, vp, vp], i32),
            "wmc_kernel_table_occupied": ([pp, vp, vp, vp], i32),
            "wmc_step": ([pp, vp, u32, vp, vp, vp], i32),
            "wmc_run": ([pp, vp, vp, vp, u32, i32, i32, i32, vp, vp], i32),
            "wmc_density": ([pp, vp, vp, vp], i32),
            "wmc_materialize": ([pp, vp, u32, vp, vp, vp, vp, i64, vp, vp], i32),
            "wmc_philox4x32_10": ([vp, u32, u32, i64, vp, vp], i32),
            "wmc_check_wait": ([pp, vp, ctypes.c_uint64, vp, vp], i32),
            "wmc_step_timing": ([i32], i32),
            "wmc_step_timing_read": ([ctypes.POINTER(ctypes.c_float)], i32),
            "wmc_kernel_eval_noalloc": ([pp, vp, vp, i32, vp, vp], i32),
            "wmc_batch_workspace_size": ([pp, i32], ctypes.c_size_t),
            "wmc_batch_layout": ([pp, i32, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)], i32),
            "wmc_batch_init": ([pp, i32, vp, ctypes.c_size_t, vp], i32),
            "wmc_batch_run": ([pp, i32, vp, vp, vp, u32, i32, i32, i32, vp, vp], i32),
            "wmc_batch_autotune": ([pp, i32, vp, vp, vp, u32, vp, ctypes.POINTER(ctypes.c_int32), vp], i32),
            "wmc_batch_get_counters": ([pp, i32, vp, ctypes.POINTER(Counters), vp], i32),
            "wmc_potential_tanh": ([pp, vp, i32, i32, i32, ctypes.c_float, vp, vp], i32),
            "wmc_potential_tanh_vjp": ([pp, vp, i32, i32, i32, ctypes.c_float, vp, vp, vp], i32),
            "wmc_kernel_eval_rows": ([pp, vp, i32, i32, vp, vp, vp], i32),
            "wmc_kernel_vjp": ([pp, vp, vp, vp, i32, vp, vp, vp, vp], i32),
            "wmc_kernel_eval_n2": ([pp, vp, vp, i32, i32, vp, vp, vp], i32),
            "wmc_set_id_base": ([pp, vp, ctypes.c_uint64, vp], i32),
            "wmc_kernel_eval_dft": ([pp, vp, vp, vp, vp], i32),
            "wmc_n2_train": ([pp, i32, vp, vp, i32, vp, i32, vp, vp, vp, vp], i32),
            "wmc_n2_eval": ([pp, vp, vp, i32, vp, vp], i32),
            "wmc_get_error": ([pp, vp, vp, ctypes.POINTER(ctypes.c_int32), ctypes.c_char_p, ctypes.c_size_t], i32),
            "wmc_philox_throughput": ([u32, u32, i32, vp, i64, vp], i32),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
        return lib


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("libwmc device arguments must be CUDA tensors")
    if not t.is_contiguous():
        raise ValueError("libwmc device arguments must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _check(name: str, code: int):
    if code != 0:
        raise WmcError(name, code)


def version() -> str:
    return load().wmc_version().decode()


def workspace_size(p: Params) -> int:
    return load().wmc_workspace_size(ctypes.byref(p))


def workspace(p: Params, device=None) -> torch.Tensor:
    n = workspace_size(p)
    if n == 0:
        raise WmcError("wmc_workspace_size", 1)
    return torch.empty(n, dtype=torch.uint8, device=device or "cuda")


def init(p: Params, ws: torch.Tensor) -> None:
    _check("wmc_init", load().wmc_init(ctypes.byref(p), _ptr(ws), ws.numel(), _stream()))


def reset_counters(p: Params, ws: torch.Tensor) -> None:
    _check("wmc_reset_counters", load().wmc_reset_counters(ctypes.byref(p), _ptr(ws), _stream()))


def check_wait(p: Params, signal: torch.Tensor, max_cycles: int, ws: torch.Tensor) -> None:
    """wmc_check_wait: a bounded device wait on signal (uint32/int32 [1]); sets
    the timeout flag in ws if nothing sets the word within max_cycles."""
    _check("wmc_check_wait", load().wmc_check_wait(ctypes.byref(p), _ptr(signal), int(max_cycles), _ptr(ws),
                                                   _stream()))


def step_timing(enable: bool) -> None:
    """wmc_step_timing: switches the library's events around the particle-step
    kernel on or off."""
    _check("wmc_step_timing", load().wmc_step_timing(1 if enable else 0))


def step_timing_read() -> float:
    """wmc_step_timing_read: milliseconds of the last particle-step kernel that
    ran with timing on (waits for it)."""
    ms = ctypes.c_float(0.0)
    _check("wmc_step_timing_read", load().wmc_step_timing_read(ctypes.byref(ms)))
    return float(ms.value)


def get_counters(p: Params, ws: torch.Tensor) -> dict:
    c = Counters()
    _check("wmc_get_counters", load().wmc_get_counters(ctypes.byref(p), _ptr(ws), ctypes.byref(c), _stream()))
    return c.as_dict()


def set_id_base(p: Params, ws: torch.Tensor, id_base: int) -> None:
    _check("wmc_set_id_base", load().wmc_set_id_base(ctypes.byref(p), _ptr(ws), int(id_base), _stream()))


def get_error(p: Params, ws: torch.Tensor) -> tuple:
    """(status code, message) of the workspace's device conditions; synchronises."""
    st = ctypes.c_int32(0)
    buf = ctypes.create_string_buffer(160)
    _check("wmc_get_error", load().wmc_get_error(ctypes.byref(p), _ptr(ws), _stream(), ctypes.byref(st), buf,
                                                   ctypes.sizeof(buf)))
    return int(st.value), buf.value.decode()


def philox_throughput(out: torch.Tensor, pairs_per_thread: int, key0: int = 1, key1: int = 2) -> None:
    """Generator throughput probe: out.numel() threads (a multiple of 256), 2 pairs_per_thread calls each."""
    _check("wmc_philox_throughput", load().wmc_philox_throughput(key0 & 0xFFFFFFFF, key1 & 0xFFFFFFFF,
                                                                   int(pairs_per_thread), _ptr(out), out.numel(),
                                                                   _stream()))


def kernel_eval(p: Params, V: torch.Tensor, occ: torch.Tensor, ws: torch.Tensor, prec: int = FP32,
                out: torch.Tensor | None = None) -> torch.Tensor:
    n = occ.numel()
    if out is None:
        out = torch.empty((n, p.h), dtype=torch.float32, device=V.device)
    _check("wmc_kernel_eval", load().wmc_kernel_eval(ctypes.byref(p), _ptr(V), _ptr(occ), n, prec, _ptr(out),
                                                     _ptr(ws), _stream()))
    return out


def kernel_eval_n2(p: Params, V: torch.Tensor, occ: torch.Tensor, ws: torch.Tensor, prec: int = FP32,
                   out: torch.Tensor | None = None) -> torch.Tensor:
    """wmc_kernel_eval_n2: half-period rows of the N = 2 barycentric network."""
    n = occ.numel()
    if out is None:
        out = torch.empty((n, p.h), dtype=torch.float32, device=V.device)
    _check("wmc_kernel_eval_n2", load().wmc_kernel_eval_n2(ctypes.byref(p), _ptr(V), _ptr(occ), n, prec, _ptr(out),
                                                           _ptr(ws), _stream()))
    return out


def kernel_eval_dft(p: Params, V: torch.Tensor, ws: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
    """wmc_kernel_eval_dft: every cell's half-period row by the FP64 sliding window."""
    if out is None:
        out = torch.empty((p.n_x, p.h), dtype=torch.float32, device=V.device)
    _check("wmc_kernel_eval_dft", load().wmc_kernel_eval_dft(ctypes.byref(p), _ptr(V), _ptr(out), _ptr(ws),
                                                             _stream()))
    return out


def n2_train(p: Params, V: torch.Tensor, VW: torch.Tensor, order: torch.Tensor, lr: torch.Tensor,
             params: torch.Tensor, loss: torch.Tensor | None = None) -> None:
    """wmc_n2_train: SGD of the trained N = 2 network; params [n_runs, Q + 4] updated in place."""
    n_ex, epochs, n_runs = V.shape[0], order.shape[0], lr.numel()
    _check("wmc_n2_train", load().wmc_n2_train(ctypes.byref(p), n_ex, _ptr(V), _ptr(VW), epochs, _ptr(order),
                                               n_runs, _ptr(lr), _ptr(params),
                                               _ptr(loss) if loss is not None else None, _stream()))


def n2_eval(p: Params, params: torch.Tensor, V: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
    """wmc_n2_eval: rows [n_pot * n_x, Q/2] of the trained N = 2 network in 1/s."""
    V2 = V.reshape(-1, p.n_x)
    if out is None:
        out = torch.empty((V2.shape[0] * p.n_x, p.h), dtype=torch.float32, device=V.device)
    _check("wmc_n2_eval", load().wmc_n2_eval(ctypes.byref(p), _ptr(params), _ptr(V2), V2.shape[0], _ptr(out),
                                             _stream()))
    return out


def kernel_eval_noalloc(p: Params, V: torch.Tensor, occ: torch.Tensor, out: torch.Tensor) -> torch.Tensor:
    """wmc_kernel_eval_noalloc: no workspace, the library allocates nothing
    (scratch in a fixed device array, Q <= 1024); out is [n_occ, Q/2] FP32."""
    _check("wmc_kernel_eval_noalloc", load().wmc_kernel_eval_noalloc(ctypes.byref(p), _ptr(V), _ptr(occ),
                                                                     occ.numel(), _ptr(out), _stream()))
    return out


def kernel_cdf(p: Params, VWh: torch.Tensor, with_cdf: bool = True):
    """(cdf int64 [n, n_M] or None, gamma float64 [n], scale int32 [n])."""
    n = VWh.shape[0]
    cdf = torch.empty((n, p.n_M), dtype=torch.int64, device=VWh.device) if with_cdf else None
    gamma = torch.empty(n, dtype=torch.float64, device=VWh.device)
    scale = torch.empty(n, dtype=torch.int32, device=VWh.device)
    _check("wmc_kernel_cdf", load().wmc_kernel_cdf(ctypes.byref(p), _ptr(VWh), n, _ptr(cdf), _ptr(gamma),
                                                   _ptr(scale), _stream()))
    return cdf, gamma, scale


def annihilate(p: Params, hist: torch.Tensor, ws: torch.Tensor, rho: torch.Tensor | None = None):
    _check("wmc_annihilate", load().wmc_annihilate(ctypes.byref(p), _ptr(hist), _ptr(rho), _ptr(ws), _stream()))
    return rho


def kernel_eval_occupied(p: Params, V: torch.Tensor, ws: torch.Tensor, prec: int = FP32) -> None:
    _check("wmc_kernel_eval_occupied",
           load().wmc_kernel_eval_occupied(ctypes.byref(p), _ptr(V), prec, _ptr(ws), _stream()))


def kernel_table_occupied(p: Params, table: torch.Tensor, ws: torch.Tensor) -> None:
    _check("wmc_kernel_table_occupied",
           load().wmc_kernel_table_occupied(ctypes.byref(p), _ptr(table), _ptr(ws), _stream()))


def step(p: Params, hist_in: torch.Tensor, t: int, hist_out: torch.Tensor, ws: torch.Tensor) -> None:
    _check("wmc_step", load().wmc_step(ctypes.byref(p), _ptr(hist_in), t, _ptr(hist_out), _ptr(ws), _stream()))


def run(p: Params, V: torch.Tensor, hist_a: torch.Tensor, hist_b: torch.Tensor, t_first: int, n_steps: int,
        ws: torch.Tensor, prec: int = FP32, use_graph: bool = True) -> None:
    _check("wmc_run", load().wmc_run(ctypes.byref(p), _ptr(V), _ptr(hist_a), _ptr(hist_b), t_first, n_steps, prec,
                                     1 if use_graph else 0, _ptr(ws), _stream()))


def density(p: Params, hist: torch.Tensor, rho: torch.Tensor | None = None) -> torch.Tensor:
    if rho is None:
        rho = torch.empty(p.n_x, dtype=torch.int64, device=hist.device)
    _check("wmc_density", load().wmc_density(ctypes.byref(p), _ptr(hist), _ptr(rho), _stream()))
    return rho


def materialize(p: Params, hist: torch.Tensor, t: int, ws: torch.Tensor, capacity: int):
    dev = hist.device
    cell = torch.empty(capacity, dtype=torch.int32, device=dev)
    f = torch.empty(capacity, dtype=torch.float32, device=dev)
    M = torch.empty(capacity, dtype=torch.int16, device=dev)
    s = torch.empty(capacity, dtype=torch.int8, device=dev)
    _check("wmc_materialize", load().wmc_materialize(ctypes.byref(p), _ptr(hist), t, _ptr(cell), _ptr(f), _ptr(M),
                                                     _ptr(s), capacity, _ptr(ws), _stream()))
    return cell, f, M, s


def philox4x32_10(ctr: torch.Tensor, key0: int, key1: int) -> torch.Tensor:
    """ctr: uint32-valued int32/int64 CUDA tensor [n, 4] (viewed as 32-bit words)."""
    c = ctr.to(torch.int32).contiguous()
    out = torch.empty_like(c)
    _check("wmc_philox4x32_10", load().wmc_philox4x32_10(_ptr(c), key0 & 0xFFFFFFFF, key1 & 0xFFFFFFFF,
                                                         c.shape[0], _ptr(out), _stream()))
    return out


# ---------------------------------------------------------------- batched form
def params_array(ps) -> ctypes.Array:
    arr = (Params * len(ps))()
    for q, p in enumerate(ps):
        arr[q] = p
    return arr


def batch_layout(ps_arr) -> tuple:
    n = len(ps_arr)
    co = (ctypes.c_int64 * (n + 1))()
    ho = (ctypes.c_int64 * (n + 1))()
    _check("wmc_batch_layout", load().wmc_batch_layout(ps_arr, n, co, ho))
    return list(co), list(ho)


def batch_workspace(ps_arr, device=None) -> torch.Tensor:
    nbytes = load().wmc_batch_workspace_size(ps_arr, len(ps_arr))
    if nbytes == 0:
        raise WmcError("wmc_batch_workspace_size", 1)
    return torch.empty(nbytes, dtype=torch.uint8, device=device or "cuda")


def batch_init(ps_arr, ws: torch.Tensor) -> None:
    _check("wmc_batch_init", load().wmc_batch_init(ps_arr, len(ps_arr), _ptr(ws), ws.numel(), _stream()))


def batch_run(ps_arr, V: torch.Tensor, hist_a: torch.Tensor, hist_b: torch.Tensor, t_first: int, n_steps: int,
              ws: torch.Tensor, per_thread: int = 0, use_graph: bool = True) -> None:
    _check("wmc_batch_run", load().wmc_batch_run(ps_arr, len(ps_arr), _ptr(V), _ptr(hist_a), _ptr(hist_b), t_first,
                                                 n_steps, per_thread, 1 if use_graph else 0, _ptr(ws), _stream()))


def batch_autotune(ps_arr, V: torch.Tensor, hist: torch.Tensor, scratch: torch.Tensor, t: int,
                   ws: torch.Tensor) -> int:
    best = ctypes.c_int32(0)
    _check("wmc_batch_autotune", load().wmc_batch_autotune(ps_arr, len(ps_arr), _ptr(V), _ptr(hist), _ptr(scratch),
                                                           t, _ptr(ws), ctypes.byref(best), _stream()))
    return best.value


def batch_get_counters(ps_arr, ws: torch.Tensor) -> dict:
    c = Counters()
    _check("wmc_batch_get_counters", load().wmc_batch_get_counters(ps_arr, len(ps_arr), _ptr(ws), ctypes.byref(c),
                                                                   _stream()))
    return c.as_dict()


# ---------------------------------------------------------------- differentiation form
def potential_tanh(p: Params, theta: torch.Tensor, n_barriers: int, n_segments: int, eps_nm: float) -> torch.Tensor:
    n_pot = theta.shape[0]
    V = torch.empty((n_pot, p.n_x), dtype=torch.float32, device=theta.device)
    _check("wmc_potential_tanh", load().wmc_potential_tanh(ctypes.byref(p), _ptr(theta), n_pot, n_barriers,
                                                           n_segments, eps_nm, _ptr(V), _stream()))
    return V


def potential_tanh_vjp(p: Params, theta: torch.Tensor, n_barriers: int, n_segments: int, eps_nm: float,
                       Vbar: torch.Tensor) -> torch.Tensor:
    tb = torch.empty_like(theta)
    _check("wmc_potential_tanh_vjp", load().wmc_potential_tanh_vjp(ctypes.byref(p), _ptr(theta), theta.shape[0],
                                                                   n_barriers, n_segments, eps_nm, _ptr(Vbar),
                                                                   _ptr(tb), _stream()))
    return tb


def kernel_eval_rows(p: Params, V: torch.Tensor, ws: torch.Tensor, prec: int = FP32) -> torch.Tensor:
    n_pot = V.shape[0]
    out = torch.empty((n_pot * p.n_x, p.h), dtype=torch.float32, device=V.device)
    _check("wmc_kernel_eval_rows", load().wmc_kernel_eval_rows(ctypes.byref(p), _ptr(V), n_pot, prec, _ptr(out),
                                                               _ptr(ws), _stream()))
    return out


def kernel_vjp(p: Params, VWh: torch.Tensor, gVW, g_gamma, n_pot: int, ws: torch.Tensor) -> torch.Tensor:
    abar = torch.empty_like(VWh)
    Vbar = torch.empty((n_pot, p.n_x), dtype=torch.float32, device=VWh.device)
    _check("wmc_kernel_vjp", load().wmc_kernel_vjp(ctypes.byref(p), _ptr(VWh), _ptr(gVW), _ptr(g_gamma), n_pot,
                                                   _ptr(abar), _ptr(Vbar), _ptr(ws), _stream()))
    return Vbar
