"""Helpers shared by the GPU parity tests: oracle-side tables and the libwmc
call sequences the tests drive (through the C ABI binding)."""
import numpy as np

import oracle

_cache = {}


def oracle_tables(w, V):
    """FP64 oracle kernel of every cell, as (full FP32 table [n_x, n_M] for the
    oracle simulator, half-period FP32 table [n_x, Q/2] for libwmc).  Both hold
    the same rounded values: the oracle kernel is exactly odd and Q-periodic."""
    key = (w.name, w.n_x, w.Q, w.n_M, w.bc_potential, V.tobytes())
    if key in _cache:
        return _cache[key]
    p = oracle.params(w)
    full = oracle.kernel_rows(p, V, np.arange(w.n_x)).astype(np.float32)
    h = w.Q // 2
    ph = oracle.params(w.replace(n_M=w.Q))
    half = oracle.kernel_rows(ph, V, np.arange(w.n_x))[:, h:2 * h].astype(np.float32)
    _cache[key] = (full, np.ascontiguousarray(half))
    return full, half


def gpu_run_table(wmc, torch, p, half_table, hist0, t_first, n_steps):
    """Steps driven call by call with the kernel taken from a table."""
    ws = wmc.workspace(p)
    wmc.init(p, ws)
    tab = torch.from_numpy(half_table).cuda()
    a = torch.from_numpy(np.ascontiguousarray(hist0, dtype=np.int32)).cuda()
    b = torch.empty_like(a)
    for st in range(n_steps):
        wmc.annihilate(p, a, ws)
        wmc.kernel_table_occupied(p, tab, ws)
        wmc.step(p, a, t_first + st, b, ws)
        a, b = b, a
    out = a.cpu().numpy()
    return out, wmc.get_counters(p, ws)


def gpu_run(wmc, torch, p, V, hist0, t_first, n_steps, use_graph=True, prec=None):
    """Production loop: wmc_run with the kernel (FP32 unless prec says otherwise)
    evaluated on occupied cells."""
    ws = wmc.workspace(p)
    wmc.init(p, ws)
    Vd = torch.from_numpy(np.ascontiguousarray(V, dtype=np.float32)).cuda()
    a = torch.from_numpy(np.ascontiguousarray(hist0, dtype=np.int32)).cuda()
    b = torch.empty_like(a)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        wmc.run(p, Vd, a, b, t_first, n_steps, ws, wmc.FP32 if prec is None else prec, use_graph)
        c = wmc.get_counters(p, ws)
    s.synchronize()
    return a.cpu().numpy(), c


def normwise(a, b):
    return float(np.max(np.abs(np.asarray(a, np.float64) - b)) / max(np.max(np.abs(b)), 1e-300))


def full_from_half(half, Q, n_M):
    """Kernel rows over the momentum grid M = k - n_M/2 from half-period rows
    (V_W odd and Q-periodic in M, zero at M = 0 and M = Q/2): the layout the
    oracle's simulator takes a table in."""
    h = Q // 2
    half = np.asarray(half, np.float32)
    r = (np.arange(n_M) - n_M // 2) % Q
    out = np.zeros((half.shape[0], n_M), np.float32)
    lo = (r > 0) & (r < h)
    hi = r > h
    out[:, lo] = half[:, r[lo]]
    out[:, hi] = -half[:, Q - r[hi]]
    return out


def reach_rows(hist0, n_steps, n_x):
    """Cells a particle of hist0 can be in during the next n_steps steps (a
    drift moves at most one cell per step)."""
    occ = np.flatnonzero(np.abs(hist0).sum(axis=1))
    if occ.size == 0:
        return occ
    lo, hi = max(0, occ.min() - n_steps - 1), min(n_x, occ.max() + n_steps + 2)
    return np.arange(lo, hi)
