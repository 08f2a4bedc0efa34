"""Domain decomposition of one simulation over ranks by cell ranges.

The step of the postulate (Sec. 2.1) is local in space: a particle moves at
most one cell per step (|D| < 1), creates its pair in its post-drift cell and
is annihilated (rule 2) with the particles of that cell.  So one simulation
splits into contiguous cell ranges, one per rank:

- every rank holds the full potential (the kernel of a cell needs V within
  +-Q/2 cells of it) and the rows of its own cells;
- the particles are numbered globally in row-major (cell, M) order, so rank r
  numbers its particles after those of the cells before its range: an
  exclusive prefix of the ranks' populations (one gathered integer per rank);
- after its step a rank finds, in the row just left and just right of its
  range, the particles that drifted out (and the pairs they created there);
  it sends those rows to the neighbour that owns them and adds the rows it
  receives to its first and last row.

With the same Philox streams (global numbering) and the same kernel values
this is bit-for-bit the one-rank run.  The exchange is one neighbour send and
receive per step; the per-rank state here is the full [n_x, n_M] histogram,
zero outside the rank's cells.

The step itself is a callable ``step_fn(hist, t, id_base) -> (hist_out,
counters)`` supplied by the caller (libwmc on a GPU: ``gpu_step_fn``);
communication goes through a ``Comm`` (``TorchComm`` over torch.distributed,
gloo or NCCL) or ``emulate_ranks`` runs all ranks in one process.
"""
from __future__ import annotations

import numpy as np


class CellRanges:
    """Contiguous cell ranges [lo_r, hi_r) of n_x cells over world ranks
    (as equal as possible; every range holds at least one cell)."""

    def __init__(self, n_x: int, world: int):
        if world < 1 or n_x < world:
            raise ValueError("need 1 <= world <= n_x")
        self.n_x = n_x
        self.world = world
        self.bounds = [(r * n_x) // world for r in range(world + 1)]

    def range(self, rank: int) -> tuple:
        return self.bounds[rank], self.bounds[rank + 1]


def exclusive_prefix(values) -> list:
    """[0, v0, v0 + v1, ...] without the total."""
    out, acc = [], 0
    for v in values:
        out.append(acc)
        acc += int(v)
    return out


def population(hist, lo: int, hi: int) -> int:
    """Survivors in rows [lo, hi) of a signed histogram (numpy or torch)."""
    rows = hist[lo:hi]
    return int(rows.abs().sum()) if hasattr(rows, "abs") else int(np.abs(rows).sum())


def _copy(row):
    return row.clone() if hasattr(row, "clone") else row.copy()


def split_halo(out, lo: int, hi: int, n_x: int):
    """Takes the rows just outside [lo, hi) out of a rank's step result: the
    row lo - 1 (for the rank on the left) and the row hi (for the rank on the
    right), None at the domain's edges; both rows are zeroed in place."""
    left = _copy(out[lo - 1]) if lo > 0 else None
    right = _copy(out[hi]) if hi < n_x else None
    if lo > 0:
        out[lo - 1] = 0
    if hi < n_x:
        out[hi] = 0
    return left, right


def merge_halo(out, lo: int, hi: int, from_left, from_right) -> None:
    """Adds the rows received from the neighbours: the left rank's row lo
    (particles that moved right into this range) and the right rank's row
    hi - 1 (those that moved left into it)."""
    if from_left is not None:
        out[lo] += from_left
    if from_right is not None:
        out[hi - 1] += from_right


COUNTER_KEYS = ("pairs", "absorbed", "absorbed_signed", "dropped", "dropped_signed", "particle_steps")


class TorchComm:
    """Rank communication over torch.distributed (an initialised process
    group, gloo or NCCL): one integer gathered from every rank, and the halo
    rows sent to and received from the neighbours."""

    def __init__(self, device=None):
        import torch
        import torch.distributed as dist
        self.torch, self.dist = torch, dist
        self.rank = dist.get_rank()
        self.world = dist.get_world_size()
        self.device = device

    def allgather_int(self, v: int) -> list:
        t = self.torch.tensor([int(v)], dtype=self.torch.int64, device=self.device)
        out = [self.torch.zeros_like(t) for _ in range(self.world)]
        self.dist.all_gather(out, t)
        return [int(x.item()) for x in out]

    def allreduce_ints(self, vals) -> list:
        t = self.torch.tensor([int(v) for v in vals], dtype=self.torch.int64, device=self.device)
        self.dist.all_reduce(t)
        return [int(x) for x in t.tolist()]

    def exchange(self, to_left, to_right, like):
        """Sends to_left to rank - 1 and to_right to rank + 1 (None at an
        edge) and returns (row from rank - 1, row from rank + 1)."""
        torch, dist = self.torch, self.dist
        as_t = lambda a: a if torch.is_tensor(a) else torch.from_numpy(np.ascontiguousarray(a))
        ops, from_left, from_right = [], None, None
        if self.rank > 0:
            from_left = torch.empty_like(as_t(like)).to(self.device) if self.device else torch.empty_like(as_t(like))
            ops.append(dist.P2POp(dist.isend, as_t(to_left).contiguous().to(from_left.device), self.rank - 1))
            ops.append(dist.P2POp(dist.irecv, from_left, self.rank - 1))
        if self.rank + 1 < self.world:
            from_right = torch.empty_like(as_t(like)).to(self.device) if self.device else torch.empty_like(as_t(like))
            ops.append(dist.P2POp(dist.isend, as_t(to_right).contiguous().to(from_right.device), self.rank + 1))
            ops.append(dist.P2POp(dist.irecv, from_right, self.rank + 1))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        back = (lambda x: x) if torch.is_tensor(like) else (lambda x: None if x is None else x.cpu().numpy())
        return back(from_left), back(from_right)


def decomposed_step(comm, ranges: CellRanges, hist, t: int, step_fn):
    """One step t of this rank's cells: hist is the rank's [n_x, n_M] state
    (zero outside its range); returns (new state, this rank's counters)."""
    lo, hi = ranges.range(comm.rank)
    bases = exclusive_prefix(comm.allgather_int(population(hist, lo, hi)))
    out, counters = step_fn(hist, t, bases[comm.rank])
    to_left, to_right = split_halo(out, lo, hi, ranges.n_x)
    from_left, from_right = comm.exchange(to_left, to_right, out[lo])
    merge_halo(out, lo, hi, from_left, from_right)
    return out, counters


def emulate_ranks(states, ranges: CellRanges, t: int, step_fn):
    """The same step for all ranks in one process, one after another (no
    rank waits on another: the exchange happens after every rank's step);
    states[r] is rank r's [n_x, n_M] state.  Returns (states, counters per rank)."""
    pops = [population(h, *ranges.range(r)) for r, h in enumerate(states)]
    bases = exclusive_prefix(pops)
    outs, counters, halos = [], [], []
    for r, h in enumerate(states):
        out, c = step_fn(h, t, bases[r])
        outs.append(out)
        counters.append(c)
        halos.append(split_halo(out, *ranges.range(r), ranges.n_x))
    for r, out in enumerate(outs):
        lo, hi = ranges.range(r)
        merge_halo(out, lo, hi, halos[r - 1][1] if r > 0 else None,
                   halos[r + 1][0] if r + 1 < ranges.world else None)
    return outs, counters


def scatter_ranges(hist, ranges: CellRanges) -> list:
    """The one-rank state cut into the ranks' states (zero outside their cells)."""
    out = []
    for r in range(ranges.world):
        lo, hi = ranges.range(r)
        h = hist * 0
        h[lo:hi] = hist[lo:hi]
        out.append(h)
    return out


def gather_ranges(states, ranges: CellRanges):
    """The ranks' states joined into the one-rank state."""
    out = states[0] * 0
    for r, h in enumerate(states):
        lo, hi = ranges.range(r)
        out[lo:hi] = h[lo:hi]
    return out


def gpu_step_fn(wmc, p, V, ws, prec=0):
    """A step_fn running one step through libwmc on the current CUDA stream:
    the rank's particles numbered from id_base (wmc_set_id_base), then
    wmc_run of one step; returns (state after the step, counters of the step)."""
    import torch

    def step(hist, t, id_base):
        a = hist.clone()
        b = torch.empty_like(a)
        wmc.reset_counters(p, ws)
        wmc.set_id_base(p, ws, id_base)
        wmc.run(p, V, a, b, t, 1, ws, prec, False)
        c = wmc.get_counters(p, ws)
        return a, {k: c[k] for k in COUNTER_KEYS}

    return step
