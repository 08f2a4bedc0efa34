"""Seeded synthetic inputs for the signed-particle Wigner Monte Carlo workloads.

This module serves both the CUDA path and the CPU oracle, and holds none of the
method's arithmetic: it builds potentials (barriers, noise, tanh-edged
barriers) and the initial signed histogram sampled from the Gaussian initial
Wigner function of Sec. 3 (every particle positive).  Everything is drawn from
numpy's PCG64 with a stated seed.

Units: lengths in metres, energies in eV, times in seconds, potentials as FP32
arrays in eV (the type the CUDA path takes; the oracle widens them exactly).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

M_E = 9.1093837015e-31          # electron mass [kg] (CODATA 2018)
HBAR_JS = 1.054571817e-34       # [J s]
EV_J = 1.602176634e-19          # [J / eV]
NM = 1e-9
FS = 1e-15


@dataclasses.dataclass(frozen=True)
class Barrier:
    height_ev: float
    width_m: float
    centre_m: float


@dataclasses.dataclass(frozen=True)
class Packet:
    x0_m: float
    sigma_m: float
    energy_ev: float
    n0: int


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    n_x: int
    dx_m: float
    Q: int                   # quadrature points L_C / dx
    n_M: int                 # momentum indices, M in [-n_M/2, n_M/2)
    dt_s: float
    steps: int
    barriers: tuple = ()
    packet: Packet | None = None
    noise_ev: float = 0.0    # uniform per-cell perturbation half-width
    noise_seed: int = 1
    seed: int = 0            # Philox key of the run and PCG64 seed of the initial sample
    mass_kg: float = M_E
    bc_potential: int = 0    # 0: V = 0 outside the domain; 1: edge value
    child_wrap: int = 0      # 0: drop children outside the momentum grid; 1: wrap
    sim: int = 0

    @property
    def length_m(self) -> float:
        return self.n_x * self.dx_m

    @property
    def L_C(self) -> float:
        return self.Q * self.dx_m

    def replace(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)


def _barrier_cells(n_x: int, dx: float, b: Barrier) -> np.ndarray:
    """Cells whose centre (i + 1/2) dx lies in [c - w/2, c + w/2)."""
    centres = (np.arange(n_x) + 0.5)
    lo = (b.centre_m - b.width_m / 2) / dx
    hi = (b.centre_m + b.width_m / 2) / dx
    # tolerance against representation error of the edges, far below half a cell
    return (centres >= lo - 1e-9) & (centres < hi - 1e-9)


def potential(w: Workload) -> np.ndarray:
    """Potential [n_x] in eV, FP32."""
    V = np.zeros(w.n_x, dtype=np.float64)
    for b in w.barriers:
        V[_barrier_cells(w.n_x, w.dx_m, b)] += b.height_ev
    if w.noise_ev:
        rng = np.random.Generator(np.random.PCG64(w.noise_seed))
        V += rng.uniform(-w.noise_ev, w.noise_ev, size=w.n_x)
    return V.astype(np.float32)


def initial_histogram(w: Workload, rng_seed: int | None = None) -> np.ndarray:
    """Signed counts [n_x, n_M] (int32) of n0 positive particles drawn from
    f0(x, M) ~ exp(-(x - x0)^2 / sigma^2) exp(-(M dk - k0)^2 sigma^2), Sec. 3,
    with dk = pi / L_C and k0 = sqrt(2 m E) / hbar; positions outside [0, L)
    are redrawn."""
    pk = w.packet
    rng = np.random.Generator(np.random.PCG64(w.seed if rng_seed is None else rng_seed))
    L = w.length_m
    xs = np.empty(0)
    need = pk.n0
    parts = []
    while need > 0:
        x = rng.normal(pk.x0_m, pk.sigma_m / math.sqrt(2.0), size=int(need * 1.05) + 16)
        x = x[(x >= 0) & (x < L)][:need]
        parts.append(x)
        need -= x.size
    xs = np.concatenate(parts) if parts else xs
    cells = np.minimum((xs / w.dx_m).astype(np.int64), w.n_x - 1)
    dk = math.pi / w.L_C
    k0 = math.sqrt(2.0 * w.mass_kg * pk.energy_ev * EV_J) / HBAR_JS
    Ms = np.arange(w.n_M) - w.n_M // 2
    wts = np.exp(-((Ms * dk - k0) ** 2) * pk.sigma_m ** 2)
    wts /= wts.sum()
    ks = rng.choice(w.n_M, size=pk.n0, p=wts)
    hist = np.bincount(cells * w.n_M + ks, minlength=w.n_x * w.n_M)
    return hist.reshape(w.n_x, w.n_M).astype(np.int32)


def random_histogram(w: Workload, n_particles: int, seed: int, signed: bool = True,
                     cells: tuple[int, int] | None = None) -> np.ndarray:
    """Arbitrary signed histogram for edge-case tests: n_particles placed
    uniformly over a cell range and all momenta, random signs."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lo, hi = cells if cells else (0, w.n_x)
    c = rng.integers(lo, hi, size=n_particles)
    k = rng.integers(0, w.n_M, size=n_particles)
    s = rng.choice([-1, 1], size=n_particles) if signed else np.ones(n_particles, np.int64)
    hist = np.zeros(w.n_x * w.n_M, np.int64)
    np.add.at(hist, c * w.n_M + k, s)
    return hist.reshape(w.n_x, w.n_M).astype(np.int32)


# --------------------------------------------------------------------------
# The workloads.  Unstated parameters take the proposed values listed in the
# design notes (c3 dt and packet centre, the double-barrier gap reading).
# --------------------------------------------------------------------------

BARRIER_100 = Workload(
    name="barrier-100", n_x=100, dx_m=1 * NM, Q=32, n_M=64, dt_s=0.1 * FS, steps=100,
    barriers=(Barrier(0.2, 6 * NM, 50 * NM),),
    packet=Packet(25 * NM, 5 * NM, 0.1, 100_000), seed=0)

BARRIER_2000 = Workload(
    name="barrier-2000", n_x=2000, dx_m=0.5 * NM, Q=128, n_M=256, dt_s=0.05 * FS, steps=1000,
    barriers=(Barrier(0.3, 10 * NM, 500 * NM),),
    packet=Packet(250 * NM, 20 * NM, 0.15, 10_000_000), seed=0)

_L3 = 16384 * 0.1 * NM
DOUBLE_BARRIER_16384 = Workload(
    name="double-barrier-16384", n_x=16384, dx_m=0.1 * NM, Q=1024, n_M=1024, dt_s=0.05 * FS, steps=200,
    barriers=(Barrier(0.25, 2 * NM, _L3 / 2 - 3.5 * NM), Barrier(0.25, 2 * NM, _L3 / 2 + 3.5 * NM)),
    packet=Packet(_L3 / 4, 50 * NM, 0.1, 100_000_000), noise_ev=5e-3, noise_seed=1, seed=0)

WORKLOADS = {w.name: w for w in (BARRIER_100, BARRIER_2000, DOUBLE_BARRIER_16384)}


def scaled(w: Workload, n0: int) -> Workload:
    """The same workload with a different initial particle count."""
    return w.replace(packet=dataclasses.replace(w.packet, n0=n0))


def batch_workloads(n_sims: int, seed: int = 2, n_x_range=(200, 4000), n0_range=(10_000, 1_000_000),
                    dt_s: float = 0.05 * FS, steps: int = 500) -> list:
    """The batched workload: n_sims independent barrier simulations with
    per-simulation draws (PCG64 seed `seed`): cells U[n_x_range] at 0.5 nm,
    n_M in {128, 256} with Q = n_M / 2, barrier height U[0.05, 0.5] eV and
    width U[2, 20] nm at the domain midpoint, packet energy U[0.05, 0.3] eV at
    L/4 with sigma = L/20, particle count U[n0_range]; Philox seed 1000 + s and
    sim index s."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    dx = 0.5 * NM
    for s in range(n_sims):
        n_x = int(rng.integers(n_x_range[0], n_x_range[1] + 1))
        n_M = int(rng.choice([128, 256]))
        V0 = float(rng.uniform(0.05, 0.5))
        width = float(rng.uniform(2, 20)) * NM
        E = float(rng.uniform(0.05, 0.3))
        n0 = int(rng.integers(n0_range[0], n0_range[1] + 1))
        L = n_x * dx
        out.append(Workload(
            name=f"batch-{s}", n_x=n_x, dx_m=dx, Q=n_M // 2, n_M=n_M, dt_s=dt_s, steps=steps,
            barriers=(Barrier(V0, width, L / 2),), packet=Packet(L / 4, L / 20, E, n0), seed=1000 + s, sim=s))
    return out


TANH_BARRIERS_4096 = Workload(
    name="tanh-barriers-4096", n_x=4096, dx_m=0.25 * NM, Q=256, n_M=512, dt_s=0.05 * FS, steps=1, seed=3)


def tanh_parameters(n_pot: int, n_x: int = 4096, dx_nm: float = 0.25, n_barriers: int = 16, n_segments: int = 16,
                    seed: int = 3) -> np.ndarray:
    """Parameters [n_pot, 3 nb + ns] (FP32) of the smooth multi-barrier
    potential: heights U[0.05, 0.3] eV, widths U[1, 5] nm, centres one per
    1/nb of the domain with a uniform jitter of a quarter of that length,
    segment offsets U[-0.02, 0.02] eV (PCG64 seed `seed`)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    L = n_x * dx_nm
    slot = L / n_barriers
    th = np.zeros((n_pot, 3 * n_barriers + n_segments))
    for b in range(n_pot):
        th[b, :n_barriers] = rng.uniform(0.05, 0.3, n_barriers)
        th[b, n_barriers:2 * n_barriers] = rng.uniform(1.0, 5.0, n_barriers)
        th[b, 2 * n_barriers:3 * n_barriers] = (np.arange(n_barriers) + 0.5) * slot + rng.uniform(
            -slot / 4, slot / 4, n_barriers)
        th[b, 3 * n_barriers:] = rng.uniform(-0.02, 0.02, n_segments)
    return th.astype(np.float32)


# The trained N = 2 network's data set (Sec. 2.3): Gaussian-bump potentials on
# 256 cells of 0.5 nm, window L_C = 32 nm (Q = 64 = n_M), kernels of one period.
N2_TRAIN = Workload(
    name="n2-train-256", n_x=256, dx_m=0.5 * NM, Q=64, n_M=64, dt_s=0.05 * FS, steps=1, seed=4)


def gaussian_bumps(n_examples: int, n_x: int = 256, dx_nm: float = 0.5, seed: int = 4) -> np.ndarray:
    """Potentials [n_examples, n_x] (FP32, eV) of single Gaussian bumps
    V0 exp(-(x - c)^2 / s^2) at the cell centres: height V0 U[0.05, 0.3] eV,
    centre c U[0.25 L, 0.75 L], dispersion s U[1, 5] nm (PCG64 seed `seed`)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    L = n_x * dx_nm
    x = (np.arange(n_x) + 0.5) * dx_nm
    out = np.empty((n_examples, n_x), np.float32)
    for e in range(n_examples):
        V0 = rng.uniform(0.05, 0.3)
        c = rng.uniform(0.25 * L, 0.75 * L)
        s = rng.uniform(1.0, 5.0)
        out[e] = (V0 * np.exp(-((x - c) / s) ** 2)).astype(np.float32)
    return out


def sgd_order(epochs: int, n_examples: int, seed: int = 5) -> np.ndarray:
    """The examples of each epoch in a fresh random order: int32 [epochs, n_examples]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.stack([rng.permutation(n_examples) for _ in range(epochs)]).astype(np.int32)
