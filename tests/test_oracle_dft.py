"""Pins of the oracle's sliding-window evaluation of Eq. (wigner-1d-discrete)
(every cell, O(n_x n_M)): it equals the direct window sum per cell, which has
its own closed-form pins, to rounding for windows shorter and longer than the
momentum grid, both boundary modes, and grids whose length is not a multiple
of the period; and on the rectangular barrier it meets the closed form."""
import math

import numpy as np
import pytest

import oracle
import wmc_inputs as wi


def _p(n_x, Q, n_M, bc=0, dx=1e-9):
    return oracle.params(wi.Workload(name="t", n_x=n_x, dx_m=dx, Q=Q, n_M=n_M, dt_s=1e-16, steps=1,
                                     bc_potential=bc))


@pytest.mark.parametrize("n_x,Q,n_M,bc", [(37, 8, 8, 0), (64, 16, 48, 1), (200, 32, 20, 0), (90, 30, 64, 1),
                                          (150, 64, 128, 0)])
def test_dft_equals_direct_sum(n_x, Q, n_M, bc):
    p = _p(n_x, Q, n_M, bc)
    V = np.random.default_rng(n_x).uniform(-0.3, 0.4, n_x)
    a = oracle.kernel_all_dft(p, V)
    b = oracle.kernel_rows(p, V, np.arange(n_x))
    assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(b))


def test_dft_rectangular_barrier_closed_form():
    w = wi.BARRIER_100
    p = oracle.params(w)
    V = wi.potential(w)
    got = oracle.kernel_all_dft(p, V)
    a, b, h, V0 = 47, 52, w.Q // 2, float(np.float32(0.2))
    c = -2.0 / (6.582119569e-16 * w.Q)

    def dsum(lo, hi, phi):
        return 0.0 if lo > hi else (math.cos((lo - 0.5) * phi) - math.cos((hi + 0.5) * phi)) / (2 * math.sin(phi / 2))

    err = 0.0
    for i in range(w.n_x):
        for k in range(w.n_M):
            M = k - w.n_M // 2
            if M % w.Q == 0:
                continue
            phi = 2 * math.pi * M / w.Q
            ref = c * V0 * (dsum(max(a - i, 1), min(b - i, h - 1), phi) - dsum(max(i - b, 1), min(i - a, h - 1), phi))
            err = max(err, abs(got[i, k] - ref))
    assert err <= 1e-12 * np.abs(got).max()
