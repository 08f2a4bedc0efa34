"""The Simulation wrapper (device buffers + wmc_run) against the CPU oracle:
the 2000-cell barrier, whose packet starts farther than L_C / 2 from the
barrier, so that its first steps see a zero kernel in both precisions and
the histograms agree bit for bit; steps split over calls resume the Philox
streams and the step counter."""
import numpy as np
import pytest

import oracle
import wmc_inputs as wi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_simulation_matches_oracle_and_resumes():
    from paper_1806_00082_gb300 import build, wmc
    from paper_1806_00082_gb300.sim import Simulation
    build.build()
    wmc.load()
    wl = wi.BARRIER_2000
    V = wi.potential(wl)
    h0 = wi.initial_histogram(wl)
    ref, st = oracle.simulate(oracle.params(wl), h0, 1, 3, V=V)
    sim = Simulation(wmc.Params.of(wl), V, h0)
    sim.run(1)
    sim.run(2)
    assert sim.t == 4
    np.testing.assert_array_equal(sim.hist.cpu().numpy(), ref)
    rho = sim.density().cpu().numpy()
    np.testing.assert_array_equal(rho, ref.sum(axis=1))
    assert sim.counters()["particle_steps"] == st[oracle.ST_PARTICLE_STEPS]
