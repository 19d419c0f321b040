"""The corrective forcing terms of Eq. (improved_forcing_scheme) on the GPU
(D2Q9): parity with the oracle carrying the same flags, every field in FP64,
mole fractions and mass in FP32."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2504_07059_gb300 import workloads as W
from parity_utils import TOL_MASS, TOL_X, compare_all_fp64, gpu_run, max_rel, oracle_run

pytestmark = pytest.mark.gpu

ALL = O.S_DIFF | O.S_P | O.S_RHO


def case(flags, walls, stream):
    """A moving ternary mixture: gravity of 1e-4 drives velocities for the
    terms to act on."""
    wl = W.random_mixture(W.D2Q9, (19, 14), walls, (1.0, 3.0, 7.0), g=(6e-5, -1e-4), stream=stream, n_amp=0.1)
    wl.flags = flags
    return wl


@pytest.mark.parametrize("flags", [O.S_DIFF, O.S_P, O.S_RHO, ALL])
@pytest.mark.parametrize("walls", [W.WALL_X | W.WALL_Y, 0])
def test_fp64_corrective_terms_match_the_oracle(evd, flags, walls):
    wl = case(flags, walls, 1300)
    steps = 30
    o = oracle_run(wl, steps)
    sim = gpu_run(evd, wl, steps, "fp64")
    compare_all_fp64(sim, o)
    # the terms change the state beyond the tolerance (the check is not vacuous)
    plain = case(0, walls, 1300)
    x0 = oracle_run(plain, steps).observables()["x"]
    assert np.abs(sim.mole_fractions() - x0).max() > 1e-10
    sim.close()


def test_fp32_with_every_corrective_term(evd):
    wl = case(ALL, W.WALL_Y, 1310)
    steps = 100
    o = oracle_run(wl, steps)
    sim = gpu_run(evd, wl, steps, "fp32")
    assert np.abs(sim.mole_fractions() - o.observables()["x"]).max() < TOL_X["fp32"]
    m0 = np.array([(wl.x[i] * wl.M[i] * wl.n).sum() for i in range(3)])
    assert max_rel(sim.species_mass(), m0) < TOL_MASS["fp32"]
    sim.close()


def test_gradient_terms_add_one_density_pass_per_step(evd):
    wl = case(O.S_P, W.WALL_Y, 1320)
    sim = evd.Simulation.from_workload(wl, "fp64")
    n0 = evd.evd_launch_count(sim.ctx)
    sim.step(10)
    assert evd.evd_launch_count(sim.ctx) - n0 == 20
    sim.close()
    wl = case(O.S_DIFF, W.WALL_Y, 1320)
    sim = evd.Simulation.from_workload(wl, "fp64")
    n0 = evd.evd_launch_count(sim.ctx)
    sim.step(10)
    assert evd.evd_launch_count(sim.ctx) - n0 == 10
    sim.close()
