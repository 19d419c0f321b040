"""The TMA-staged D3Q19 step (the default for walled x/y boxes in FP32/FP16
storage) against the FP64 oracle and against the general kernel: ragged
tiles, several z-chunks, periodic z, one to three species, walls on every
face (edges and corners included)."""
import numpy as np
import pytest

from paper_2504_07059_gb300 import workloads as W
from parity_utils import TOL_MASS, TOL_X, max_rel, oracle_run

pytestmark = pytest.mark.gpu

WXY = W.WALL_X | W.WALL_Y
WALL3 = WXY | W.WALL_Z

CASES = {
    "box-32x8x8-ternary": (lambda: W.random_mixture(W.D3Q19, (32, 8, 8), WALL3, (16.0, 28.0, 44.0),
                                                      g=(1e-5, -2e-5, 1e-5), stream=500), 20),
    "ragged-40x7x11-ternary": (lambda: W.random_mixture(W.D3Q19, (40, 7, 11), WALL3, (16.0, 28.0, 44.0),
                                                          g=(0, -3e-5, 0), stream=510, n_amp=0.05), 20),
    "chunks-8x5x70-binary": (lambda: W.random_mixture(W.D3Q19, (8, 5, 70), WALL3, (1.0, 3.0),
                                                        g=(0, 0, -2e-5), stream=520), 15),
    "periodic-z-16x6x40": (lambda: W.random_mixture(W.D3Q19, (16, 6, 40), WXY, (16.0, 28.0, 44.0),
                                                      g=(1e-5, 0, 2e-5), stream=530), 15),
    "single-species-24x9x6": (lambda: W.random_mixture(W.D3Q19, (24, 9, 6), WALL3, (5.0,),
                                                         g=(0, -1e-4, 0), stream=540), 15),
    "stratification-32": (lambda: W.stratification_3d(shape=(32, 32, 32)), 10),
}


def _run(evd, wl, steps, precision, kernel, rows=4):
    sim = evd.Simulation(wl.lattice, wl.shape, wl.wall_mask, wl.M, wl.D, wl.tau1, wl.g, precision)
    evd.evd_set_kernel(sim.ctx, kernel)
    assert evd.evd_get_kernel(sim.ctx) == kernel
    if kernel == evd.EVD_KERNEL_TMA:
        evd.evd_set_tile_rows(sim.ctx, rows)
    sim.set_fields(wl.x, wl.n)
    sim.step(steps)
    return sim


@pytest.mark.parametrize("rows", [4, 2])
@pytest.mark.parametrize("precision", ["fp32", "fp16"])
@pytest.mark.parametrize("name", list(CASES))
def test_tma_step_matches_oracle(evd, name, precision, rows):
    make, steps = CASES[name]
    wl = make()
    if precision == "fp16" and wl.shape[0] % 8:
        pytest.skip("rows must be a multiple of 16 bytes for TMA")
    o = oracle_run(wl, steps)
    sim = _run(evd, wl, steps, precision, evd.EVD_KERNEL_TMA, rows)
    ob = o.observables()
    x = sim.mole_fractions()
    assert np.abs(x - ob["x"]).max() < TOL_X[precision], np.abs(x - ob["x"]).max()
    rho = sim.densities()
    assert max_rel(rho, ob["rho"]) < (1e-5 if precision == "fp32" else 2e-3)
    u, ui = sim.velocities()
    assert np.abs(u - ob["u"]).max() < (1e-6 if precision == "fp32" else 1e-4)
    m0 = np.array([(wl.x[i] * wl.M[i] * (1.0 if wl.n is None else wl.n)).sum() for i in range(wl.ns)])
    assert max_rel(sim.species_mass(), m0) < TOL_MASS[precision]
    sim.check()
    sim.close()


@pytest.mark.parametrize("name", ["ragged-40x7x11-ternary", "chunks-8x5x70-binary", "periodic-z-16x6x40"])
def test_tma_and_general_kernels_agree(evd, name):
    make, steps = CASES[name]
    wl = make()
    a = _run(evd, wl, steps, "fp32", evd.EVD_KERNEL_TMA)
    b = _run(evd, wl, steps, "fp32", evd.EVD_KERNEL_GENERAL)
    c = _run(evd, wl, steps, "fp32", evd.EVD_KERNEL_TMA, rows=2)
    fa, fb, fc = a.populations(), b.populations(), c.populations()
    assert max_rel(fa, fb) < 1e-5
    assert np.array_equal(fa, fc)          # tile shape does not change the arithmetic
    assert max_rel(a.species_mass(), b.species_mass()) < 1e-6


def test_tma_kernel_is_rejected_where_it_does_not_apply(evd):
    wl = W.random_mixture(W.D3Q19, (6, 6, 6), W.WALL_Y | W.WALL_Z, (1.0, 2.0), stream=550)   # periodic x
    sim = evd.Simulation(wl.lattice, wl.shape, wl.wall_mask, wl.M, wl.D, wl.tau1, wl.g, "fp32")
    assert evd.evd_get_kernel(sim.ctx) == evd.EVD_KERNEL_GENERAL
    with pytest.raises(evd.EVDError) as ei:
        evd.evd_set_kernel(sim.ctx, evd.EVD_KERNEL_TMA)
    assert ei.value.status == evd.EVD_ERR_ARG
    sim.close()
    wl = W.random_mixture(W.D3Q19, (8, 6, 6), WALL3, (1.0, 2.0), stream=560)
    sim = evd.Simulation(wl.lattice, wl.shape, wl.wall_mask, wl.M, wl.D, wl.tau1, wl.g, "fp32")
    assert evd.evd_get_kernel(sim.ctx) == evd.EVD_KERNEL_TMA     # the default where it applies
    sim.close()


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_tma_wait_timeout_reports_and_leaves_the_device_usable(evd, precision):
    """The failure path of the tile-copy waits: with a poll limit of zero every
    wait of the step gives up at once; the CTAs wait for their copies still
    in flight, the step reports EVD_ERR_TIMEOUT, the context is destroyed, and
    a fresh context on the same device still matches the oracle."""
    make, steps = CASES["box-32x8x8-ternary"]
    wl = make()
    sim = _run(evd, wl, 0, precision, evd.EVD_KERNEL_TMA, rows=2)
    evd.evd_set_wait_limit(sim.ctx, 0)
    evd.evd_step(sim.ctx, 1)
    with pytest.raises(evd.EVDError) as ei:
        evd.evd_check(sim.ctx)
    assert ei.value.status == evd.EVD_ERR_TIMEOUT
    assert "gave up" in evd.evd_last_error(sim.ctx)
    # the default limit back and fresh fields: the same context steps again
    evd.evd_set_wait_limit(sim.ctx, -1)
    sim.set_fields(wl.x, wl.n)
    sim.step(2)
    sim.check()
    sim.close()
    o = oracle_run(wl, steps)
    fresh = _run(evd, wl, steps, precision, evd.EVD_KERNEL_TMA, rows=2)
    x = fresh.mole_fractions()
    assert np.abs(x - o.observables()["x"]).max() < TOL_X[precision]
    fresh.check()
    fresh.close()
