"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle on the
same seeded inputs: FP64 to 1e-12 relative on every field, FP32 and
FP16-storage to 2e-5 and 1e-3 on mole fractions, species mass to 1e-6."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2504_07059_gb300 import workloads as W
from parity_utils import (TOL_MASS, TOL_X, compare_all_fp64, gpu_run, max_rel, oracle_run,
                          window)

pytestmark = pytest.mark.gpu

WY = W.WALL_Y
WXY = W.WALL_X | W.WALL_Y
WALL3 = W.WALL_X | W.WALL_Y | W.WALL_Z

SMALL_CASES = {
    # name: (workload, steps)
    "d2q9-binary-tube-4x256": (lambda: W.loschmidt_binary(), 2000),
    "d2q9-ternary-ragged-walls-y": (lambda: W.random_mixture(W.D2Q9, (37, 29), WY, (2.0, 28.0, 44.0),
                                                               g=(1e-5, -3e-5), n_amp=0.1), 60),
    "d2q9-ternary-box-corners": (lambda: W.random_mixture(W.D2Q9, (19, 23), WXY, (1.0, 3.0, 7.0),
                                                            g=(2e-5, -1e-5), stream=20), 60),
    "d2q9-binary-periodic": (lambda: W.random_mixture(W.D2Q9, (17, 13), 0, (1.0, 2.5),
                                                        g=(2e-5, 1e-5), stream=30), 60),
    "d2q9-single-species": (lambda: W.random_mixture(W.D2Q9, (9, 12), WY, (3.0,), g=(0, -1e-4), stream=40), 60),
    "d2q9-equal-masses": (lambda: W.random_mixture(W.D2Q9, (8, 10), WXY, (4.0, 4.0, 4.0), stream=50), 60),
    "d2q9-one-wide-channel": (lambda: W.random_mixture(W.D2Q9, (1, 16), WXY, (1.0, 2.0), g=(0, -1e-4), stream=60), 60),
    "d2q9-one-row-periodic": (lambda: W.random_mixture(W.D2Q9, (24, 1), 0, (1.0, 5.0), g=(1e-5, 0), stream=70), 60),
    "d3q19-ternary-closed-box": (lambda: W.random_mixture(W.D3Q19, (11, 9, 7), WALL3, (16.0, 28.0, 44.0),
                                                            g=(1e-5, -2e-5, 3e-5), stream=80), 25),
    "d3q19-binary-channel": (lambda: W.random_mixture(W.D3Q19, (13, 6, 5), W.WALL_Y | W.WALL_Z, (1.0, 3.0),
                                                        g=(3e-5, 0, 0), stream=90), 25),
    "d3q19-flat-periodic": (lambda: W.random_mixture(W.D3Q19, (7, 5, 1), 0, (2.0, 3.0, 5.0), stream=100), 25),
    "d3q19-stratification-32": (lambda: W.stratification_3d(shape=(32, 32, 32)), 6),
}


@pytest.mark.parametrize("name", list(SMALL_CASES))
def test_fp64_matches_oracle_on_every_field(evd, name):
    make, steps = SMALL_CASES[name]
    wl = make()
    o = oracle_run(wl, steps)
    sim = gpu_run(evd, wl, steps, "fp64")
    assert sim.t == steps
    compare_all_fp64(sim, o)
    sim.close()


def test_fp64_time_zero_readout_is_the_initial_state(evd):
    wl = W.random_mixture(W.D2Q9, (6, 7), WY, (1.0, 2.0, 3.0), g=(0, -1e-4), n_amp=0.2)
    o = oracle_run(wl, 0)
    sim = gpu_run(evd, wl, 0, "fp64")
    compare_all_fp64(sim, o)
    # after one step as well (the first gather of the post-collision state)
    o.step(1)
    sim.step(1)
    compare_all_fp64(sim, o)


REDUCED = [(n, p) for n in ["d2q9-binary-tube-4x256", "d2q9-ternary-ragged-walls-y",
                             "d2q9-ternary-box-corners", "d3q19-ternary-closed-box",
                             "d3q19-stratification-32"] for p in ("fp32", "fp16")]


@pytest.mark.parametrize("name,precision", REDUCED)
def test_reduced_precision_mole_fractions_and_mass(evd, name, precision):
    make, steps = SMALL_CASES[name]
    wl = make()
    o = oracle_run(wl, steps)
    sim = gpu_run(evd, wl, steps, precision)
    x = sim.mole_fractions()
    err = np.abs(x - o.observables()["x"]).max()
    assert err < TOL_X[precision], err
    m0 = np.array([(wl.x[i] * wl.M[i] * (1.0 if wl.n is None else wl.n)).sum() for i in range(wl.ns)])
    assert max_rel(sim.species_mass(), m0) < TOL_MASS[precision]
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
def test_loschmidt_ternary_gravity_full_grid(evd, precision):
    """The 64x1024 ternary tube with gravity at full size, a few steps, every node."""
    wl = W.loschmidt_ternary_gravity()
    steps = 5
    o = oracle_run(wl, steps)
    sim = gpu_run(evd, wl, steps, precision)
    x = sim.mole_fractions()
    xo = o.observables()["x"]
    if precision == "fp64":
        compare_all_fp64(sim, o)
    else:
        assert np.abs(x - xo).max() < TOL_X[precision]
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
def test_stratification_256_sampled_windows(evd, precision):
    """The 256^3 closed box in the launch configuration the benchmark times:
    after k steps, sampled nodes (corners, edges, faces, interior) against the
    oracle run on a window that determines them exactly."""
    wl = W.stratification_3d(n=256)
    k = 3
    sim = gpu_run(evd, wl, k, precision)
    x = sim.mole_fractions()
    rho = sim.densities()
    n = 256
    samples = [(0, 0, 0), (255, 255, 255), (0, 255, 17), (128, 0, 200), (255, 77, 0),
               (1, 1, 1), (100, 150, 3), (37, 254, 128), (128, 128, 128), (200, 60, 90)]
    for c in samples:
        sub, loc = window(wl, c, k)
        o = oracle_run(sub, k)
        ob = o.observables()
        xo = ob["x"][:, loc[2], loc[1], loc[0]]
        ro = ob["rho"][:, loc[2], loc[1], loc[0]]
        xg = x[:, c[2], c[1], c[0]]
        rg = rho[:, c[2], c[1], c[0]]
        tol = 1e-12 if precision == "fp64" else TOL_X[precision]
        assert np.abs(xg - xo).max() < tol, (c, xg, xo)
        assert max_rel(rg, ro) < {"fp64": 1e-12, "fp32": 1e-5, "fp16": 2e-3}[precision], (c, rg, ro)
    m0 = np.array([(wl.x[i] * wl.M[i]).sum() for i in range(3)])
    assert max_rel(sim.species_mass(), m0) < TOL_MASS[precision]
    sim.close()
