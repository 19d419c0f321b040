"""Reduced precision at the full horizons of the synthetic cases: FP32 and
FP16-storage mole fractions against the FP64 GPU step after the stated number
of steps (max |dx| over every node and species), species mass against its
initial value.  The FP64 step matches the oracle to 1e-12 on every field at
every horizon the oracle can reach (the parity tests), and each case repeats
that check here at a short horizon on its own grid."""
import numpy as np
import pytest

from paper_2504_07059_gb300 import workloads as W
from parity_utils import TOL_MASS, TOL_X, compare_all_fp64, gpu_run, max_rel, oracle_run

pytestmark = pytest.mark.gpu


def _initial_mass(wl):
    return np.array([(wl.x[i] * wl.M[i] * (1.0 if wl.n is None else wl.n)).sum() for i in range(wl.ns)])


def _against_fp64(evd, wl, steps, precisions):
    ref = gpu_run(evd, wl, steps, "fp64")
    xr = ref.mole_fractions()
    ref.check()
    ref.close()
    m0 = _initial_mass(wl)
    out = {}
    for p in precisions:
        sim = gpu_run(evd, wl, steps, p)
        x = sim.mole_fractions()
        out[p] = (float(np.abs(x - xr).max()), max_rel(sim.species_mass(), m0))
        sim.check()
        sim.close()
    return out


def _oracle_check(evd, wl, steps):
    o = oracle_run(wl, steps)
    sim = gpu_run(evd, wl, steps, "fp64")
    compare_all_fp64(sim, o)
    sim.close()


def test_ternary_tube_with_gravity_at_50k_steps(evd):
    """The 64 x 1024 ternary Loschmidt tube with gravity (M = 2/28/44)."""
    wl = W.loschmidt_ternary_gravity()
    _oracle_check(evd, wl, 8)
    err = _against_fp64(evd, wl, 50000, ("fp32", "fp16"))
    for p, (dx, dm) in err.items():
        assert dx < TOL_X[p], (p, dx)
        assert dm < TOL_MASS[p], (p, dm)


def test_stratification_64_cube_at_20k_steps(evd):
    """A 64^3 copy of the closed D3Q19 box under gravity (M = 16/28/44)."""
    wl = W.stratification_3d(n=64)
    _oracle_check(evd, W.stratification_3d(n=16), 10)
    err = _against_fp64(evd, wl, 20000, ("fp32", "fp16"))
    for p, (dx, dm) in err.items():
        assert dx < TOL_X[p], (p, dx)
        assert dm < TOL_MASS[p], (p, dm)


def test_inverse_problem_tube_at_20k_steps(evd):
    """The 128 x 512 ternary tube with gravity of the inverse problem, FP32."""
    wl = W.loschmidt_ternary_gravity(nx=128, ny=512)
    _oracle_check(evd, wl, 5)
    err = _against_fp64(evd, wl, 20000, ("fp32",))
    dx, dm = err["fp32"]
    assert dx < TOL_X["fp32"], dx
    assert dm < TOL_MASS["fp32"], dm


def test_tube_sweep_members_at_10k_steps(evd):
    """The 512-tube sweep advanced 10k steps in FP32 by the batched step;
    sampled members (shortest, longest, the heaviest ternary and binary, two
    more) against the FP64 single-lattice step of the same tube."""
    tubes = W.batched_tubes()
    steps = 10000
    b = evd.Batch(tubes, "fp32")
    b.set_fields([t.x for t in tubes])
    b.step(steps)
    b.check()
    xs = b.mole_fractions()
    ms = b.species_mass()
    b.close()
    lengths = [t.shape[1] for t in tubes]
    tern = [i for i, t in enumerate(tubes) if t.ns == 3]
    binr = [i for i, t in enumerate(tubes) if t.ns == 2]
    picks = {int(np.argmin(lengths)), int(np.argmax(lengths)), max(tern, key=lambda i: tubes[i].M[-1]),
             max(binr, key=lambda i: tubes[i].M[-1]), 100, 333}
    for i in sorted(picks):
        ref = gpu_run(evd, tubes[i], steps, "fp64")
        xr = ref.mole_fractions()
        ref.close()
        assert np.abs(xs[i] - xr).max() < TOL_X["fp32"], i
        assert max_rel(ms[i], _initial_mass(tubes[i])) < TOL_MASS["fp32"], i
