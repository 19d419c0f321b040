"""Helpers shared by the GPU parity tests: run the oracle and the CUDA path on
the same seeded workload and compare element by element."""
from __future__ import annotations

import numpy as np

from oracle import oracle as O
from paper_2504_07059_gb300 import workloads as W

# Tolerances stated for the hot path: FP64 agrees with the oracle to 1e-12
# relative on all fields; FP32 and FP16-storage agree to 2e-5 and 1e-3 on mole
# fractions (absolute: mole fractions are O(1)); species mass to 1e-6 relative.
TOL_X = {"fp64": 1e-12, "fp32": 2e-5, "fp16": 1e-3}
TOL_MASS = {"fp64": 1e-12, "fp32": 1e-6, "fp16": 1e-6}


def oracle_run(wl: W.Workload, steps: int) -> O.Oracle:
    o = O.Oracle(wl.lattice, wl.shape, wl.wall_mask, wl.M, wl.D, wl.tau1, wl.g,
                 flags=getattr(wl, "flags", 0))
    if getattr(wl, "force", None) is not None:
        o.set_force_field(wl.force)
    o.init(wl.x, wl.n)
    o.step(steps)
    return o


def gpu_run(evd, wl: W.Workload, steps: int, precision: str = "fp64"):
    sim = evd.Simulation.from_workload(wl, precision)
    sim.step(steps)
    return sim


def max_rel(a, b) -> float:
    """max |a - b| / max |b| (max-norm relative error)."""
    scale = np.abs(b).max()
    return float(np.abs(a - b).max() / (scale if scale > 0 else 1.0))


def norm_rel(a, b, floor: float = 0.0) -> float:
    """||a - b||_2 / max(||b||_2, floor) (normwise relative error)."""
    nb = float(np.linalg.norm(b.ravel()))
    return float(np.linalg.norm((a - b).ravel()) / max(nb, floor, 1e-300))


def compare_all_fp64(sim, o, tol=1e-12):
    """Every readout field of the CUDA path against the oracle."""
    ob = o.observables()
    D = sim.D
    x = sim.mole_fractions()
    rho = sim.densities()
    u, ui = sim.velocities()
    f = sim.populations()
    fo = o.get_f()
    assert max_rel(x, ob["x"]) < tol, ("x", max_rel(x, ob["x"]))
    assert max_rel(rho, ob["rho"]) < tol, ("rho", max_rel(rho, ob["rho"]))
    assert max_rel(f, fo) < tol, ("populations", max_rel(f, fo))
    # velocities: absolute error against the larger of the oracle's largest
    # velocity and 1e-3 (a lattice-velocity scale; fields that vanish up to
    # roundoff would otherwise be compared noise against noise)
    for name, a, b in (("u", u, ob["u"][:D]), ("ui", ui, ob["ui"][:, :D])):
        err = float(np.abs(a - b).max()) / max(float(np.abs(b).max()), 1e-3)
        assert err < tol, (name, err)
    m = sim.species_mass()
    assert max_rel(m, o.mass()) < tol, ("mass", m, o.mass())


def window(wl: W.Workload, centre: tuple, k: int):
    """A sub-workload around ``centre`` (x, y, z) whose oracle run gives the
    exact state of the full run at ``centre`` after k steps: half-width k+1,
    walls kept where the window reaches a real wall (the far side then gets an
    artificial wall at distance >= k+1), periodic otherwise.  Returns the
    window workload and the centre's index inside it."""
    r = k + 1
    nn = wl.shape
    idx, shape, mask, local = [], [], 0, []
    for d in range(3):
        n, c = nn[d], centre[d]
        walled = (wl.wall_mask >> (2 * d)) & 3
        if n <= 2 * r + 1:
            ids = np.arange(n)
            if walled:
                mask |= 3 << (2 * d)
            local.append(c)
        elif walled and (c - r <= 0 or c + r >= n - 1):
            lo, hi = max(0, c - r), min(n - 1, c + r)
            ids = np.arange(lo, hi + 1)
            mask |= 3 << (2 * d)
            local.append(c - lo)
        else:
            ids = (np.arange(c - r, c + r + 1)) % n
            local.append(r)
        idx.append(ids)
        shape.append(len(ids))
    if wl.lattice == W.D2Q9:
        shape[2] = 1
    ix = np.ix_(range(wl.ns), idx[2], idx[1], idx[0])
    x = wl.x[ix]
    nf = None if wl.n is None else wl.n[np.ix_(idx[2], idx[1], idx[0])]
    sub = W.Workload(wl.name + "-window", wl.lattice, tuple(shape), mask, wl.M, wl.D, wl.tau1, wl.g,
                     k, np.ascontiguousarray(x), None if nf is None else np.ascontiguousarray(nf), wl.seed)
    return sub, tuple(local)
