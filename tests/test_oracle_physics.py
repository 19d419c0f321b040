"""Whole-step pins of the oracle against closed-form physics the paper fixes.

* Species mass is conserved with the impermeable-wall scheme (App. A; Sec. 4.1
  mass-history figure).  Bound: every population's weights sum to one up to a
  few roundings, so the relative drift after T steps is below T * 4 eps.
* Gravity-free binary interdiffusion in the closed tube follows the linearised
  (Fick) solution with the Maxwell-Stefan diffusivity D_12 (Sec. 4.1 uses it as
  the Ga = 0 reference): here the erf profile, since the diffusion length stays
  far from the ends.  This pins tau_12 (Eq. Luo&Girimaji_tau) through D_12.
* Under uniform gravity an ideal mixture settles, by Eq. (MS_equation) with all
  species velocities zero and mechanical equilibrium grad p = rho g, into
  independent barometric profiles rho_i ~ exp(g_y M_i y / (M_1 c_s1^2)), the
  law of the ultracentrifuge of Sec. 4.2 with a linear potential.
* In a fully periodic box the total momentum grows by exactly (sum rho) g per
  step: the self collision adds F/(2 tau), the forcing term (1 - 1/(2 tau)) F,
  the cross collision sums to zero over species and streaming conserves.
* A shear wave decays with the common kinematic viscosity
  nu = (tau_1 - 1/2) c_s1^2 that every species shares (Sec. 3).
* The initial state is at rest (Sec. 4.1, 4.2) and reads back the fields it
  was made from.
"""
import numpy as np
import pytest
from scipy.optimize import minimize_scalar
from scipy.special import erf

from oracle import oracle as O
from paper_2504_07059_gb300 import workloads as W

EPS = np.finfo(float).eps


@pytest.fixture(scope="module")
def loschmidt_binary_run():
    wl = W.loschmidt_binary()
    o = O.Oracle(wl.lattice, wl.shape, wl.wall_mask, wl.M, wl.D, wl.tau1, wl.g)
    o.init(wl.x)
    m0 = o.mass()
    o.step(wl.steps)
    return wl, o, m0


def test_species_mass_is_conserved_with_walls(loschmidt_binary_run):
    wl, o, m0 = loschmidt_binary_run
    drift = np.abs(o.mass() / m0 - 1.0)
    assert np.all(drift < wl.steps * 4 * EPS), drift
    # the initial masses are the integrals of rho_i = x_i M_i n
    assert np.allclose(m0, [(wl.x[i] * wl.M[i]).sum() for i in range(2)], rtol=1e-14)


def test_binary_interdiffusion_follows_erf(loschmidt_binary_run):
    wl, o, _ = loschmidt_binary_run
    x1 = o.observables()["x"][0, 0, :, :]
    assert np.ptp(x1, axis=1).max() < 1e-12          # uniform across the periodic width
    x1 = x1[:, 0]
    y = np.arange(wl.shape[1])
    D12, T, y0 = wl.D[0, 1], wl.steps, wl.shape[1] / 2 - 0.5
    profile = lambda D: 0.5 - 0.4 * erf((y - y0) / (2 * np.sqrt(D * T)))
    bulk = slice(8, wl.shape[1] - 8)                 # away from the wall boundary layer
    assert np.abs(x1[bulk] - profile(D12)[bulk]).max() < 1e-3
    fit = minimize_scalar(lambda D: np.sum((x1[16:-16] - profile(D)[16:-16]) ** 2),
                          bounds=(0.5 * D12, 2 * D12), method="bounded").x
    assert abs(fit / D12 - 1) < 1e-2, fit


@pytest.mark.parametrize("M,g,ny", [((1.0, 3.0), 5e-4, 24), ((1.0, 2.0, 4.0), 3e-4, 24)])
def test_gravity_gives_barometric_stratification(M, g, ny):
    ns = len(M)
    D = np.full((ns, ns), 0.1)
    o = O.Oracle(0, (2, ny), W.WALL_Y, M, D, 1.0, [0.0, -g, 0.0])
    x = np.full((ns, 1, ny, 2), 1.0 / ns)
    o.init(x)
    m0 = o.mass()
    o.step(20000)
    ob = o.observables()
    rho = ob["rho"][:, 0, :, 0]
    yy = np.arange(ny)
    inner = slice(4, ny - 4)
    for i in range(ns):
        slope = np.polyfit(yy[inner], np.log(rho[i][inner]), 1)[0]
        expect = -g * M[i] / (M[0] / 3.0)
        assert abs(slope / expect - 1) < 1e-3, (i, slope, expect)
    # heaviest species sinks, lightest rises in mole fraction
    xs = ob["x"][:, 0, :, 0]
    assert xs[0, -1] > xs[0, 0] and xs[-1, 0] > xs[-1, -1]
    # steady: the real species velocities of Eq. (CE_EQ83) vanish in the bulk
    # (the wall boundary layer of the interpolated species decays geometrically)
    assert np.abs(ob["ui"][:, :, 0, 8:ny - 8, :]).max() < 1e-6
    assert np.allclose(o.mass(), m0, rtol=20000 * 4 * EPS)


@pytest.mark.parametrize("lattice,shape,M,g", [
    (0, (6, 5), (2.0, 28.0, 44.0), (1e-5, -2e-5, 0.0)),
    (1, (4, 3, 5), (16.0, 28.0, 44.0), (1e-5, 2e-5, -3e-5)),
    (0, (3, 4), (1.0, 1.0), (0.0, 4e-5, 0.0))])
def test_periodic_box_momentum_grows_by_the_total_force(lattice, shape, M, g):
    wl = W.random_mixture(lattice, shape, 0, M, g=g)
    o = O.Oracle(lattice, shape, 0, M, wl.D, 1.0, wl.g)
    o.init(wl.x)
    e = O.lattice_info(lattice)[0].astype(float)
    c = o.species_info()[0]

    def momentum():
        f = o.get_f().reshape(o.ns, o.Q, -1).sum(axis=2)
        return sum((c[i] * e).T @ f[i] for i in range(o.ns))

    p0, mass = momentum(), o.mass().sum()
    o.step(40)
    p1 = momentum()
    np.testing.assert_allclose(p1 - p0, 40 * mass * np.array(wl.g), rtol=1e-10, atol=1e-15)


@pytest.mark.parametrize("M,tau1,tol", [((1.0, 2.0), 1.0, 1e-2), ((2.0, 28.0, 44.0), 0.8, 5e-2)])
def test_shear_wave_decays_with_the_common_viscosity(M, tau1, tol):
    ns, nx, ny = len(M), 2, 32
    o = O.Oracle(0, (nx, ny), 0, M, np.full((ns, ns), 0.05), tau1, [0, 0, 0])
    e, w, _ = O.lattice_info(0)
    c, cs2, _ = o.species_info()
    k, U = 2 * np.pi / ny, 1e-3
    y = np.arange(ny)
    f = np.zeros((ns, 9, 1, ny, nx))
    for i in range(ns):
        for yy in range(ny):
            u = np.array([U * np.sin(k * yy), 0.0, 0.0])
            eu = (c[i] * e) @ u
            feq = w * (0.3 + 0.2 * i) * (1 + eu / cs2[i] + eu**2 / (2 * cs2[i] ** 2) - u @ u / (2 * cs2[i]))
            f[i, :, 0, yy, :] = feq[:, None]
    o.set_f(f)
    amps, times = [], [200, 400, 800]
    t = 0
    for tt in times:
        o.step(tt - t)
        t = tt
        ux = o.observables()["u"][0, 0, :, 0]
        amps.append(2 / ny * np.sum(ux * np.sin(k * y)))
    rate = -np.polyfit(times, np.log(amps), 1)[0]
    nu = (tau1 - 0.5) / 3.0
    assert abs(rate / (nu * k * k) - 1) < tol, rate / (nu * k * k)


# ---------------------------------------------------------------- force field
def test_force_field_of_zeros_and_uniform_field_reduce_to_plain_gravity():
    wl = W.random_mixture(W.D2Q9, (6, 9), W.WALL_Y, (1.0, 2.0, 5.0), g=(1e-5, -2e-5), stream=700)
    a = O.Oracle(wl.lattice, wl.shape, wl.wall_mask, wl.M, wl.D, wl.tau1, wl.g)
    a.init(wl.x)
    a.step(20)
    b = O.Oracle(wl.lattice, wl.shape, wl.wall_mask, wl.M, wl.D, wl.tau1, wl.g)
    b.set_force_field(np.zeros((3,) + wl.x.shape[1:]))
    b.init(wl.x)
    b.step(20)
    assert np.array_equal(a.get_f(), b.get_f())
    # g = 0 plus a uniform field equal to g: F_i = rho_i (0 + g), the same numbers
    c = O.Oracle(wl.lattice, wl.shape, wl.wall_mask, wl.M, wl.D, wl.tau1, (0.0, 0.0, 0.0))
    k = np.zeros((3,) + wl.x.shape[1:])
    k[0], k[1] = wl.g[0], wl.g[1]
    c.set_force_field(k)
    c.init(wl.x)
    c.step(20)
    assert np.array_equal(a.get_f(), c.get_f())


def _ultracentrifuge_C(x1, r, r_ref):
    """Least-squares C of ln[x1(r)(1 - x1(r_ref)) / (x1(r_ref)(1 - x1(r)))]
    = C (r^2 - r_ref^2) / 2, the separation law of Case II."""
    i0 = list(r).index(r_ref)
    lhs = np.log(x1 * (1.0 - x1[i0]) / (x1[i0] * (1.0 - x1)))
    q = (r.astype(float) ** 2 - float(r_ref) ** 2) / 2.0
    return float((q * lhs).sum() / (q * q).sum())


def test_ultracentrifuge_steady_profile_follows_the_closed_form():
    """Sec. 4.2 Case II: at steady state the separation factor obeys
    1/alpha = exp(C r^2 / 2) with C = (M1 - M2) omega^2 / (M1 c_s1^2).  A small
    cavity (R = 48) with a stronger mass contrast (M = 1, 2) and a larger
    diffusivity reaches steady state quickly (18000 steps, about 15 diffusion
    times); the fitted C over the bulk rows (away from the wall boundary layer)
    must match to 1e-4 (observed 3e-6)."""
    R, H, omega2 = 48, 3, 2e-6
    wl = W.ultracentrifuge(R=R, H=H, xbar=0.4, tau1=1.0, D12=0.2)
    wl = W.Workload(wl.name, wl.lattice, wl.shape, wl.wall_mask, (1.0, 2.0), wl.D, wl.tau1, wl.g, 0,
                    wl.x, np.full(wl.n.shape, 1.0 / (0.4 * 1.0 + 0.6 * 2.0)),
                    force=np.zeros_like(wl.force))
    wl.force[1] = (omega2 * np.arange(R))[None, :, None]
    C = (1.0 - 2.0) * omega2 / (1.0 / 3.0)
    o = O.Oracle(wl.lattice, wl.shape, wl.wall_mask, wl.M, wl.D, wl.tau1, wl.g)
    o.set_force_field(wl.force)
    o.init(wl.x, wl.n)
    o.step(18000)
    x1 = o.observables()["x"][0, 0].mean(axis=1)   # average over the periodic width
    r = np.arange(R)
    bulk = slice(8, R - 8)
    Cfit = _ultracentrifuge_C(x1[bulk], r[bulk], 8)
    assert abs(Cfit / C - 1.0) < 1e-4, (Cfit, C)
    # and the species mass stays exact up to rounding (T steps x 4 eps)
    m0 = np.array([(wl.x[i] * wl.M[i] * wl.n).sum() for i in range(2)])
    assert np.abs(o.mass() / m0 - 1.0).max() < 18000 * 4 * np.finfo(float).eps


@pytest.mark.parametrize("lattice,shape,mask,M,g", [
    (W.D2Q9, (5, 7), W.WALL_Y, (1.0, 3.0, 7.0), (2e-5, -3e-5)),
    (W.D3Q19, (3, 4, 5), W.WALL_X | W.WALL_Y | W.WALL_Z, (16.0, 28.0, 44.0), (1e-5, -2e-5, 3e-5))])
def test_initial_state_is_at_rest_and_reads_back_its_fields(lattice, shape, mask, M, g):
    """Sec. 4.1 and 4.2 start every species at rest: with the forced
    u_i^eq = j_i/rho_i + g/2 (Eq. first_order_moment_force) the initial
    populations carry u_i0 = -g/2, so the read-out species and mixture
    velocities are zero; rho_i = x_i M_i n, and the readout x_i = rho_i/(n M_i)
    returns the mole fractions it started from."""
    wl = W.random_mixture(lattice, shape, mask, M, g=g, stream=1450, n_amp=0.1)
    o = O.Oracle(lattice, shape, mask, M, wl.D, 1.0, g)
    o.init(wl.x, wl.n)
    obs = o.observables()
    # rounding of the first moments of O(0.1) populations: ~1e-17, against
    # |g| ~ 3e-5 for a sign slip
    assert np.abs(obs["u"]).max() < 1e-15
    assert np.abs(obs["ui"]).max() < 1e-15
    n = wl.n.reshape(obs["x"].shape[1:])
    # a handful of roundings (sums of Q populations, n, one division):
    # observed 6.7e-16
    for i, Mi in enumerate(M):
        assert np.allclose(obs["rho"][i], wl.x[i] * Mi * n, rtol=4e-15, atol=0)
    assert np.allclose(obs["x"], wl.x, rtol=4e-15, atol=0)
