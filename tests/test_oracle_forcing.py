"""Pins of the corrective forcing terms S_diff, S_p and S_rho of
Eq. (improved_forcing_scheme) in the oracle.  Each is w_a T(e):X with
T = (e e - c_s^2 I) contracted with a velocity, so by the lattice's isotropy
(sum w e e = c_s^2 I, fourth moment c_s^4 (dd + dd + dd)) it adds no mass and
no momentum, and its second moment is u X + X u (S_diff, S_p: tensor over
c_s^4 with the mixture u) or c_s^2 (u_i^eq Y + Y u_i^eq) (S_rho: over c_s^2
with u_i^eq).  Densities linear in x have an exact lattice gradient at nodes
whose neighbours are all fluid, which pins the gradients S_p and S_rho use."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2504_07059_gb300 import workloads as W


def second_moments(df, e):
    """Zeroth, first and second moments over directions of df [Q]."""
    return df.sum(), e.T @ df, np.einsum("a,ak,al->kl", df, e, e)


def moving_state(shape, M, slope, U, noise_stream=None):
    """D2Q9 populations f = w rho_i (1 + e.U/c_s^2) (times 1 + noise on
    the non-rest directions, when asked) with rho_i = 1 + slope_i x."""
    nx, ny = shape
    e, w, _ = O.lattice_info(W.D2Q9)
    c = np.sqrt(M[0] / np.asarray(M))
    xs = np.arange(nx, dtype=float)
    f = np.empty((len(M), 9, 1, ny, nx))
    for i in range(len(M)):
        rho = np.broadcast_to(1.0 + slope[i] * xs, (1, ny, nx))
        for a in range(9):
            f[i, a] = w[a] * rho * (1.0 + c[i] * (e[a] @ np.asarray(U)) / (c[i] ** 2 / 3.0))
    if noise_stream is not None:
        f *= 1.0 + 1e-3 * (2 * W.uniform01(noise_stream, f.size).reshape(f.shape) - 1)
    return f, e, c


def test_s_diff_adds_no_mass_or_momentum_and_the_symmetric_second_moment():
    M = (1.0, 3.0, 7.0)
    D = W.pair_diffusivities(3, 0.02, 0.1, 1200)
    f, e, c = moving_state((4, 4), M, (0.0, 0.0, 0.0), (0.02, -0.01, 0.0), noise_stream=1201)
    node = f[:, :, 0, 1, 2]
    plain = O.Oracle(W.D2Q9, (4, 4), 0, M, D, 1.0, (1e-4, 0.0))
    corr = O.Oracle(W.D2Q9, (4, 4), 0, M, D, 1.0, (1e-4, 0.0), flags=O.S_DIFF)
    fa, dga = plain.collide_node(node)
    fb, dgb = corr.collide_node(node)
    da, db = O.diag_arrays(dga, 3, 9), O.diag_arrays(dgb, 3, 9)
    u = db["u"]
    for i in range(3):
        dS = db["S"][i] - da["S"][i]
        m0, m1, m2 = second_moments(dS, c[i] * e)
        X = db["theta"][i] / (2 * db["tau"][i] - 1.0)
        expect = np.outer(u, X) + np.outer(X, u)
        assert np.abs(expect).max() > 1e-9          # not vacuous
        assert abs(m0) < 1e-17 and np.abs(m1).max() < 1e-17
        assert np.abs(m2 - expect).max() < 1e-12 * np.abs(expect).max()
        # the update adds (1 - 1/(2 tau_i)) of it (Eq. LBE_forcing)
        df = np.asarray(fb).reshape(3, 9)[i] - np.asarray(fa).reshape(3, 9)[i]
        assert np.abs(df - (1 - 1 / (2 * db["tau"][i])) * dS).max() < 1e-15


@pytest.mark.parametrize("flag", ["S_P", "S_RHO"])
def test_gradient_terms_on_densities_linear_in_x(flag):
    """Walls in x, densities linear in x, uniform velocity: one collision with
    the term minus one without is (1 - 1/(2 tau_i)) times a term with moments
    0, 0 and the tensor above, built from the exact slopes."""
    shape, M = (12, 4), (1.0, 2.0)
    slope = np.array([0.01, -0.02])
    D = np.array([[0, 0.05], [0.05, 0]])
    f, e, c = moving_state(shape, M, slope, (0.015, 0.01, 0.0))
    bit = getattr(O, flag)
    a = O.Oracle(W.D2Q9, shape, W.WALL_X, M, D, 1.0, (0.0, 0.0))
    b = O.Oracle(W.D2Q9, shape, W.WALL_X, M, D, 1.0, (0.0, 0.0), flags=bit)
    for o in (a, b):
        o.set_f(f)
        o.collide_only()
    fa, fb = a.get_f(), b.get_f()
    checked = 0
    for x in range(1, shape[0] - 1):       # every neighbour fluid along x
        node = f[:, :, 0, 2, x]
        _, dg = a.collide_node(node)
        d = O.diag_arrays(dg, 2, 9)
        rho = d["rho"]
        for i in range(2):
            df = fb[i, :, 0, 2, x] - fa[i, :, 0, 2, x]
            m0, m1, m2 = second_moments(df / (1 - 1 / (2 * d["tau"][i])), c[i] * e)
            cs2 = c[i] ** 2 / 3.0
            if flag == "S_P":   # enters with a minus sign, X = grad(rho_i c_s^2)
                X = -cs2 * np.array([slope[i], 0.0, 0.0])
                expect = np.outer(d["u"], X) + np.outer(X, d["u"])
            else:               # Y = w_i grad rho
                Y = rho[i] / rho.sum() * np.array([slope.sum(), 0.0, 0.0])
                expect = cs2 * (np.outer(d["ueq"][i], Y) + np.outer(Y, d["ueq"][i]))
            assert np.abs(expect).max() > 1e-7
            assert abs(m0) < 1e-16 and np.abs(m1).max() < 1e-16
            assert np.abs(m2 - expect).max() < 1e-10 * np.abs(expect).max()
            checked += 1
    assert checked == 2 * (shape[0] - 2)


def test_no_flags_is_the_standard_forcing_term_bit_for_bit():
    wl = W.random_mixture(W.D2Q9, (7, 6), W.WALL_Y, (1.0, 2.0, 5.0), g=(1e-5, -1e-5), stream=1220)
    runs = []
    for flags in (0, O.S_DIFF | O.S_P | O.S_RHO):
        o = O.Oracle(wl.lattice, wl.shape, wl.wall_mask, wl.M, wl.D, wl.tau1, wl.g, flags=flags)
        o.init(wl.x)
        o.step(5)
        runs.append(o.get_f())
    a = O.Oracle(wl.lattice, wl.shape, wl.wall_mask, wl.M, wl.D, wl.tau1, wl.g)
    a.init(wl.x)
    a.step(5)
    assert np.array_equal(a.get_f(), runs[0])
    assert not np.array_equal(runs[0], runs[1])
    # all three conserve each species' mass
    m0 = np.array([(wl.x[i] * wl.M[i]).sum() for i in range(3)])
    o = O.Oracle(wl.lattice, wl.shape, wl.wall_mask, wl.M, wl.D, wl.tau1, wl.g, flags=7)
    o.init(wl.x)
    o.step(50)
    assert np.abs(o.mass() / m0 - 1).max() < 50 * 4 * np.finfo(float).eps
