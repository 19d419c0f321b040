"""Pins of the oracle's collision (Sec. 2-3) by the moment identities the
paper states or that follow from its definitions, on random node states.

Each identity constrains a different term, so a dropped term, a flipped sign or
a swapped species index in the oracle fails at least one of them:
  * Sum f^(0) = rho_i, Sum e f^(0) = rho_i u_i^eq  (Eq. feqi0 built to this end)
  * Sum S = 0, Sum e S = F_i                       (Eq. CE_EQ52, CE_EQ54)
  * Sum e e S = u F + F u                          (the second-order part of S)
  * Sum Omega^ij = 0, Sum e Omega^ij = -rho_i rho_j/(rho tau_ij)(u_i^eq - u_j^eq)
    (from Eq. Cross_collision_Sirovich and the equilibrium moments), whose sum
    over j is -Theta_i (Eq. CE_theta_definition), and Sum_i Theta_i = 0
  * Sum e Omega^ii = F_i/(2 tau_i) with u_i^eq from Eq. first_order_moment_force
"""
import numpy as np
import pytest

from oracle import oracle as O

CASES = [
    (0, [1.0, 2.0], (1e-4, -2e-4, 0.0)),
    (0, [2.0, 28.0, 44.0], (0.0, -3e-4, 0.0)),
    (0, [1.0, 1.5, 4.0, 9.0], (2e-4, 1e-4, 0.0)),
    (1, [16.0, 28.0, 44.0], (1e-4, -2e-4, 3e-4)),
    (1, [1.0, 3.0], (0.0, 0.0, -1e-4)),
]


def _random_state(o, rng):
    e, w, _ = O.lattice_info(o.lattice)
    c, cs2, _ = o.species_info()
    f = np.zeros((o.ns, o.Q))
    for i in range(o.ns):
        rho = rng.uniform(0.2, 2.0)
        u = rng.uniform(-0.05, 0.05, 3) * c[i]
        if o.lattice == 0:
            u[2] = 0.0
        eu = (c[i] * e) @ u
        feq = w * rho * (1 + eu / cs2[i] + eu**2 / (2 * cs2[i] ** 2) - u @ u / (2 * cs2[i]))
        f[i] = feq * (1 + rng.uniform(-0.05, 0.05, o.Q))
    return f


@pytest.mark.parametrize("lattice,M,g", CASES)
def test_node_identities(lattice, M, g):
    rng = np.random.default_rng(7 + len(M) + 10 * lattice)
    ns = len(M)
    D = np.zeros((ns, ns))
    for i in range(ns):
        for j in range(i + 1, ns):
            D[i, j] = D[j, i] = rng.uniform(0.02, 0.1)
    o = O.Oracle(lattice, (2, 2, 2) if lattice == 1 else (2, 2), 0, M, D, 0.9, g)
    e, w, _ = O.lattice_info(lattice)
    c, cs2, tau = o.species_info()
    gv = np.array(g)
    for trial in range(5):
        f = _random_state(o, rng)
        fstar, dg = o.collide_node(f)
        d = O.diag_arrays(dg, ns, o.Q)
        rho = f.sum(axis=1)
        rho_mix = rho.sum()
        for i in range(ns):
            ei = c[i] * e.astype(float)
            j_i = ei.T @ f[i]
            F_i = rho[i] * gv
            # moments (Eq. zeroth_order_moment, first_order_moment_force)
            assert abs(d["rho"][i] - rho[i]) < 1e-14 * rho[i]
            assert np.allclose(d["ueq"][i], j_i / rho[i] + F_i / (2 * rho[i]), atol=1e-15)
            # f^(0): zeroth and first moments
            assert abs(d["f0"][i].sum() - rho[i]) < 1e-13
            assert np.allclose(ei.T @ d["f0"][i], rho[i] * d["ueq"][i], atol=1e-14)
            # f^(eq): moments up to second order with the mixture velocity
            u = d["u"]
            assert abs(d["feq"][i].sum() - rho[i]) < 1e-13
            assert np.allclose(ei.T @ d["feq"][i], rho[i] * u, atol=1e-14)
            Dm = 2 if lattice == 0 else 3
            P = np.einsum("a,ak,al->kl", d["feq"][i], ei, ei)[:Dm, :Dm]
            assert np.allclose(P, rho[i] * (cs2[i] * np.eye(Dm) + np.outer(u, u)[:Dm, :Dm]), atol=1e-13)
            # forcing term: zeroth, first and second moments (the last, u F + F u,
            # from the lattice's fourth-order isotropy; it is the only one of the
            # three that the second-order part of Eq. CE_forcing_term_discretized
            # contributes to)
            assert abs(d["S"][i].sum()) < 1e-15
            assert np.allclose(ei.T @ d["S"][i], F_i, atol=1e-16)
            PS = np.einsum("a,ak,al->kl", d["S"][i], ei, ei)[:Dm, :Dm]
            uF = (np.outer(u, F_i) + np.outer(F_i, u))[:Dm, :Dm]
            if np.abs(F_i).max() > 0:
                assert np.allclose(PS, uF, rtol=1e-10, atol=1e-12 * np.abs(uF).max())
            # self collision: mass zero, momentum F/(2 tau)
            assert abs(d["om_self"][i].sum()) < 1e-14
            assert np.allclose(ei.T @ d["om_self"][i], F_i / (2 * tau[i]), atol=1e-15)
            # cross collision, pair by pair
            theta = np.zeros(3)
            for j in range(ns):
                if j == i:
                    continue
                om = d["om_pair"][i, j]
                assert abs(om.sum()) < 1e-15
                expect = -rho[i] * rho[j] / (rho_mix * d["tau_x"][i, j]) * (d["ueq"][i] - d["ueq"][j])
                assert np.allclose(ei.T @ om, expect, atol=1e-15)
                theta -= ei.T @ om
            assert np.allclose(theta, d["theta"][i], atol=1e-15)
            # the update itself: Eq. (LBE_forcing) before streaming
            cross = sum(d["om_pair"][i, j] for j in range(ns) if j != i)
            upd = f[i] + d["om_self"][i] + cross + (1 - 1 / (2 * tau[i])) * d["S"][i]
            assert np.allclose(fstar[i], upd, atol=1e-15)
            # collision conserves species mass
            assert abs(fstar[i].sum() - rho[i]) < 1e-13
        assert np.allclose(d["theta"].sum(axis=0), 0.0, atol=1e-15)
        # total momentum gains exactly the total force
        P0 = sum((c[i] * e.astype(float)).T @ f[i] for i in range(ns))
        P1 = sum((c[i] * e.astype(float)).T @ fstar[i] for i in range(ns))
        assert np.allclose(P1 - P0, rho_mix * gv, atol=1e-15)
        # mixture velocity is the mass-weighted mean (Eq. Sirovich_mixture_velocity)
        assert np.allclose(d["u"], (rho[:, None] * d["ueq"]).sum(0) / rho_mix, atol=1e-16)
        # ideal mixture: n = sum rho_i/M_i, p = n M_1 c_s1^2
        assert abs(d["n"] - (rho / np.array(M)).sum()) < 1e-14
        assert abs(d["p"] - d["n"] * M[0] / 3.0) < 1e-15


def test_equal_species_velocities_make_cross_collision_vanish():
    # Eq. (Cross_collision_Sirovich) is proportional to u_i^eq - u_j^eq, and
    # Eq. (feqi0) reduces to f^(eq) when u_i^eq = u.
    M = [1.0, 2.0, 5.0]
    ns = 3
    D = np.full((3, 3), 0.05)
    o = O.Oracle(0, (2, 2), 0, M, D, 1.0, [0, 0, 0])
    e, w, _ = O.lattice_info(0)
    c, cs2, _ = o.species_info()
    u = np.array([0.01, -0.02, 0.0])
    f = np.zeros((ns, 9))
    for i in range(ns):
        rho = 0.5 + i
        # a distribution whose first moment is exactly rho u: equilibrium at u
        eu = (c[i] * e) @ u
        f[i] = w * rho * (1 + eu / cs2[i] + eu**2 / (2 * cs2[i] ** 2) - u @ u / (2 * cs2[i]))
    fstar, dg = o.collide_node(f)
    d = O.diag_arrays(dg, ns, 9)
    assert np.allclose(d["om_pair"], 0.0, atol=1e-15)
    assert np.allclose(d["f0"], d["feq"], atol=1e-15)
    assert np.allclose(d["om_self"], -(f - d["feq"]) / d["tau"][:, None], atol=1e-15)
    # at equilibrium with no force, nothing changes
    assert np.allclose(fstar, f, atol=1e-15)
