"""Pins of the cross relaxation times (Sec. 3, Eq. relation_tauij_diff_coeff;
Sec. 4.1 ternary closed forms; Eq. Luo&Girimaji_tau)."""
import numpy as np
import pytest

from oracle import oracle as O


def _residual(M, D, rho, tau):
    """Residual of the linear system in 1/tau_ij for every pair i<j,
    A_ij/tau_ij + (1/D_ij) sum_{s != i,j} rho_s/tau_sj - B_ij, with
    A_ij = (rho_i + rho_j)/D_ij + 2 n^2 M_i M_j/p and B_ij = 2 rho/D_ij, dt = 1."""
    ns = len(M)
    n = sum(rho[i] / M[i] for i in range(ns))
    p = n * M[0] / 3.0
    rho_mix = sum(rho)
    res = []
    for i in range(ns):
        for j in range(i + 1, ns):
            A = (rho[i] + rho[j]) / D[i, j] + 2 * n * n * M[i] * M[j] / p
            B = 2 * rho_mix / D[i, j]
            r = A / tau[i, j] + sum(rho[s] / tau[s, j] for s in range(ns) if s not in (i, j)) / D[i, j] - B
            res.append(r / B)
    return np.array(res)


def _cfg(M, D):
    return O.make_config(0, (2, 2), 0, M, D, 1.0, [0, 0, 0])


def test_binary_dense_solve_reduces_to_luo_girimaji():
    rng = np.random.default_rng(1)
    for _ in range(20):
        M = sorted(rng.uniform(1, 50, 2))
        D = np.zeros((2, 2)); D[0, 1] = D[1, 0] = rng.uniform(0.01, 0.2)
        rho = rng.uniform(0.05, 5, 2)
        cfg = _cfg(M, D)
        t_closed = O.tau_cross(cfg, rho)
        t_dense = O.tau_cross(cfg, rho, dense=True)
        assert abs(t_closed[0, 1] - t_dense[0, 1]) < 1e-13 * t_dense[0, 1]
        assert np.all(np.abs(_residual(M, D, rho, t_closed)) < 1e-13)
        # Luo-Girimaji: tau_12 - 1/2 is proportional to D_12 at fixed state
        D2 = D * 3.0
        t3 = O.tau_cross(_cfg(M, D2), rho)
        assert abs((t3[0, 1] - 0.5) - 3.0 * (t_closed[0, 1] - 0.5)) < 1e-12


def test_ternary_closed_form_solves_the_system():
    rng = np.random.default_rng(2)
    for _ in range(50):
        M = sorted(rng.uniform(1, 50, 3))
        D = np.zeros((3, 3))
        for i, j in ((0, 1), (0, 2), (1, 2)):
            D[i, j] = D[j, i] = rng.uniform(0.01, 0.15)
        rho = rng.uniform(0.02, 40, 3)
        cfg = _cfg(M, D)
        tc = O.tau_cross(cfg, rho)
        td = O.tau_cross(cfg, rho, dense=True)
        assert np.allclose(tc, tc.T, rtol=0, atol=0)
        assert np.allclose(tc, td, rtol=1e-12)
        assert np.all(np.abs(_residual(M, D, rho, tc)) < 1e-12)


@pytest.mark.parametrize("ns", [4, 5, 6])
def test_dense_solve_for_more_species(ns):
    rng = np.random.default_rng(ns)
    M = sorted(rng.uniform(1, 50, ns))
    D = np.zeros((ns, ns))
    for i in range(ns):
        for j in range(i + 1, ns):
            D[i, j] = D[j, i] = rng.uniform(0.02, 0.1)
    rho = rng.uniform(0.1, 5, ns)
    t = O.tau_cross(_cfg(M, D), rho)
    assert np.all(np.abs(_residual(M, D, rho, t)) < 1e-12)


def test_tau_is_invariant_under_a_common_mass_scale():
    # Only mass ratios enter tau_ij: with rho_i = x_i M_i n, the combination
    # n^2 M_i M_j/(p rho) has degree zero in a common scale of the masses.
    M = np.array([2.0, 28.0, 44.0])
    D = np.zeros((3, 3))
    D[0, 1] = D[1, 0] = 0.03; D[0, 2] = D[2, 0] = 0.07; D[1, 2] = D[2, 1] = 0.05
    x = np.array([0.2, 0.3, 0.5])
    t1 = O.tau_cross(_cfg(M, D), x * M)
    t2 = O.tau_cross(_cfg(M * 8.0, D), x * M * 8.0)
    assert np.allclose(t1, t2, rtol=1e-13)
