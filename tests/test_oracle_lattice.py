"""Pins of the oracle's lattice and species tables against what the paper and
lattice isotropy fix (no GPU)."""
import itertools
import math

import numpy as np
import pytest

from oracle import oracle as O


def test_d2q9_velocities_follow_the_paper_angles():
    # Eq. (discrete_velocity_DLS): alpha = 1..4 at angle (alpha-1) pi/2 with
    # magnitude c; alpha = 5..8 at (alpha-5) pi/2 + pi/4 with magnitude c sqrt(2).
    e, w, opp = O.lattice_info(0)
    assert e.shape == (9, 3)
    assert np.all(e[0] == 0)
    for a in range(1, 5):
        ang = (a - 1) * math.pi / 2
        assert e[a, 0] == round(math.cos(ang)) and e[a, 1] == round(math.sin(ang))
    for a in range(5, 9):
        ang = (a - 5) * math.pi / 2 + math.pi / 4
        assert e[a, 0] == round(math.sqrt(2) * math.cos(ang))
        assert e[a, 1] == round(math.sqrt(2) * math.sin(ang))
    assert np.all(e[:, 2] == 0)


@pytest.mark.parametrize("lattice,Q", [(0, 9), (1, 19)])
def test_weights_are_isotropic_with_cs2_one_third(lattice, Q):
    e, w, opp = O.lattice_info(lattice)
    D = 2 if lattice == 0 else 3
    E = e[:, :D].astype(float)
    assert len(w) == Q
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(np.einsum("a,ai->i", w, E), 0.0, atol=1e-16)
    assert np.allclose(np.einsum("a,ai,aj->ij", w, E, E), np.eye(D) / 3.0, atol=1e-15)
    assert np.allclose(np.einsum("a,ai,aj,ak->ijk", w, E, E, E), 0.0, atol=1e-16)
    m4 = np.einsum("a,ai,aj,ak,al->ijkl", w, E, E, E, E)
    d = np.eye(D)
    iso = (np.einsum("ij,kl->ijkl", d, d) + np.einsum("ik,jl->ijkl", d, d)
           + np.einsum("il,jk->ijkl", d, d)) / 9.0
    assert np.allclose(m4, iso, atol=1e-15)
    for a in range(Q):
        assert np.all(e[opp[a]] == -e[a])
    # no duplicate velocities
    assert len({tuple(v) for v in e}) == Q


def test_species_speeds_and_equal_viscosity():
    # Eq. (speed_DLS): c_i = sqrt(M_1/M_i), c_1 = 1 and c_s,i^2 = c_i^2/3; the
    # equal-viscosity constraint (tau_i - 1/2) c_s,i^2 = nu for every species.
    M = [2.0, 28.0, 44.0]
    o = O.Oracle(0, (3, 3), 0, M, np.full((3, 3), 0.05), 0.8, [0, 0, 0])
    c, cs2, tau = o.species_info()
    assert c[0] == 1.0
    for i in range(3):
        assert abs(c[i] ** 2 * M[i] - M[0]) < 1e-13
        assert abs(cs2[i] - c[i] ** 2 / 3.0) < 1e-16
    nu = (tau - 0.5) * cs2
    assert np.allclose(nu, (0.8 - 0.5) / 3.0, rtol=1e-14)


def test_oracle_rejects_bad_configurations():
    D = np.full((2, 2), 0.05)
    with pytest.raises(ValueError):
        O.Oracle(0, (4, 4), 0, [2.0, 1.0], D, 1.0, [0, 0, 0])      # masses not sorted
    with pytest.raises(ValueError):
        O.Oracle(0, (4, 4), 0, [1.0, 2.0], D, 0.5, [0, 0, 0])      # tau1 <= 1/2
    with pytest.raises(ValueError):
        O.Oracle(0, (4, 4), 0b0100, [1.0, 2.0], D, 1.0, [0, 0, 0])  # one-sided wall
    with pytest.raises(ValueError):
        O.Oracle(0, (4, 4, 2), 0, [1.0, 2.0], D, 1.0, [0, 0, 0])   # D2Q9 with nz > 1
