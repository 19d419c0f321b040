"""Pins of the oracle's streaming: the second-order interpolation
(Eq. Second_order_spatial_interpolation) and the impermeable-wall scheme of
App. A, checked against
  * the paper's own wall equations, transcribed below in pull form for the
    right, left, upper and bottom walls of a D2Q9 domain;
  * exact streaming and half-way bounce-back when all masses are equal (App. A,
    last paragraph; Eq. standard_BBscheme);
  * the closed-form Fourier amplification of the 1-D three-point scheme
    (the Lax-Wendroff factor 1 - s^2 (1 - cos k) - i s sin k);
  * exact conservation of every species' mass with walls (App. A argument);
  * an independent gather-form restatement on tiny grids, corners included.
"""
import itertools

import numpy as np
import pytest

from oracle import oracle as O
from paper_2504_07059_gb300 import workloads as W

# node letters of the paper's interpolation figure, offsets (dx, dy) from O
LETTER = {"O": (0, 0), "A": (1, 0), "B": (0, 1), "C": (-1, 0), "D": (0, -1),
          "E": (1, 1), "F": (-1, 1), "G": (-1, -1), "H": (1, -1)}
OPP2 = [0, 3, 4, 1, 2, 7, 8, 5, 6]


def standard_terms(xi, eta):
    """Coefficient of f(X') for each node letter X in Eq.
    (Second_order_spatial_interpolation)."""
    return {
        "O": (1 - eta**2) * (1 - xi**2),
        "C": xi * (1 - eta**2) * (1 + xi) / 2,
        "D": eta * (1 + eta) * (1 - xi**2) / 2,
        "G": eta * xi * (1 + eta) * (1 + xi) / 4,
        "A": -xi * (1 - xi) * (1 - eta**2) / 2,
        "B": -eta * (1 - eta) * (1 - xi**2) / 2,
        "F": -eta * xi * (1 + xi) * (1 - eta) / 4,
        "H": -eta * xi * (1 - xi) * (1 + eta) / 4,
        "E": eta * xi * (1 - xi) * (1 - eta) / 4,
    }


def _val(fs, a, x, y, letter):
    ny, nx = fs.shape[-2:]
    dx, dy = LETTER[letter]
    return fs[a, 0, (y + dy) % ny, (x + dx) % nx]


def paper_pull(fs, c, x, y, wall):
    """f_alpha(O) for all alpha at node (x, y) from the post-collision field fs
    [Q][1][ny][nx] of one species with lattice speed c, following App. A for a
    node next to ``wall`` ('right', 'left', 'upper', 'bottom' or None)."""
    e = O.lattice_info(0)[0]
    out = np.zeros(9)
    solid = {"right": "AEH", "left": "CFG", "upper": "BEF", "bottom": "DGH", None: ""}[wall]
    F = lambda a, L: _val(fs, a, x, y, L)
    for a in range(9):
        xi, eta = c * e[a, 0], c * e[a, 1]
        ab = OPP2[a]
        if wall == "right" and a == 3:
            x1 = c  # xi_1
            out[a] = (F(3, "O") + x1**2 / 2 * (F(1, "O") + F(3, "C") - F(3, "O"))
                      + x1 / 2 * (F(1, "O") - F(3, "C") - F(3, "O")))
        elif wall == "right" and a in (6, 7):
            out[a] = (((1 - eta**2) * (1 - xi**2) + xi * (1 + xi) / 2) * F(a, "O")
                      + xi * (1 + xi) * (1 - eta**2) / 2 * F(a, "C")
                      + eta * (1 + eta) * (1 - xi**2) / 2 * F(a, "D")
                      + eta * xi * (1 + eta) * (1 + xi) / 4 * F(a, "G")
                      - eta * (1 - eta) * (1 - xi**2) / 2 * F(a, "B")
                      - eta * xi * (1 + xi) * (1 - eta) / 4 * F(a, "F")
                      - xi * (1 - xi) / 2 * F(ab, "O"))
        elif wall == "left" and a == 1:
            x1 = c
            out[a] = (F(1, "O") + x1**2 / 2 * (F(3, "O") + F(1, "A") - F(1, "O"))
                      + x1 / 2 * (F(3, "O") - F(1, "A") - F(1, "O")))
        elif wall == "left" and a in (5, 8):
            out[a] = (((1 - eta**2) * (1 - xi**2) - xi * (1 - xi) / 2) * F(a, "O")
                      - xi * (1 - xi) * (1 - eta**2) / 2 * F(a, "A")
                      - eta * (1 - eta) * (1 - xi**2) / 2 * F(a, "B")
                      + eta * (1 + eta) * (1 - xi**2) / 2 * F(a, "D")
                      - eta * xi * (1 - xi) * (1 + eta) / 4 * F(a, "H")
                      + eta * xi * (1 - xi) * (1 - eta) / 4 * F(a, "E")
                      + xi * (1 + xi) / 2 * F(ab, "O"))
        elif wall == "upper" and a == 4:
            e2 = c  # eta_2
            out[a] = (F(4, "O") + e2**2 / 2 * (F(2, "O") + F(4, "D") - F(4, "O"))
                      + e2 / 2 * (F(2, "O") - F(4, "D") - F(4, "O")))
        elif wall == "upper" and a in (7, 8):
            out[a] = (((1 - eta**2) * (1 - xi**2) + eta * (1 + eta) / 2) * F(a, "O")
                      + eta * (1 - xi**2) * (1 + eta) / 2 * F(a, "D")
                      + xi * (1 + xi) * (1 - eta**2) / 2 * F(a, "C")
                      - xi * (1 - xi) * (1 - eta**2) / 2 * F(a, "A")
                      + eta * xi * (1 + eta) * (1 + xi) / 4 * F(a, "G")
                      - eta * xi * (1 - xi) * (1 + eta) / 4 * F(a, "H")
                      - eta * (1 - eta) / 2 * F(ab, "O"))
        elif wall == "bottom" and a == 2:
            e2 = c
            out[a] = (F(2, "O") + e2**2 / 2 * (F(4, "O") + F(2, "B") - F(2, "O"))
                      + e2 / 2 * (F(4, "O") - F(2, "B") - F(2, "O")))
        elif wall == "bottom" and a in (5, 6):
            out[a] = (((1 - eta**2) * (1 - xi**2) - eta * (1 - eta) / 2) * F(a, "O")
                      + xi * (1 - eta**2) * (1 + xi) / 2 * F(a, "C")
                      - xi * (1 - xi) * (1 - eta**2) / 2 * F(a, "A")
                      - eta * (1 - eta) * (1 - xi**2) / 2 * F(a, "B")
                      - eta * xi * (1 + xi) * (1 - eta) / 4 * F(a, "F")
                      + eta * xi * (1 - xi) * (1 - eta) / 4 * F(a, "E")
                      + eta * (1 + eta) / 2 * F(ab, "O"))
        else:
            # every other direction: the interior formula without solid nodes
            out[a] = sum(coef * F(a, L) for L, coef in standard_terms(xi, eta).items()
                         if L not in solid)
    return out


@pytest.mark.parametrize("walls", ["x", "y"])
@pytest.mark.parametrize("M2", [2.0, 7.0, 1.3])
def test_wall_equations_of_appendix_a(walls, M2):
    nx, ny = 7, 6
    mask = W.WALL_X if walls == "x" else W.WALL_Y
    M = [1.0, M2]
    o = O.Oracle(0, (nx, ny), mask, M, np.full((2, 2), 0.05), 1.0, [0, 0, 0])
    c, _, _ = o.species_info()
    rng = np.random.default_rng(int(M2 * 10))
    fs = rng.uniform(0.1, 1.0, (2, 9, 1, ny, nx))
    o.set_f(fs)
    o.stream_only()
    f = o.get_f()
    for i in range(2):
        for y in range(ny):
            for x in range(nx):
                wall = None
                if walls == "x" and x == nx - 1:
                    wall = "right"
                elif walls == "x" and x == 0:
                    wall = "left"
                elif walls == "y" and y == ny - 1:
                    wall = "upper"
                elif walls == "y" and y == 0:
                    wall = "bottom"
                expect = paper_pull(fs[i], c[i], x, y, wall)
                np.testing.assert_allclose(f[i, :, 0, y, x], expect, rtol=1e-14, atol=1e-15,
                                           err_msg=f"species {i} node ({x},{y}) wall {wall}")


@pytest.mark.parametrize("lattice,shape,mask", [
    (0, (5, 4), 0), (0, (5, 4), W.WALL_Y), (0, (3, 6), W.WALL_X | W.WALL_Y),
    (1, (3, 4, 5), 0), (1, (4, 3, 3), W.WALL_X | W.WALL_Y | W.WALL_Z)])
def test_equal_masses_give_exact_streaming_and_halfway_bounce_back(lattice, shape, mask):
    # App. A: with equal masses |xi| = |eta| = 1 and the scheme becomes Eq.
    # (standard_BBscheme); away from walls streaming is an exact shift.
    e, _, opp = O.lattice_info(lattice)
    Q = len(e)
    o = O.Oracle(lattice, shape, mask, [3.0, 3.0], np.full((2, 2), 0.05), 1.0, [0, 0, 0])
    rng = np.random.default_rng(3)
    grid = o.grid
    fs = rng.uniform(0.1, 1.0, (2, Q) + grid)
    o.set_f(fs)
    o.stream_only()
    f = o.get_f()
    nz, ny, nx = grid
    expect = np.zeros_like(fs)
    for i in range(2):
        for a in range(Q):
            for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
                dest = [x + e[a, 0], y + e[a, 1], z + e[a, 2]]
                nn = [nx, ny, nz]
                hit = False
                for k in range(3):
                    if dest[k] < 0 or dest[k] >= nn[k]:
                        if (mask >> (2 * k)) & 3:
                            hit = True
                        else:
                            dest[k] %= nn[k]
                if hit:
                    expect[i, opp[a], z, y, x] += fs[i, a, z, y, x]
                else:
                    expect[i, a, dest[2], dest[1], dest[0]] += fs[i, a, z, y, x]
    assert np.array_equal(f, expect)


@pytest.mark.parametrize("M2", [2.0, 4.0, 1.7])
def test_fourier_amplification_matches_lax_wendroff(M2):
    nx, ny = 32, 16
    o = O.Oracle(0, (nx, ny), 0, [1.0, M2], np.full((2, 2), 0.05), 1.0, [0, 0, 0])
    c, _, _ = o.species_info()
    e, _, _ = O.lattice_info(0)
    s = c[1]
    kx, ky = 2 * np.pi * 3 / nx, 2 * np.pi * 2 / ny
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
    phase = kx * X + ky * Y + 0.3
    fs = np.zeros((2, 9, 1, ny, nx))
    fs[1, :, 0] = np.cos(phase)[None]
    o.set_f(fs)
    o.stream_only()
    f = o.get_f()
    G = lambda sk, k: 1 - sk**2 * (1 - np.cos(k)) - 1j * sk * np.sin(k)
    for a in range(9):
        amp = G(s * e[a, 0], kx) * G(s * e[a, 1], ky)
        expect = np.real(amp * np.exp(1j * phase))
        np.testing.assert_allclose(f[1, a, 0], expect, atol=2e-15)


@pytest.mark.parametrize("lattice,shape,mask,M", [
    (0, (6, 5), W.WALL_X | W.WALL_Y, [1.0, 2.0, 9.0]),
    (0, (1, 7), W.WALL_X | W.WALL_Y, [1.0, 5.0]),
    (1, (5, 4, 6), W.WALL_X | W.WALL_Y | W.WALL_Z, [16.0, 28.0, 44.0]),
    (1, (4, 4, 3), W.WALL_Z, [1.0, 3.0])])
def test_streaming_conserves_each_species_mass(lattice, shape, mask, M):
    ns = len(M)
    o = O.Oracle(lattice, shape, mask, M, np.full((ns, ns), 0.05), 1.0, [0, 0, 0])
    rng = np.random.default_rng(11)
    fs = rng.uniform(0.1, 1.0, (ns, o.Q) + o.grid)
    o.set_f(fs)
    m0 = o.mass()
    o.stream_only()
    m1 = o.mass()
    assert np.allclose(m1, m0, rtol=2e-15)
    assert np.allclose(m0, fs.reshape(ns, -1).sum(axis=1), rtol=1e-14)


def gather_restatement(fs, lattice, c, mask):
    """Pull-form restatement of the oracle's streaming rule for one species:
    f_a(O) = sum over fluid sources O - d of W_a(d) fs_a(O - d)
           + [sum over solid targets O + d with e_a . d_s <= 0 of W_a(d)] fs_a(O)
           + [sum over solid targets O + d with e_abar . d_s > 0 of W_abar(d)] fs_abar(O)."""
    e, _, opp = O.lattice_info(lattice)
    Q = len(e)
    nz, ny, nx = fs.shape[1:]
    nn = (nx, ny, nz)
    Dm = 2 if lattice == 0 else 3

    def W1(s, d):
        return {0: 1 - s * s, 1: s * (1 + s) / 2, -1: -s * (1 - s) / 2}[d]

    offs = list(itertools.product(*([(-1, 0, 1)] * Dm)))
    out = np.zeros_like(fs)
    for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
        O_ = (x, y, z)
        for a in range(Q):
            acc = 0.0
            for d in offs:
                d3 = tuple(d) + (0,) * (3 - Dm)
                wgt = np.prod([W1(c * e[a, k], d3[k]) for k in range(Dm)])
                # pull: source O - d
                src = list(O_[k] - d3[k] for k in range(3))
                ok = True
                for k in range(3):
                    if src[k] < 0 or src[k] >= nn[k]:
                        if (mask >> (2 * k)) & 3:
                            ok = False
                        else:
                            src[k] %= nn[k]
                if ok:
                    acc += wgt * fs[a, src[2], src[1], src[0]]
                # push targets from O for the lumped terms
                for b, into in ((a, "self"), (opp[a], "opp")):
                    wb = np.prod([W1(c * e[b, k], d3[k]) for k in range(Dm)])
                    dot, crossed = 0, False
                    for k in range(3):
                        t = O_[k] + d3[k]
                        if (t < 0 or t >= nn[k]) and (mask >> (2 * k)) & 3:
                            crossed = True
                            dot += e[b, k] * d3[k]
                    if not crossed:
                        continue
                    if into == "self" and dot <= 0:
                        acc += wb * fs[a, z, y, x]
                    if into == "opp" and dot > 0:
                        acc += wb * fs[b, z, y, x]
            out[a, z, y, x] = acc
    return out


@pytest.mark.parametrize("lattice,shape,mask,M", [
    (0, (4, 5), W.WALL_X | W.WALL_Y, [1.0, 2.5]),
    (0, (2, 3), W.WALL_Y, [1.0, 6.0]),
    (1, (3, 4, 3), W.WALL_X | W.WALL_Y | W.WALL_Z, [1.0, 1.9]),
    (1, (3, 3, 4), W.WALL_Y, [2.0, 5.0])])
def test_scatter_matches_gather_restatement(lattice, shape, mask, M):
    o = O.Oracle(lattice, shape, mask, M, np.full((2, 2), 0.05), 1.0, [0, 0, 0])
    c, _, _ = o.species_info()
    rng = np.random.default_rng(5)
    fs = rng.uniform(0.1, 1.0, (2, o.Q) + o.grid)
    o.set_f(fs)
    o.stream_only()
    f = o.get_f()
    for i in range(2):
        g = gather_restatement(fs[i], lattice, c[i], mask)
        np.testing.assert_allclose(f[i], g, rtol=1e-13, atol=1e-15)
