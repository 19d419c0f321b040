"""Seeded synthetic workloads for the EVD lattice Boltzmann step.

This module only draws numbers: species tables, diffusivities, body forces and
initial mole-fraction fields.  It contains none of the method's arithmetic, so
both the CUDA path and the CPU oracle can be fed from it.  Every random number
comes from SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) used as a counter-based generator: draw k of
stream s is ``splitmix64(seed + (s * 2**40 + k + 1) * 0x9E3779B97F4A7C15)``.

The paper has no public dataset.  The workloads below are stand-ins shaped like
its cases: the Loschmidt tube with gravity of Sec. 4.1 (two gases, one in each
half, periodic sides, impermeable ends) and a closed box relaxing to
gravitational stratification.

Field layout: ``x`` is float64 ``[ns][nz][ny][nx]`` (x fastest), mole fractions
summing to 1 at every node.  ``n`` (total number density) is ``None`` for the
uniform value 1.0.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED = 2504070591

WALL_X = 0b000011
WALL_Y = 0b001100
WALL_Z = 0b110000

D2Q9 = 0
D3Q19 = 1

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(stream: int, count: int, seed: int = SEED, start: int = 0) -> np.ndarray:
    """``count`` uint64 draws of stream ``stream`` beginning at index ``start``."""
    with np.errstate(over="ignore"):
        k = np.arange(start, start + count, dtype=np.uint64)
        ctr = np.uint64(stream) * np.uint64(1 << 40) + k + np.uint64(1)
        z = np.uint64(seed) + ctr * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(stream: int, count: int, seed: int = SEED) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits."""
    return (splitmix64(stream, count, seed) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(stream: int, count: int, seed: int = SEED) -> np.ndarray:
    """Standard normal draws by the Box-Muller transform of two uniform streams."""
    u1 = uniform01(stream, count, seed)
    u2 = uniform01(stream + 1, count, seed)
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


@dataclass
class Workload:
    name: str
    lattice: int
    shape: tuple            # (nx, ny, nz)
    wall_mask: int
    M: tuple                # molar masses, non-decreasing (species 0 lightest)
    D: np.ndarray           # [ns][ns] symmetric Maxwell-Stefan diffusivities, lattice units
    tau1: float             # self relaxation time of the lightest species
    g: tuple                # specific body force (gx, gy, gz), lattice units
    steps: int              # number of time steps of the full case
    x: np.ndarray = field(repr=False)   # [ns][nz][ny][nx]
    n: np.ndarray | None = field(default=None, repr=False)
    seed: int = SEED
    force: np.ndarray | None = field(default=None, repr=False)   # [3][nz][ny][nx] added to g
    flags: int = 0          # corrective forcing terms (bit 0 S_diff, 1 S_p, 2 S_rho)

    @property
    def ns(self) -> int:
        return len(self.M)

    @property
    def Q(self) -> int:
        return 9 if self.lattice == D2Q9 else 19

    @property
    def nsites(self) -> int:
        nx, ny, nz = self.shape
        return nx * ny * nz

    def describe(self) -> dict:
        nx, ny, nz = self.shape
        return {
            "workload": self.name,
            "lattice": "D2Q9" if self.lattice == D2Q9 else "D3Q19",
            "grid": [nx, ny] if self.lattice == D2Q9 else [nx, ny, nz],
            "species": self.ns,
            "molar_mass": list(self.M),
            "g": list(self.g),
            "tau1": self.tau1,
            "walls": wall_names(self.wall_mask),
            "seed": self.seed,
        }


def wall_names(mask: int) -> list:
    names = ["x-", "x+", "y-", "y+", "z-", "z+"]
    return [names[k] for k in range(6) if mask >> k & 1]


def pair_diffusivities(ns: int, lo: float, hi: float, stream: int, seed: int = SEED) -> np.ndarray:
    """Symmetric D_ij ~ U[lo, hi] for pairs (0,1),(0,2),...,(1,2),..., zero diagonal."""
    npair = ns * (ns - 1) // 2
    u = uniform01(stream, npair, seed)
    D = np.zeros((ns, ns))
    k = 0
    for i in range(ns):
        for j in range(i + 1, ns):
            D[i, j] = D[j, i] = lo + (hi - lo) * u[k]
            k += 1
    return D


def _renormalise(x: np.ndarray) -> np.ndarray:
    return x / x.sum(axis=0, keepdims=True)


def loschmidt_binary(nx: int = 4, ny: int = 256, steps: int = 2000) -> Workload:
    """Binary Loschmidt tube without gravity: M = (1, 2), D_12 = 0.05, x_1 = 0.9
    in rows y < ny/2 and 0.1 above, n = 1, walls at both ends of y, periodic x."""
    x = np.empty((2, 1, ny, nx))
    x[0, :, : ny // 2, :] = 0.9
    x[0, :, ny // 2:, :] = 0.1
    x[1] = 1.0 - x[0]
    D = np.array([[0.0, 0.05], [0.05, 0.0]])
    return Workload(f"loschmidt-binary-d2q9-{nx}x{ny}", D2Q9, (nx, ny, 1), WALL_Y,
                    (1.0, 2.0), D, 1.0, (0.0, 0.0, 0.0), steps, x)


GAS_A = (0.001, 0.299, 0.7)     # Sec. 4.1, gas A (x_1, x_2 = 1 - x_1 - x_3, x_3)
GAS_B = (0.8, 0.199, 0.001)     # Sec. 4.1, gas B


INTERFACE_WIDTH = 4.0


def loschmidt_ternary_gravity(nx: int = 64, ny: int = 1024, steps: int = 50000,
                              g: float = 1e-6, seed: int = SEED,
                              width: float = INTERFACE_WIDTH) -> Workload:
    """Ternary Loschmidt tube with gravity: M = (2, 28, 44), D_ij ~ U[0.02, 0.1],
    gravity g along -y, gas B in the lower half and gas A in the upper half.
    The two gases meet in an erf profile of half-width ``width`` nodes centred
    between rows ny/2 - 1 and ny/2 (a one-node jump of a 700:1 trace-species
    contrast is not resolvable by the lattice), then each mole fraction is
    scaled by (1 + 0.01 u), u ~ U[-1, 1], and renormalised."""
    from math import erf
    ns = 3
    x = np.empty((ns, 1, ny, nx))
    s = np.array([0.5 * (1.0 + erf((y + 0.5 - ny / 2) / width)) for y in range(ny)])
    for i in range(ns):
        x[i, 0, :, :] = (GAS_B[i] * (1.0 - s) + GAS_A[i] * s)[:, None]
    u = 2.0 * uniform01(2, x.size, seed).reshape(x.shape) - 1.0
    x = _renormalise(x * (1.0 + 0.01 * u))
    D = pair_diffusivities(ns, 0.02, 0.1, 1, seed)
    return Workload(f"loschmidt-ternary-gravity-d2q9-{nx}x{ny}", D2Q9, (nx, ny, 1), WALL_Y,
                    (2.0, 28.0, 44.0), D, 1.0, (0.0, -g, 0.0), steps, x, seed=seed)


def stratification_3d(n: int = 256, steps: int = 20000, g: float = 2e-6,
                      seed: int = SEED, shape: tuple | None = None) -> Workload:
    """Closed D3Q19 box, walls on all six faces, M = (16, 28, 44),
    D_ij ~ U[0.02, 0.1], gravity g along -y, x_i = (1/3)(1 + 0.01 N(0,1)) clipped
    positive and renormalised."""
    ns = 3
    nx, ny, nz = shape if shape is not None else (n, n, n)
    z = normal(4, ns * nx * ny * nz, seed).reshape(ns, nz, ny, nx)
    x = np.maximum((1.0 / 3.0) * (1.0 + 0.01 * z), 1e-6)
    x = _renormalise(x)
    D = pair_diffusivities(ns, 0.02, 0.1, 3, seed)
    return Workload(f"stratification-d3q19-{nx}x{ny}x{nz}", D3Q19, (nx, ny, nz),
                    WALL_X | WALL_Y | WALL_Z, (16.0, 28.0, 44.0), D, 1.0, (0.0, -g, 0.0),
                    steps, x, seed=seed)


def random_mixture(lattice: int, shape: tuple, wall_mask: int, M: tuple,
                   g: tuple = (0.0, 0.0, 0.0), tau1: float = 1.0,
                   dlo: float = 0.02, dhi: float = 0.1, amp: float = 0.2,
                   seed: int = SEED, stream: int = 10, n_amp: float = 0.0) -> Workload:
    """Small generic case for parity tests: uniform mixture with seeded
    mole-fraction noise of relative amplitude ``amp`` (and optionally a
    number-density field 1 + n_amp * U[-1, 1])."""
    ns = len(M)
    nx, ny, nz = (tuple(shape) + (1, 1))[:3]
    u = uniform01(stream, ns * nx * ny * nz, seed).reshape(ns, nz, ny, nx)
    x = _renormalise(np.full((ns, nz, ny, nx), 1.0 / ns) * (1.0 + amp * (2.0 * u - 1.0)))
    D = pair_diffusivities(ns, dlo, dhi, stream + 1, seed)
    nfield = None
    if n_amp:
        nfield = 1.0 + n_amp * (2.0 * uniform01(stream + 2, nx * ny * nz, seed).reshape(nz, ny, nx) - 1.0)
    gg = tuple(g) + (0.0,) * (3 - len(g))
    name = f"random-{'d2q9' if lattice == D2Q9 else 'd3q19'}-{nx}x{ny}x{nz}-ns{ns}"
    return Workload(name, lattice, (nx, ny, nz), wall_mask, tuple(float(m) for m in M), D,
                    tau1, gg, 0, x, nfield, seed)


def ultracentrifuge(R: int = 500, H: int = 3, xbar: float = 0.3, C: float = -1.2358e-8,
                    mass_ratio: float = 0.991481, tau1: float = 0.6, D12: float = 0.08,
                    steps: int = 2_000_000) -> Workload:
    """Case II of Sec. 4.2: a binary mixture (the paper's UF6 isotopes, M1/M2 =
    0.991481) in a cavity of R nodes along the radius r (the y axis, walls at
    both ends) and H nodes across (periodic), under the centrifugal specific
    force k(r) = omega^2 r along r, r = the node index.  The constant
    C = (M1 - M2) omega^2 / (R_U T) of the analytical profile fixes omega^2,
    with R_U T = M1 c_s1^2 and c_s1^2 = 1/3 (species 1 moves one node per
    step).  Initial state: mole fractions xbar, 1 - xbar everywhere and total
    mass density 1 (so n = 1 / sum x_i M_i)."""
    M1 = 1.0
    M2 = M1 / mass_ratio
    omega2 = C * M1 / 3.0 / (M1 - M2)
    x = np.empty((2, 1, R, H))
    x[0] = xbar
    x[1] = 1.0 - xbar
    n = np.full((1, R, H), 1.0 / (xbar * M1 + (1.0 - xbar) * M2))
    k = np.zeros((3, 1, R, H))
    k[1] = (omega2 * np.arange(R, dtype=np.float64))[None, :, None]
    D = np.array([[0.0, D12], [D12, 0.0]])
    return Workload(f"ultracentrifuge-d2q9-{H}x{R}", D2Q9, (H, R, 1), WALL_Y, (M1, M2), D, tau1,
                    (0.0, 0.0, 0.0), steps, x, n, force=k)


TUBE_BELOW = {2: (0.9, 0.1), 3: (0.7, 0.2, 0.1)}   # mole fractions in the lower half
TUBE_ABOVE = {2: (0.1, 0.9), 3: (0.1, 0.2, 0.7)}   # and in the upper half


def tube_length_and_species(k: int, lmin: int = 128, lmax: int = 4096, seed: int = SEED) -> tuple:
    """Length L and species count of tube k of the sweep below (the first two
    draws of its stream), without building its fields."""
    u = uniform01(1000 + 4 * k, 2, seed)
    return int(round(lmin * (lmax / lmin) ** u[0])), (2 if u[1] < 0.5 else 3)


def batched_tubes(count: int = 512, width: int = 32, lmin: int = 128, lmax: int = 4096,
                  steps: int = 10000, seed: int = SEED, width_interface: float = 0.0) -> list:
    """A sweep of independent D2Q9 Loschmidt tubes (periodic across the width,
    impermeable ends): tube k draws, from stream 1000 + 4k, its length
    L = lmin (lmax/lmin)^u log-uniform, 2 or 3 species (even odds), the mass
    ratio M_max/M_min ~ U[1, 10] (M_min = 1, an intermediate mass uniform in
    between), D_ij ~ U[0.01, 0.1] for two species and U[0.06, 0.1] for three
    (stream 1001 + 4k) and gravity g ~ U[0, 5e-6] along -y.  Ternary tubes
    with a mass ratio near 10 and D_ij below about 0.05 diverge within tens of
    steps even in FP64 (the cross relaxation over-relaxes), hence their
    narrower range.  Fill: a step profile at L/2 between the two compositions
    of TUBE_BELOW / TUBE_ABOVE (an erf of half-width ``width_interface`` nodes
    if it is > 0), number density 1."""
    from math import erf
    out = []
    for k in range(count):
        base = 1000 + 4 * k
        u = uniform01(base, 5, seed)
        L, ns = tube_length_and_species(k, lmin, lmax, seed)
        r = 1.0 + 9.0 * u[2]
        M = (1.0, r) if ns == 2 else (1.0, 1.0 + (r - 1.0) * u[3], r)
        g = 5e-6 * u[4]
        D = pair_diffusivities(ns, 0.01 if ns == 2 else 0.06, 0.1, base + 1, seed)
        if width_interface > 0:
            s = np.array([0.5 * (1.0 + erf((y + 0.5 - L / 2) / width_interface)) for y in range(L)])
        else:
            s = (np.arange(L) >= L // 2).astype(np.float64)
        x = np.empty((ns, 1, L, width))
        for i in range(ns):
            x[i, 0, :, :] = (TUBE_BELOW[ns][i] * (1.0 - s) + TUBE_ABOVE[ns][i] * s)[:, None]
        out.append(Workload(f"tube{k}-d2q9-{width}x{L}-ns{ns}", D2Q9, (width, L, 1), WALL_Y,
                            M, D, 1.0, (0.0, -g, 0.0), steps, x, seed=seed))
    return out


def by_name(name: str) -> Workload:
    """The full-size workloads by short name."""
    table = {
        "loschmidt-binary": loschmidt_binary,
        "loschmidt-ternary-gravity": loschmidt_ternary_gravity,
        "stratification-3d": stratification_3d,
    }
    return table[name]()
