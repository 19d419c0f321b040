"""The oracle's own discrete adjoint of the forced EVD step (D2Q9, FP64).

TEST INFRASTRUCTURE ONLY.  Only ``tests/`` may import this module; the CUDA
library never does, and it shares nothing with it.

The forward map is the oracle's discrete map theta -> L, restated with plain
PyTorch CPU tensor operations in float64 (vectorised over the nodes, in the
same order of terms as ``evd_oracle.c``), so that ``torch.autograd`` -- a
library primitive -- takes its exact reverse-mode derivative.  theta is the
Maxwell-Stefan diffusivity of each species pair and the body force (g_x, g_y);
L = sum_i sum_y (xbar_i(y) - target_i(y))^2 with xbar_i(y) the mean over x of
the mole fractions after N steps.  Steps, in the paper's order:

  initial state   f = [1 + e.u_i0/c_s^2] w rho_i, rho_i = x_i M_i n,
                  u_i0 = -g dt/2 (Sec. 4.1/4.2, Eq. feqi0 with u = 0)
  moments         Eq. zeroth_order_moment, Eq. first_order_moment_force,
                  Eq. Sirovich_mixture_velocity
  tau_ij          Eq. Luo&Girimaji_tau (binary), the closed forms of Sec. 4.1
                  (ternary), from Eq. relation_tauij_diff_coeff
  collision       Eq. LBE_forcing term by term: Omega^ii (Eq. BGK_self_collision,
                  with f^(0) of Eq. feqi0), Omega^ij pair by pair (Eq.
                  Cross_collision_Sirovich), S^i (Eq. CE_forcing_term_discretized)
  streaming       Eq. Second_order_spatial_interpolation as a scatter with the
                  tensor-product weights W(s;0) = 1 - s^2, W(s;+1) = s(1+s)/2,
                  W(s;-1) = -s(1-s)/2; weight that would reach a solid node is
                  kept at the source node, in the opposite direction when the
                  population heads into the crossed wall(s) and in the same
                  direction otherwise (App. A; at edges and corners the tie
                  keeps the direction)
  readout         x_i = rho_i / (n M_i), n = sum_j rho_j / M_j

Pinned in ``tests/test_oracle_adjoint.py``: the forward populations and loss
against the C oracle, the gradient against finite differences of the C
oracle's loss, and reverse against forward mode (the dot-product test).
"""
from __future__ import annotations

import numpy as np
import torch

# D2Q9 in the order of Eq. (discrete_velocity_DLS): rest, the four axis
# directions at angles (a-1) pi/2, the four diagonals at (a-5) pi/2 + pi/4.
E = ((0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1))
WEIGHT = (4.0 / 9.0,) + (1.0 / 9.0,) * 4 + (1.0 / 36.0,) * 4
OPP = (0, 3, 4, 1, 2, 7, 8, 5, 6)
Q = 9
DT = 1.0


def _w1(s: float, d: int) -> float:
    if d == 0:
        return 1.0 - s * s
    if d == 1:
        return s * (1.0 + s) / 2.0
    return -s * (1.0 - s) / 2.0


def _f64(v):
    """float64 tensor of v (a tensor keeps its autograd graph)."""
    if isinstance(v, torch.Tensor):
        if v.dtype != torch.float64:
            raise TypeError("parameters must be float64")
        return v
    return torch.as_tensor(np.asarray(v, dtype=np.float64))


class Model:
    """The discrete map for one lattice: ``shape`` (nx, ny), ``wall_mask``
    bits 0/1 the x faces and 2/3 the y faces (both or neither), molar masses
    non-decreasing (species 0 the lightest, c = 1), two or three species."""

    def __init__(self, shape, wall_mask: int, M, tau1: float):
        self.nx, self.ny = int(shape[0]), int(shape[1])
        self.walled = (bool(wall_mask & 3), bool((wall_mask >> 2) & 3))
        self.M = tuple(float(m) for m in M)
        self.ns = len(self.M)
        if self.ns not in (2, 3):
            raise ValueError("two or three species")
        M1 = self.M[0]
        self.c = [float(np.sqrt(M1 / m)) for m in self.M]
        self.cs2 = [c * c / 3.0 for c in self.c]
        # equal kinematic viscosity: (tau_i - 1/2) cs2_i = (tau_1 - 1/2) cs2_1
        self.tau = [0.5 + (tau1 - 0.5) * (self.cs2[0] / cs2) for cs2 in self.cs2]
        self._stream_plan = self._plan()

    # -------------------------------------------------------------- streaming
    def _plan(self):
        """Per (species, direction): the (weight, dx, dy) terms of the scatter
        and, per term, the source masks of the wall rule."""
        xs = torch.arange(self.nx).view(1, -1).expand(self.ny, self.nx)
        ys = torch.arange(self.ny).view(-1, 1).expand(self.ny, self.nx)
        plan = []
        for i in range(self.ns):
            per_a = []
            for a in range(Q):
                sx, sy = self.c[i] * E[a][0], self.c[i] * E[a][1]
                terms = []
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        wgt = 1.0 * _w1(sx, dx) * _w1(sy, dy)
                        if wgt == 0.0:
                            continue
                        cx = self.walled[0] & ((xs + dx < 0) | (xs + dx >= self.nx))
                        cy = self.walled[1] & ((ys + dy < 0) | (ys + dy >= self.ny))
                        crossed = cx | cy
                        dot = E[a][0] * dx * cx.long() + E[a][1] * dy * cy.long()
                        into = crossed & (dot > 0)      # kept in the opposite direction
                        keep = crossed & ~(dot > 0)     # kept in the same direction
                        terms.append((wgt, dx, dy, (~crossed).double(), keep.double(), into.double()))
                per_a.append(terms)
            plan.append(per_a)
        return plan

    def stream(self, fs: torch.Tensor) -> torch.Tensor:
        """fs [ns][Q][ny][nx] post-collision -> post-stream populations."""
        out = []
        for i in range(self.ns):
            acc = [torch.zeros(self.ny, self.nx, dtype=fs.dtype) for _ in range(Q)]
            for a in range(Q):
                src = fs[i, a]
                for wgt, dx, dy, free, keep, into in self._stream_plan[i][a]:
                    part = wgt * src
                    # fluid destinations (a walled dimension never wraps here)
                    acc[a] = acc[a] + torch.roll(part * free, shifts=(dy, dx), dims=(0, 1))
                    acc[a] = acc[a] + part * keep
                    acc[OPP[a]] = acc[OPP[a]] + part * into
            out.append(torch.stack(acc))
        return torch.stack(out)

    # -------------------------------------------------------------- collision
    def tau_cross(self, rho, D):
        """tau_ij per node from Eq. relation_tauij_diff_coeff (closed forms)."""
        n = 0.0
        rho_mix = 0.0
        for i in range(self.ns):
            n = n + rho[i] / self.M[i]
            rho_mix = rho_mix + rho[i]
        p = n * self.M[0] * (1.0 / 3.0)
        if self.ns == 2:
            t12 = DT / 2.0 + n * n * self.M[0] * self.M[1] / (p * rho_mix) * D[(0, 1)]
            return {(0, 1): t12, (1, 0): t12}
        r1, r2, r3 = rho[0], rho[1], rho[2]
        D12, D13, D23 = D[(0, 1)], D[(0, 2)], D[(1, 2)]
        M1, M2, M3 = self.M
        A12 = (r1 + r2) / D12 + 2.0 * n * n * M1 * M2 / (p * DT)
        A13 = (r1 + r3) / D13 + 2.0 * n * n * M1 * M3 / (p * DT)
        A23 = (r2 + r3) / D23 + 2.0 * n * n * M2 * M3 / (p * DT)
        B12 = 2.0 * rho_mix / (D12 * DT)
        B13 = 2.0 * rho_mix / (D13 * DT)
        B23 = 2.0 * rho_mix / (D23 * DT)
        t23 = (A23 - r1 * r2 / (A13 * D13 * D23)) / (B23 - r1 * B13 / (A13 * D23))
        t12 = 1.0 / (B12 / A12 - r3 / (A12 * D12 * t23))
        t13 = 1.0 / (B13 / A13 - r2 / (A13 * D13 * t23))
        return {(0, 1): t12, (1, 0): t12, (0, 2): t13, (2, 0): t13, (1, 2): t23, (2, 1): t23}

    def moments(self, f, g):
        """rho_i, u_i^eq (forced), mixture density and velocity per node."""
        rho, ueq = [], []
        rho_mix = 0.0
        for i in range(self.ns):
            r = 0.0
            mom = [0.0, 0.0]
            for a in range(Q):
                fa = f[i, a]
                r = r + fa
                for k in range(2):
                    mom[k] = mom[k] + self.c[i] * E[a][k] * fa
            F = [r * g[k] for k in range(2)]   # F_i = rho_i g
            ueq.append([mom[k] / r + F[k] * DT / (2.0 * r) for k in range(2)])
            rho.append(r)
            rho_mix = rho_mix + r
        u = [0.0, 0.0]
        for i in range(self.ns):
            for k in range(2):
                u[k] = u[k] + (rho[i] / rho_mix) * ueq[i][k]
        return rho, ueq, rho_mix, u

    def collide(self, f, D, g):
        rho, ueq, rho_mix, u = self.moments(f, g)
        tx = self.tau_cross(rho, D)
        out = []
        for i in range(self.ns):
            cs2, tau_i = self.cs2[i], self.tau[i]
            F = [rho[i] * g[k] for k in range(2)]
            rows = []
            for a in range(Q):
                ei = [self.c[i] * E[a][k] for k in range(2)]
                emu = [ei[k] - u[k] for k in range(2)]
                eu = 0.0
                usq = 0.0
                proj = 0.0
                for k in range(2):
                    eu = eu + ei[k] * u[k]
                    usq = usq + u[k] * u[k]
                    proj = proj + emu[k] * (ueq[i][k] - u[k])
                feq = WEIGHT[a] * rho[i] * (1.0 + eu / cs2 + (eu * eu) / (2.0 * cs2 * cs2) - usq / (2.0 * cs2))
                f0 = (1.0 + proj / cs2) * feq
                om_self = -(f[i, a] - f0) / tau_i
                om_cross = 0.0
                for j in range(self.ns):
                    if j == i:
                        continue
                    dv = 0.0
                    for k in range(2):
                        dv = dv + emu[k] * (ueq[i][k] - ueq[j][k])
                    om_cross = om_cross + -(1.0 / tx[(i, j)]) * (rho[j] / rho_mix) * (feq / cs2) * dv
                S = 0.0
                for k in range(2):
                    v = ei[k] / cs2
                    for l in range(2):
                        v = v + (ei[k] * ei[l] - cs2 * (1.0 if k == l else 0.0)) / (cs2 * cs2) * u[l]
                    S = S + v * F[k]
                S = S * WEIGHT[a]
                rows.append(f[i, a] + om_self + om_cross + (1.0 - DT / (2.0 * tau_i)) * S)
            out.append(torch.stack(rows))
        return torch.stack(out)

    # ---------------------------------------------------------- state, readout
    def initial(self, x0, n0, g):
        """x0 [ns][ny][nx] mole fractions, n0 [ny][nx] or None."""
        x0 = torch.as_tensor(np.asarray(x0, dtype=np.float64).reshape(self.ns, self.ny, self.nx))
        n = (torch.ones(self.ny, self.nx, dtype=torch.float64) if n0 is None
             else torch.as_tensor(np.asarray(n0, dtype=np.float64).reshape(self.ny, self.nx)))
        out = []
        for i in range(self.ns):
            rho_i = x0[i] * self.M[i] * n
            ui0 = [0.0 - rho_i * g[k] * DT / (2.0 * rho_i) for k in range(2)]
            rows = []
            for a in range(Q):
                eu0 = 0.0
                for k in range(2):
                    eu0 = eu0 + self.c[i] * E[a][k] * ui0[k]
                rows.append((1.0 + eu0 / self.cs2[i]) * WEIGHT[a] * rho_i)
            out.append(torch.stack(rows))
        return torch.stack(out)

    def mole_fractions(self, f):
        rho = []
        for i in range(self.ns):
            r = 0.0
            for a in range(Q):
                r = r + f[i, a]
            rho.append(r)
        n = 0.0
        for i in range(self.ns):
            n = n + rho[i] / self.M[i]
        return torch.stack([rho[i] / (n * self.M[i]) for i in range(self.ns)])

    def run(self, x0, n0, nsteps: int, d_pairs, g):
        """Post-stream populations f_N [ns][Q][ny][nx] (differentiable in
        d_pairs, one per pair i < j, and g = (g_x, g_y))."""
        d_pairs, g = _f64(d_pairs), _f64(g)
        D = {}
        k = 0
        for i in range(self.ns):
            for j in range(i + 1, self.ns):
                D[(i, j)] = D[(j, i)] = d_pairs[k]
                k += 1
        gg = [g[0], g[1]]
        f = self.initial(x0, n0, gg)
        for _ in range(nsteps):
            f = self.stream(self.collide(f, D, gg))
        return f

    def loss(self, x0, n0, nsteps, target, d_pairs, g):
        f = self.run(x0, n0, nsteps, d_pairs, g)
        xbar = self.mole_fractions(f).mean(dim=2)       # [ns][ny]
        t = torch.as_tensor(np.asarray(target, dtype=np.float64).reshape(self.ns, self.ny))
        return ((xbar - t) ** 2).sum()


def loss_and_gradient(shape, wall_mask, M, tau1, x0, target, nsteps, d_pairs, g, n0=None):
    """(L, dL/d d_pairs, dL/d(g_x, g_y)) by reverse mode through the map."""
    model = Model(shape, wall_mask, M, tau1)
    d = torch.tensor(np.asarray(d_pairs, dtype=np.float64), requires_grad=True)
    gt = torch.tensor(np.asarray(g, dtype=np.float64)[:2], requires_grad=True)
    L = model.loss(x0, n0, nsteps, target, d, gt)
    dd, dg = torch.autograd.grad(L, (d, gt))
    return float(L.detach()), dd.numpy().copy(), dg.numpy().copy()
