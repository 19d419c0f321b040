"""Pins of the oracle's own discrete adjoint (oracle/discrete_adjoint.py): its
forward map is the C oracle's step restated with PyTorch tensor operations,
so (1) its populations after N steps and its loss equal the C oracle's to
rounding; (2) its reverse-mode gradient equals fourth-order finite
differences of the C oracle's loss (independent code) to the differences'
own accuracy; (3) reverse mode equals forward mode along random directions
(the dot-product test <grad L, v> = dL(theta + s v)/ds).  Mistakes planted
in the restatement (the force ignored in the collision, the wall rule
reversed, one diffusivity cut off from the autograd graph) fail the pin that
guards them."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from oracle import discrete_adjoint as DA
from paper_2504_07059_gb300 import workloads as W


def pairs_to_matrix(ns, d_pairs):
    D = np.zeros((ns, ns))
    k = 0
    for i in range(ns):
        for j in range(i + 1, ns):
            D[i, j] = D[j, i] = d_pairs[k]
            k += 1
    return D


# name: shape, walls, M, D pairs, g, steps, seed stream, number-density amplitude
CASES = {
    "ternary-walls-y": ((10, 24), W.WALL_Y, (1.0, 3.0, 7.0), (0.06, 0.08, 0.07), (2e-6, -1e-5), 40, 1400, 0.0),
    "binary-closed-box": ((8, 12), W.WALL_X | W.WALL_Y, (1.0, 2.5), (0.05,), (1e-5, -2e-5), 30, 1410, 0.1),
    "ternary-periodic": ((9, 10), 0, (1.0, 2.0, 5.0), (0.03, 0.09, 0.05), (3e-6, 4e-6), 25, 1430, 0.0),
}


def setup(name):
    shape, walls, M, dp, g, steps, stream, n_amp = CASES[name]
    wl = W.random_mixture(W.D2Q9, shape, walls, M, stream=stream, n_amp=n_amp)
    n0 = None if wl.n is None else wl.n
    # a target unlike the initial profile: a linear ramp of each mole fraction
    ny, ns = shape[1], len(M)
    ramp = np.linspace(-1.0, 1.0, ny)
    target = np.array([1.0 / ns + 0.02 * (i - 1) * ramp for i in range(ns)])
    return shape, walls, M, dp, g, steps, wl, n0, target


def c_oracle_loss(shape, walls, M, x0, n0, steps, target, d_pairs, g):
    o = O.Oracle(W.D2Q9, shape, walls, M, pairs_to_matrix(len(M), d_pairs), 1.0, (g[0], g[1]))
    o.init(x0, n0)
    o.step(steps)
    xbar = o.observables()["x"][:, 0].mean(axis=2)
    return float(((xbar - target) ** 2).sum()), o


@pytest.mark.parametrize("name", list(CASES))
def test_forward_map_is_the_c_oracle(name):
    shape, walls, M, dp, g, steps, wl, n0, target = setup(name)
    L_c, o = c_oracle_loss(shape, walls, M, wl.x, n0, steps, target, dp, g)
    model = DA.Model(shape, walls, M, 1.0)
    f = model.run(wl.x, n0, steps, dp, g).numpy()
    fc = o.get_f()[:, :, 0]
    assert np.abs(f - fc).max() <= 2e-15 * np.abs(fc).max()
    L = float(model.loss(wl.x, n0, steps, target, dp, g))
    assert abs(L - L_c) <= 1e-13 * L_c


@pytest.mark.parametrize("name", list(CASES))
def test_gradient_matches_finite_differences_of_the_c_oracle(name):
    """Fourth-order differences with a step per component where truncation
    and roundoff balance: 1e-3 |D_ij| for the diffusivities, 0.3 |g_k| for
    the body force (L is nearly polynomial in g; at small steps the
    difference of a small g derivative is roundoff-limited)."""
    shape, walls, M, dp, g, steps, wl, n0, target = setup(name)
    L, dd, dg = DA.loss_and_gradient(shape, walls, M, 1.0, wl.x, target, steps, dp, g, n0)
    theta = np.array(list(dp) + list(g))
    adj = np.concatenate([dd, dg])
    nd = len(dp)
    Lc = lambda t: c_oracle_loss(shape, walls, M, wl.x, n0, steps, target, t[:nd], t[nd:])[0]
    fd = np.zeros_like(theta)
    for k in range(len(theta)):
        e = np.zeros_like(theta)
        e[k] = (1e-3 if k < nd else 0.3) * abs(theta[k])
        fd[k] = (8 * (Lc(theta + e) - Lc(theta - e)) - (Lc(theta + 2 * e) - Lc(theta - 2 * e))) / (12 * e[k])
    assert np.all(np.abs(fd) > 0)
    rel = np.abs(adj - fd) / np.abs(fd)
    assert rel[:nd].max() < 1e-8, rel
    assert rel[nd:].max() < 1e-6, rel


def test_reverse_mode_equals_forward_mode():
    """<grad L, v> (reverse) against the directional derivative (forward
    mode, torch.func.jvp) along three seeded directions."""
    shape, walls, M, dp, g, steps, wl, n0, target = setup("ternary-walls-y")
    steps = 12
    model = DA.Model(shape, walls, M, 1.0)
    theta = torch.tensor(list(dp) + list(g), dtype=torch.float64)
    nd = len(dp)
    loss = lambda t: model.loss(wl.x, n0, steps, target, t[:nd], t[nd:])
    t = theta.clone().requires_grad_(True)
    (grad,) = torch.autograd.grad(loss(t), t)
    scale = theta.abs()
    for s in range(3):
        v = torch.as_tensor(2.0 * W.uniform01(1440 + s, len(theta)) - 1.0) * scale
        _, dL = torch.func.jvp(loss, (theta,), (v,))
        assert abs(float(dL) - float(grad @ v)) <= 1e-12 * abs(float(dL)), (float(dL), float(grad @ v))


class _NoForceInCollision(DA.Model):
    """Planted mistake: the collision ignores the body force."""
    def collide(self, f, D, g):
        zero = [g[0] * 0.0, g[1] * 0.0]
        return super().collide(f, D, zero)


class _WallRuleReversed(DA.Model):
    """Planted mistake: weight crossing a wall is kept in the opposite
    direction when it heads away from the wall, and vice versa."""
    def _plan(self):
        plan = super()._plan()
        return [[[(w, dx, dy, free, into, keep) for (w, dx, dy, free, keep, into) in terms]
                 for terms in per_a] for per_a in plan]


class _DiffusivityDetached(DA.Model):
    """Planted mistake: tau_ij sees D_12 as a constant, so the forward map is
    exact but the gradient misses every path from D_12 through tau."""
    def tau_cross(self, rho, D):
        return super().tau_cross(rho, {k: (v.detach() if k in ((0, 1), (1, 0)) else v) for k, v in D.items()})


@pytest.mark.parametrize("mutant,pin", [(_NoForceInCollision, "forward"), (_WallRuleReversed, "forward"),
                                        (_DiffusivityDetached, "gradient")])
def test_planted_mistakes_fail_a_pin(monkeypatch, mutant, pin):
    """Each mistake planted in the tensor restatement fails the pin that
    guards it: the forward map against the C oracle, or the gradient against
    finite differences of the C oracle's loss."""
    shape, walls, M, dp, g, steps, wl, n0, target = setup("ternary-walls-y")
    m = mutant(shape, walls, M, 1.0)
    if pin == "forward":
        _, o = c_oracle_loss(shape, walls, M, wl.x, n0, steps, target, dp, g)
        f = m.run(wl.x, n0, steps, dp, g).numpy()
        fc = o.get_f()[:, :, 0]
        assert np.abs(f - fc).max() > 1e-6 * np.abs(fc).max()
    else:
        monkeypatch.setattr(DA, "Model", mutant)
        L, dd, dg = DA.loss_and_gradient(shape, walls, M, 1.0, wl.x, target, steps, dp, g, n0)
        L0, _ = c_oracle_loss(shape, walls, M, wl.x, n0, steps, target, dp, g)
        assert abs(L - L0) <= 1e-13 * L0            # the forward map is untouched
        k = 0
        e = np.zeros(len(dp))
        e[k] = 1e-3 * dp[k]
        Lc = lambda d: c_oracle_loss(shape, walls, M, wl.x, n0, steps, target, d, g)[0]
        dp_ = np.asarray(dp)
        fd = (8 * (Lc(dp_ + e) - Lc(dp_ - e)) - (Lc(dp_ + 2 * e) - Lc(dp_ - 2 * e))) / (12 * e[k])
        assert abs(dd[k] - fd) > 1e-3 * abs(fd)    # far outside the 1e-8 the pin allows
