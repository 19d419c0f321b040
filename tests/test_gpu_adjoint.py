"""The discrete adjoint (evd_loss_gradient, D2Q9 FP64) against the oracle's
own discrete adjoint (reverse mode through the oracle's map) and against
central finite differences of the FP64 oracle's loss (independent code), the
loss itself against the oracle, checkpoint invariance, and the
torch.autograd wrapper."""
import numpy as np
import pytest

from oracle import discrete_adjoint as DA
from oracle import oracle as O
from paper_2504_07059_gb300 import adjoint as ADJ
from paper_2504_07059_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def oracle_loss(prob: ADJ.Problem, d_pairs, g):
    ns = len(prob.molar_mass)
    o = O.Oracle(W.D2Q9, prob.shape, prob.wall_mask, prob.molar_mass, ADJ.pairs_to_matrix(ns, d_pairs),
                 prob.tau1, (g[0], g[1]))
    o.init(prob.x0, prob.n0)
    o.step(prob.nsteps)
    xbar = o.observables()["x"][:, 0].mean(axis=2)
    return float(((xbar - prob.target) ** 2).sum())


def make_problem(shape, walls, M, d_pairs, g, steps, stream):
    """A seeded mixture and a target profile: the oracle's row averages after
    the same number of steps with every parameter perturbed (the recipe of the
    inverse problem: D x 1.1, g x 0.9)."""
    wl = W.random_mixture(W.D2Q9, shape, walls, M, stream=stream)
    prob = ADJ.Problem(shape, walls, tuple(M), 1.0, wl.x, np.zeros((len(M), shape[1])), steps)
    ns = len(M)
    o = O.Oracle(W.D2Q9, shape, walls, M, ADJ.pairs_to_matrix(ns, 1.1 * np.asarray(d_pairs)), 1.0,
                 (0.9 * g[0], 0.9 * g[1]))
    o.init(wl.x)
    o.step(steps)
    prob.target = o.observables()["x"][:, 0].mean(axis=2)
    return prob


CASES = {
    "ternary-walls-y": (lambda: make_problem((10, 24), W.WALL_Y, (1.0, 3.0, 7.0), (0.06, 0.08, 0.07),
                                             (2e-6, -1e-5), 40, 1400), (0.06, 0.08, 0.07), (2e-6, -1e-5)),
    "binary-closed-box": (lambda: make_problem((8, 12), W.WALL_X | W.WALL_Y, (1.0, 2.5), (0.05,),
                                               (1e-5, -2e-5), 30, 1410), (0.05,), (1e-5, -2e-5)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_adjoint_gradient_matches_central_differences_of_the_oracle(evd, name):
    """Every component within 1e-4 relative of the oracle's finite differences:
    central differences with h = 1e-4 |theta_k| for the diffusivities
    (observed 7e-8 to 1e-7: the h^2 truncation); for the body force, whose
    loss derivative can be small enough that differences at that step are
    roundoff-limited, a fourth-order difference with h = 1e-2 |g_k| (observed
    <= 4e-6)."""
    make, d, g = CASES[name]
    prob = make()
    loss, dd, dg = ADJ.loss_and_gradient(prob, d, g)
    L0 = oracle_loss(prob, d, g)
    assert abs(loss - L0) <= 1e-10 * abs(L0), (loss, L0)
    theta = np.array(list(d) + list(g))
    adj = np.concatenate([dd, dg])
    nd = len(d)
    L = lambda t: oracle_loss(prob, t[:nd], t[nd:])
    fd = np.zeros_like(theta)
    for k in range(len(theta)):
        e = np.zeros_like(theta)
        if k < nd:
            e[k] = 1e-4 * abs(theta[k])
            fd[k] = (L(theta + e) - L(theta - e)) / (2 * e[k])
        else:
            e[k] = 1e-2 * abs(theta[k])
            fd[k] = (8 * (L(theta + e) - L(theta - e)) - (L(theta + 2 * e) - L(theta - 2 * e))) / (12 * e[k])
    assert np.all(np.abs(fd) > 0)
    rel = np.abs(adj - fd) / np.abs(fd)
    assert rel.max() < 1e-4, (rel, adj, fd)


@pytest.mark.parametrize("mode", ["reverse", "dual"])
@pytest.mark.parametrize("name", list(CASES))
def test_adjoint_gradient_matches_the_oracles_discrete_adjoint(evd, name, mode):
    """Both are the exact gradient of the same discrete map (the CUDA one by
    a hand-written reverse sweep, or dual-number Jacobians, and a transposed
    gather; the oracle's by reverse mode through its tensor restatement), so
    they differ by rounding only: 1e-9 relative per component, 1e-12 on the
    loss."""
    make, d, g = CASES[name]
    prob = make()
    prob.mode = evd.EVD_ADJOINT_REVERSE if mode == "reverse" else evd.EVD_ADJOINT_DUAL
    loss, dd, dg = ADJ.loss_and_gradient(prob, d, g)
    L, odd, odg = DA.loss_and_gradient(prob.shape, prob.wall_mask, prob.molar_mass, prob.tau1, prob.x0,
                                       prob.target, prob.nsteps, d, g, prob.n0)
    assert abs(loss - L) <= 1e-12 * L, (loss, L)
    ours, theirs = np.concatenate([dd, dg]), np.concatenate([odd, odg])
    assert np.all(np.abs(ours - theirs) <= 1e-9 * np.abs(theirs)), (ours, theirs)


@pytest.mark.parametrize("name", list(CASES))
def test_reverse_and_dual_modes_agree(evd, name):
    """The hand-written reverse sweep against the dual-number Jacobian of the
    step's own collision code: the same products, summed in another order.
    Normwise, to 1e-12 of the largest component: a component that is small
    through cancellation (g_x here, 3e-4 of the largest) carries the rounding
    of the large terms it cancels (observed 4.6e-12 of itself)."""
    make, d, g = CASES[name]
    prob = make()
    out = []
    for mode in (evd.EVD_ADJOINT_REVERSE, evd.EVD_ADJOINT_DUAL):
        prob.mode = mode
        out.append(ADJ.loss_and_gradient(prob, d, g))
    assert out[0][0] == out[1][0]
    a, b = np.concatenate(out[0][1:]), np.concatenate(out[1][1:])
    assert np.all(np.abs(a - b) <= 1e-12 * np.abs(b).max()), (a, b)


def test_checkpoint_interval_does_not_change_the_gradient(evd):
    make, d, g = CASES["ternary-walls-y"]
    prob = make()
    results = []
    for k in (1, 0, 7, prob.nsteps):
        prob.checkpoint_every = k
        results.append(ADJ.loss_and_gradient(prob, d, g))
    for r in results[1:]:
        assert r[0] == results[0][0]
        assert np.array_equal(r[1], results[0][1]) and np.array_equal(r[2], results[0][2])


def test_torch_autograd_function_returns_the_adjoint_gradient(evd):
    import torch
    make, d, g = CASES["binary-closed-box"]
    prob = make()
    dt = torch.tensor(d, dtype=torch.float64, requires_grad=True)
    gt = torch.tensor(g, dtype=torch.float64, requires_grad=True)
    loss = ADJ.MoleFractionMisfit.apply(dt, gt, prob)
    (2.0 * loss).backward()
    ref = ADJ.loss_and_gradient(prob, d, g)
    assert float(loss.detach()) == ref[0]
    assert np.allclose(dt.grad.numpy(), 2.0 * ref[1], rtol=0, atol=0)
    assert np.allclose(gt.grad.numpy(), 2.0 * ref[2], rtol=0, atol=0)


def test_adjoint_rejects_what_it_does_not_cover(evd):
    wl = W.random_mixture(W.D2Q9, (6, 6), W.WALL_Y, (1.0, 2.0), stream=1420)
    sim = evd.Simulation(wl.lattice, wl.shape, wl.wall_mask, wl.M, wl.D, wl.tau1, wl.g, "fp32")
    with pytest.raises(evd.EVDError) as ei:
        evd.evd_loss_gradient(sim.ctx, wl.x, np.zeros((2, 6)), 5)
    assert ei.value.status == evd.EVD_ERR_ARG
    with pytest.raises(evd.EVDError) as ei:
        evd.evd_set_adjoint_mode(sim.ctx, 7)
    assert ei.value.status == evd.EVD_ERR_ARG
    sim.close()


# ---------------------------------------------------------------- the inverse problem at full size
def gpu_loss(prob: ADJ.Problem, d_pairs, g, precision="fp64"):
    """The loss from the library's forward step alone (no adjoint code): FP64
    (or FP32) steps, mole fractions read back, L summed here."""
    from paper_2504_07059_gb300 import evd
    ns = len(prob.molar_mass)
    sim = evd.Simulation(evd.EVD_D2Q9, prob.shape, prob.wall_mask, prob.molar_mass,
                         ADJ.pairs_to_matrix(ns, d_pairs), prob.tau1, (float(g[0]), float(g[1])), precision)
    try:
        sim.set_fields(prob.x0, prob.n0)
        sim.step(prob.nsteps)
        xbar = sim.mole_fractions()[:, 0].mean(axis=2)
    finally:
        sim.close()
    return float(((xbar - prob.target) ** 2).sum())


def inverse_problem(steps):
    """The 128 x 512 ternary tube with gravity (M = 2/28/44); the target is
    the FP64 run with every diffusivity x 1.1 and the force x 0.9."""
    wl = W.loschmidt_ternary_gravity(nx=128, ny=512)
    d = [wl.D[0, 1], wl.D[0, 2], wl.D[1, 2]]
    g = (0.0, wl.g[1])
    prob = ADJ.Problem(wl.shape[:2], wl.wall_mask, wl.M, wl.tau1, wl.x, np.zeros((3, 512)), steps)
    from paper_2504_07059_gb300 import evd
    sim = evd.Simulation(evd.EVD_D2Q9, prob.shape, prob.wall_mask, prob.molar_mass,
                         ADJ.pairs_to_matrix(3, 1.1 * np.asarray(d)), prob.tau1, (0.0, 0.9 * g[1]), "fp64")
    sim.set_fields(prob.x0)
    sim.step(steps)
    prob.target = sim.mole_fractions()[:, 0].mean(axis=2)
    sim.close()
    return prob, d, g


def test_inverse_problem_gradient_against_central_differences_at_full_size(evd):
    """128 x 512, 2000 steps: every diffusivity component and g_y within 1e-4
    relative of central differences (h = 1e-4 |theta_k|) of the loss of the
    FP64 forward step (code independent of the adjoint)."""
    prob, d, g = inverse_problem(2000)
    loss, dd, dg = ADJ.loss_and_gradient(prob, d, g)
    assert abs(loss - gpu_loss(prob, d, g)) <= 1e-12 * loss
    for k in range(3):
        h = 1e-4 * d[k]
        dp, dm = list(d), list(d)
        dp[k] += h
        dm[k] -= h
        fd = (gpu_loss(prob, dp, g) - gpu_loss(prob, dm, g)) / (2 * h)
        assert abs(dd[k] - fd) <= 1e-4 * abs(fd), (k, dd[k], fd)
    h = 1e-4 * abs(g[1])
    fd = (gpu_loss(prob, d, (0.0, g[1] + h)) - gpu_loss(prob, d, (0.0, g[1] - h))) / (2 * h)
    assert abs(dg[1] - fd) <= 1e-4 * abs(fd), (dg[1], fd)


def test_adjoint_dot_product_along_seeded_directions(evd):
    """<grad L, v> against the directional central difference of the FP64
    forward loss along seeded unit directions v in (D12, D13, D23, g_y),
    scaled by the parameters: agreement within 1e-4 relative."""
    prob, d, g = inverse_problem(1000)
    loss, dd, dg = ADJ.loss_and_gradient(prob, d, g)
    theta = np.array(list(d) + [g[1]])
    grad = np.concatenate([dd, [dg[1]]])
    u = W.uniform01(1500, 8).reshape(2, 4) * 2.0 - 1.0
    for v in u:
        v = v / np.linalg.norm(v) * theta          # direction scaled by the parameters
        eps = 1e-4
        lp = gpu_loss(prob, list(theta[:3] + eps * v[:3]), (0.0, theta[3] + eps * v[3]))
        lm = gpu_loss(prob, list(theta[:3] - eps * v[:3]), (0.0, theta[3] - eps * v[3]))
        fd = (lp - lm) / (2 * eps)
        assert abs(float(grad @ v) - fd) <= 1e-4 * abs(fd), (float(grad @ v), fd)


def test_fp32_forward_gradient_against_the_fp64_adjoint(evd):
    """The FP32-forward mode (FP32 steps and recomputation, FP64 reverse
    sweep) on the 128 x 512 tube, 2000 steps: its loss and gradient against
    the FP64 adjoint's, normwise within 1e-3 relative (the FP32 trajectory's
    mole fractions stay within ~1e-6 of the FP64 ones at this horizon)."""
    prob, d, g = inverse_problem(2000)
    l64, dd64, dg64 = ADJ.loss_and_gradient(prob, d, g)
    prob.forward = "fp32"
    l32, dd32, dg32 = ADJ.loss_and_gradient(prob, d, g)
    g64 = np.concatenate([dd64, dg64[1:2]])
    g32 = np.concatenate([dd32, dg32[1:2]])
    assert abs(l32 - l64) <= 1e-3 * l64, (l32, l64)
    assert np.linalg.norm(g32 - g64) <= 1e-3 * np.linalg.norm(g64), (g32, g64)
