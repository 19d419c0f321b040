"""The batch of independent lattices (include/evd_batch.h) on the GPU: every
member against the FP64 oracle run alone, the batch against the single-lattice
path, and the schedule, graph and autotuner leaving the results unchanged."""
import numpy as np
import pytest

from paper_2504_07059_gb300 import workloads as W
from parity_utils import TOL_MASS, TOL_X, gpu_run, max_rel, oracle_run

pytestmark = pytest.mark.gpu

WY = W.WALL_Y
WXY = W.WALL_X | W.WALL_Y


def mixed_d2q9():
    """Uneven members: sizes (ragged, one row, one column), 1-3 species,
    walls and periodic sides, gravity, a number-density field."""
    return [
        W.random_mixture(W.D2Q9, (32, 45), WY, (1.0, 4.0), g=(0, -3e-6), stream=200),
        W.random_mixture(W.D2Q9, (17, 13), WXY, (1.0, 3.0, 7.0), g=(1e-5, -2e-5), stream=210, n_amp=0.1),
        W.random_mixture(W.D2Q9, (24, 1), 0, (1.0, 5.0), g=(1e-5, 0), stream=220),
        W.random_mixture(W.D2Q9, (1, 16), WXY, (2.0,), g=(0, -1e-4), stream=230),
        W.random_mixture(W.D2Q9, (9, 130), WY, (2.0, 28.0, 44.0), g=(0, -1e-6), stream=240),
        W.loschmidt_binary(nx=4, ny=64),
    ]


def mixed_d3q19():
    return [
        W.random_mixture(W.D3Q19, (11, 9, 7), W.WALL_X | W.WALL_Y | W.WALL_Z, (16.0, 28.0, 44.0),
                         g=(1e-5, -2e-5, 3e-5), stream=300),
        W.random_mixture(W.D3Q19, (13, 6, 5), W.WALL_Y | W.WALL_Z, (1.0, 3.0), g=(3e-5, 0, 0), stream=310),
        W.random_mixture(W.D3Q19, (7, 5, 1), 0, (2.0, 3.0, 5.0), stream=320),
    ]


def batch_run(evd, members, steps, precision, schedule=None, graph=None, mc=None):
    b = evd.Batch(members, precision)
    if schedule:
        evd.evd_batch_set_schedule(b.b, *schedule)
    if mc is not None:
        evd.evd_batch_set_mass_correction(b.b, mc)
    if graph is not None:
        evd.evd_batch_set_graph(b.b, graph)
    b.set_fields([m.x for m in members], [m.n for m in members])
    b.step(steps)
    return b


@pytest.mark.parametrize("lattice,steps", [("d2q9", 40), ("d3q19", 12)])
def test_fp64_members_match_the_oracle_on_every_field(evd, lattice, steps):
    members = mixed_d2q9() if lattice == "d2q9" else mixed_d3q19()
    b = batch_run(evd, members, steps, "fp64")
    assert b.t == steps
    xs, rhos = b.mole_fractions(), b.densities()
    us, uis = b.velocities()
    ms = b.species_mass()
    for k, m in enumerate(members):
        o = oracle_run(m, steps)
        ob = o.observables()
        assert max_rel(xs[k], ob["x"]) < 1e-12, (k, "x")
        assert max_rel(rhos[k], ob["rho"]) < 1e-12, (k, "rho")
        D = b.D
        for name, a, ref in (("u", us[k], ob["u"][:D]), ("ui", uis[k], ob["ui"][:, :D])):
            err = float(np.abs(a - ref).max()) / max(float(np.abs(ref).max()), 1e-3)
            assert err < 1e-12, (k, name, err)
        assert max_rel(ms[k], o.mass()) < 1e-12, (k, "mass")
    b.close()


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_reduced_precision_members_match_the_oracle(evd, precision):
    members = mixed_d2q9()
    steps = 200
    b = batch_run(evd, members, steps, precision)
    xs, ms = b.mole_fractions(), b.species_mass()
    for k, m in enumerate(members):
        m0 = np.array([(m.x[i] * m.M[i] * (1.0 if m.n is None else m.n)).sum() for i in range(m.ns)])
        assert max_rel(ms[k], m0) < TOL_MASS[precision], k
        o = oracle_run(m, steps)
        assert np.abs(xs[k] - o.observables()["x"]).max() < TOL_X[precision], k
    b.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_agrees_with_the_single_lattice_step(evd, precision):
    """Same per-node arithmetic as the general single-lattice kernel (mass
    correction off): the two are compiled separately, so the compiler may fuse
    different multiply-adds; in FP32 both store the node-reference encoding
    with the same per-step dither seeds, so agreement is to rounding (a value
    within rounding of a dither threshold may round the other way: one unit
    in the last place of FP32 storage)."""
    members = mixed_d2q9()
    steps = 30
    b = batch_run(evd, members, steps, precision, mc=0)
    xs = b.mole_fractions()
    for k, m in enumerate(members):
        sim = evd.Simulation(m.lattice, m.shape, m.wall_mask, m.M, m.D, m.tau1, m.g, precision)
        evd.evd_set_kernel(sim.ctx, evd.EVD_KERNEL_GENERAL)
        evd.evd_set_mass_correction(sim.ctx, 0)
        if precision == "fp32":
            evd.evd_set_reference_mode(sim.ctx, evd.EVD_REF_NODE)
        sim.set_fields(m.x, m.n)
        sim.step(steps)
        tol = 1e-13 if precision == "fp64" else 1e-6
        assert np.abs(xs[k] - sim.mole_fractions()).max() < tol, k
        sim.close()
    b.close()


def test_schedule_and_graph_do_not_change_results(evd):
    members = mixed_d2q9()
    steps = 37   # not a multiple of the graph length
    ref = batch_run(evd, members, steps, "fp32", schedule=(128, 0), graph=0, mc=0)
    xr = ref.mole_fractions()
    for sched, graph in [((256, 2), 8), ((2048, 16), 16), ((512, 4), 2), ((128, 1), 0)]:
        b = batch_run(evd, members, steps, "fp32", schedule=sched, graph=graph, mc=0)
        for a, r in zip(b.mole_fractions(), xr):
            assert np.array_equal(a, r), (sched, graph)
        b.close()
    # with the mass correction on, graph replay and direct launches agree
    # bitwise for one schedule
    a = batch_run(evd, members, 64, "fp32", schedule=(256, 4), graph=0)
    g = batch_run(evd, members, 64, "fp32", schedule=(256, 4), graph=16)
    for p, q in zip(a.mole_fractions(), g.mole_fractions()):
        assert np.array_equal(p, q)
    for p, q in zip(a.species_mass(), g.species_mass()):
        assert np.array_equal(p, q)
    ref.close(), a.close(), g.close()


def test_autotune_restores_the_state_and_keeps_a_valid_schedule(evd):
    members = mixed_d2q9()
    a = batch_run(evd, members, 10, "fp32", mc=0)
    b = batch_run(evd, members, 10, "fp32", mc=0)
    item, ctas = evd.evd_batch_autotune(b.b, 4)
    assert item in (128, 256, 512, 1024, 2048) and ctas in (0, 2, 4, 8, 16)
    assert evd.evd_batch_get_schedule(b.b) == (item, ctas)
    assert b.t == 10
    a.step(20)
    b.step(20)
    for p, q in zip(a.mole_fractions(), b.mole_fractions()):
        assert np.array_equal(p, q)
    a.close(), b.close()


def test_launch_count_and_time(evd):
    members = mixed_d2q9()
    b = batch_run(evd, members, 0, "fp32")
    n0 = evd.evd_batch_launch_count(b.b)
    b.step(40)    # 40 steps, mass correction every 8 steps: 5 reductions
    assert b.t == 40
    assert evd.evd_batch_launch_count(b.b) - n0 == 45
    b.close()


def test_an_unstable_member_is_reported(evd):
    members = mixed_d2q9()[:2]
    bad = W.random_mixture(W.D2Q9, (8, 8), WY, (1.0, 2.0), g=(0, -0.5), stream=250)
    b = evd.Batch(members + [bad], "fp64")
    b.set_fields([m.x for m in members + [bad]], [m.n for m in members + [bad]])
    b.step(50)
    with pytest.raises(evd.EVDError) as ei:
        b.check()
    assert ei.value.status == evd.EVD_ERR_UNSTABLE
    b.close()


def test_tube_sweep_at_full_size_sampled_members(evd):
    """The 512-tube sweep in the launch configuration the benchmark times
    (FP32, graph replay, mass correction): sampled members against the oracle
    run alone (shortest, longest, largest mass ratio among the ternaries)."""
    tubes = W.batched_tubes()
    k = 16
    b = evd.Batch(tubes, "fp32")
    b.set_fields([t.x for t in tubes])
    b.step(k)
    b.check()
    xs = b.mole_fractions()
    lengths = [t.shape[1] for t in tubes]
    tern = [i for i, t in enumerate(tubes) if t.ns == 3]
    picks = {int(np.argmin(lengths)), int(np.argmax(lengths)), max(tern, key=lambda i: tubes[i].M[-1])}
    for i in sorted(picks):
        o = oracle_run(tubes[i], k)
        assert np.abs(xs[i] - o.observables()["x"]).max() < TOL_X["fp32"], i
    ms = b.species_mass()
    for i in (0, 100, 511):
        t = tubes[i]
        m0 = np.array([(t.x[s] * t.M[s]).sum() for s in range(t.ns)])
        assert max_rel(ms[i], m0) < TOL_MASS["fp32"], i
    b.close()
