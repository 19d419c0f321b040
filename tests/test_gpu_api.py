"""Behaviour of the C ABI on the GPU: state machine and errors, caller-owned
buffers, device-array readouts, reproducibility, the FP64 mass correction of
the reduced-precision paths, and the device error flag."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2504_07059_gb300 import workloads as W
from parity_utils import gpu_run, max_rel, oracle_run

pytestmark = pytest.mark.gpu


def _small(lattice=W.D2Q9):
    if lattice == W.D2Q9:
        return W.random_mixture(W.D2Q9, (23, 19), W.WALL_Y, (2.0, 28.0, 44.0), g=(1e-5, -3e-5), stream=200)
    return W.random_mixture(W.D3Q19, (9, 8, 7), W.WALL_X | W.WALL_Y | W.WALL_Z, (16.0, 28.0, 44.0),
                            g=(0, -2e-5, 1e-5), stream=210)


def test_step_before_fields_is_a_state_error(evd):
    wl = _small()
    sim = evd.Simulation(wl.lattice, wl.shape, wl.wall_mask, wl.M, wl.D, wl.tau1, wl.g, "fp64")
    with pytest.raises(evd.EVDError) as ei:
        sim.step(1)
    assert ei.value.status == evd.EVD_ERR_STATE
    with pytest.raises(evd.EVDError):
        sim.mole_fractions()
    sim.set_fields(wl.x)
    sim.step(0)
    assert sim.t == 0
    with pytest.raises(evd.EVDError) as ei:
        evd.evd_step(sim.ctx, -1)
    assert ei.value.status == evd.EVD_ERR_ARG
    bad = wl.x.copy()
    bad[0, 0, 0, 0] = 0.0
    with pytest.raises(evd.EVDError) as ei:
        sim.set_fields(bad)
    assert ei.value.status == evd.EVD_ERR_ARG
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
def test_runs_are_bitwise_reproducible(evd, precision):
    wl = _small(W.D3Q19)
    a = gpu_run(evd, wl, 30, precision)
    b = gpu_run(evd, wl, 30, precision)
    assert np.array_equal(a.populations(), b.populations())
    assert np.array_equal(a.species_mass(), b.species_mass())


def test_set_populations_round_trip_and_step(evd):
    wl = _small()
    o = oracle_run(wl, 7)
    f7 = o.get_f()
    sim = evd.Simulation(wl.lattice, wl.shape, wl.wall_mask, wl.M, wl.D, wl.tau1, wl.g, "fp64")
    sim.set_populations(f7)
    assert np.array_equal(sim.populations(), f7)
    o.step(5)
    sim.step(5)
    assert max_rel(sim.populations(), o.get_f()) < 1e-12
    sim.close()


def test_caller_owned_buffers_and_device_readout(evd):
    torch = pytest.importorskip("torch")
    wl = _small(W.D3Q19)
    dev = torch.device("cuda", 0)
    grid = evd.make_grid(wl.lattice, evd.EVD_FP32, wl.shape, wl.wall_mask)
    sp = evd.SpeciesTable(wl.M, wl.D, wl.tau1, wl.g)
    nbytes = evd.evd_required_bytes(grid, sp)
    bufa = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    bufb = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(dev)
    ctx = evd.evd_create_with_buffers(grid, sp, stream, bufa, bufb, nbytes)
    x_dev = torch.from_numpy(np.ascontiguousarray(wl.x)).to(dev)
    torch.cuda.synchronize(dev)
    evd.evd_set_fields_device(ctx, x_dev, None)
    evd.evd_step(ctx, 20)
    xo = torch.empty_like(x_dev)
    rho = torch.empty_like(x_dev)
    u = torch.empty((3,) + tuple(x_dev.shape[1:]), dtype=torch.float64, device=dev)
    ui = torch.empty((3, 3) + tuple(x_dev.shape[1:]), dtype=torch.float64, device=dev)
    m = torch.empty(3, dtype=torch.float64, device=dev)
    evd.evd_readout_device(ctx, xo, rho, u, ui)
    evd.evd_species_mass_device(ctx, m)
    stream.synchronize()
    evd.evd_check(ctx)
    o = oracle_run(wl, 20)
    ob = o.observables()
    assert np.abs(xo.cpu().numpy() - ob["x"]).max() < 2e-5
    assert max_rel(rho.cpu().numpy(), ob["rho"]) < 2e-5
    assert np.abs(u.cpu().numpy() - ob["u"]).max() < 1e-6
    assert max_rel(m.cpu().numpy(), o.mass()) < 1e-6
    # a second context on the same buffers sizes is independent
    with pytest.raises(evd.EVDError):
        evd.evd_create_with_buffers(grid, sp, stream, bufa, bufa, nbytes)
    evd.evd_destroy(ctx)


def test_reduced_precision_mass_correction_holds_mass(evd):
    """Without the FP64 correction the FP32 interpolation drifts the species
    mass by roundoff each step; with it the drift stays below 1e-6."""
    wl = W.loschmidt_binary()
    m0 = np.array([(wl.x[i] * wl.M[i]).sum() for i in range(2)])
    drifts = {}
    for every in (0, 8):
        sim = evd.Simulation.from_workload(wl, "fp32")
        evd.evd_set_mass_correction(sim.ctx, every)
        target = np.empty(2)
        evd.evd_get_target_mass(sim.ctx, target)
        assert max_rel(target, m0) < 1e-14
        sim.step(2000)
        drifts[every] = max_rel(sim.species_mass(), m0)
        sim.close()
    assert drifts[8] < 1e-6, drifts
    assert drifts[8] <= drifts[0], drifts


def test_instability_sets_the_error_flag_without_faulting(evd):
    # a body force far beyond the lattice's range drives densities negative;
    # the kernels flag it and the context stays usable
    wl = W.random_mixture(W.D2Q9, (8, 12), W.WALL_Y, (1.0, 4.0), g=(0.0, -0.5), stream=300)
    sim = evd.Simulation.from_workload(wl, "fp64")
    sim.step(200)
    with pytest.raises(evd.EVDError) as ei:
        sim.check()
    assert ei.value.status == evd.EVD_ERR_UNSTABLE
    assert "unstable" in evd.evd_last_error(sim.ctx)
    # fresh fields clear the flag (evd_set_fields checks it before returning)
    sim.set_fields(wl.x)
    sim.check()
    assert sim.t == 0
    sim.close()


def test_launch_count_accounts_for_every_kernel(evd):
    wl = _small()
    sim = evd.Simulation.from_workload(wl, "fp32")
    evd.evd_set_mass_correction(sim.ctx, 4)
    n0 = evd.evd_launch_count(sim.ctx)
    sim.step(16)
    # 16 step kernels + 4 mass-correction reductions
    assert evd.evd_launch_count(sim.ctx) - n0 == 20
    sim.close()


def test_fma_rate_measures_the_arithmetic_roofs(evd):
    """evd_fma_rate (the FMA chains behind the bench's arithmetic roofs):
    positive rates, double below float by the GPU's FP64 ratio, and the
    counted operations those of the launch (2 per FMA, 8 chains, 8 blocks of
    256 threads per SM)."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    rates = {}
    for kind in (0, 1, 2):
        flops, ms = evd.evd_fma_rate(kind, 1 << 12)
        per_thread = 2 * 8 * (1 << 12) * (2 if kind == 2 else 1)
        assert flops == per_thread * 8 * 256 * sms
        assert ms > 0.0
        rates[kind] = flops / ms
    assert rates[1] > 8 * rates[0]
