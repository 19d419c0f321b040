"""The C-ABI library on the CPU: it builds for sm_103a, loads without a GPU,
exports every entry point include/evd.h declares, and validates arguments
before touching the device."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(evd_\w+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(evd):
    names = declared_functions()
    assert len(names) >= 20
    L = evd.lib()
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(evd._SIGNATURES), "binding and header disagree"


def test_version_and_required_bytes(evd):
    assert evd.evd_version() == 1
    sp = evd.SpeciesTable([2.0, 28.0, 44.0], np.full((3, 3), 0.05), 1.0, (0, -1e-6, 0))
    g = evd.make_grid(evd.EVD_D2Q9, evd.EVD_FP32, (64, 1024), evd.EVD_WALL_YM | evd.EVD_WALL_YP)
    assert evd.evd_required_bytes(g, sp) == 64 * 1024 * 27 * 4
    g3 = evd.make_grid(evd.EVD_D3Q19, evd.EVD_FP16_STORE, (5, 7, 3), 0)
    # planes padded to 64 elements: 105 sites -> 128; half storage keeps one
    # node-density plane per species besides the 57 population planes
    assert evd.evd_required_bytes(g3, sp) == 128 * (57 + 3) * 2


@pytest.mark.parametrize("bad", [
    dict(lattice=7), dict(precision=9), dict(nz=2), dict(nx=0), dict(wall_mask=0b000100),
    dict(M=[2.0, 1.0]), dict(M=[1.0, -2.0]), dict(tau1=0.5), dict(D=[[0, 0.05], [0.07, 0]]),
    dict(D=[[0, -1.0], [-1.0, 0]]), dict(g=(0, 0, 1e-6)), dict(M=[1.0, 2.0, 3.0, 4.0, 5.0, 6.0, 7.0]),
    dict(lattice=1, nz=2, M=[1.0, 2.0, 3.0, 4.0]), dict(wall_mask=0b010000)])
def test_invalid_configurations_are_rejected_before_any_cuda_call(evd, bad):
    M = bad.get("M", [1.0, 2.0])
    ns = len(M)
    D = bad.get("D", np.full((ns, ns), 0.05))
    sp = evd.SpeciesTable(M, D, bad.get("tau1", 1.0), bad.get("g", (0, 0, 0)))
    g = evd.evd_grid(bad.get("lattice", 0), bad.get("precision", 0), bad.get("nx", 4), 8,
                     bad.get("nz", 1), bad.get("wall_mask", 0))
    assert evd.evd_required_bytes(g, sp) == 0
    with pytest.raises(evd.EVDError) as ei:
        evd.evd_create(g, sp)
    assert ei.value.status == evd.EVD_ERR_ARG
    assert evd.evd_last_error(None)


def test_null_context_calls_fail_cleanly(evd):
    L = evd.lib()
    assert L.evd_step(None, 1) == evd.EVD_ERR_ARG
    assert L.evd_check(None) == evd.EVD_ERR_ARG
    assert L.evd_destroy(None) == evd.EVD_OK
    assert L.evd_time(None) == -1
    assert L.evd_launch_count(None) == -1
    assert L.evd_set_mass_correction(None, 4) == evd.EVD_ERR_ARG
    assert L.evd_set_adjoint_mode(None, evd.EVD_ADJOINT_DUAL) == evd.EVD_ERR_ARG


def test_batch_rejects_invalid_members_before_any_cuda_call(evd):
    good = evd.SpeciesTable([1.0, 2.0], np.full((2, 2), 0.05), 1.0)
    bad = evd.SpeciesTable([2.0, 1.0], np.full((2, 2), 0.05), 1.0)   # decreasing masses
    arr = (evd.evd_member * 2)(evd.evd_member(8, 8, 1, 0, good.struct), evd.evd_member(8, 8, 1, 0, bad.struct))
    with pytest.raises(evd.EVDError) as ei:
        evd.evd_batch_create(evd.EVD_D2Q9, evd.EVD_FP32, arr)
    assert ei.value.status == evd.EVD_ERR_ARG
    assert "member 1" in evd.evd_batch_last_error(None)
    with pytest.raises(evd.EVDError):
        evd.evd_batch_create(evd.EVD_D2Q9, 7, arr)
    with pytest.raises(evd.EVDError):
        evd.evd_batch_create(evd.EVD_D2Q9, evd.EVD_FP32, (evd.evd_member * 0)())


def test_null_batch_calls_fail_cleanly(evd):
    L = evd.lib()
    assert L.evd_batch_step(None, 1) == evd.EVD_ERR_ARG
    assert L.evd_batch_check(None) == evd.EVD_ERR_ARG
    assert L.evd_batch_set_schedule(None, 128, 0) == evd.EVD_ERR_ARG
    assert L.evd_batch_time(None) == -1 and L.evd_batch_launch_count(None) == -1
    assert L.evd_batch_destroy(None) == evd.EVD_OK


def test_corrective_forcing_flags_are_checked(evd):
    sp3 = evd.SpeciesTable([1.0, 2.0], np.full((2, 2), 0.05), 1.0, flags=evd.EVD_FORCE_S_P)
    g3 = evd.make_grid(evd.EVD_D3Q19, evd.EVD_FP64, (4, 4, 4), 0)
    with pytest.raises(evd.EVDError) as ei:           # D2Q9 only
        evd.evd_create(g3, sp3)
    assert ei.value.status == evd.EVD_ERR_ARG and "D2Q9" in evd.evd_last_error(None)
    bad = evd.SpeciesTable([1.0, 2.0], np.full((2, 2), 0.05), 1.0, flags=8)
    g2 = evd.make_grid(evd.EVD_D2Q9, evd.EVD_FP64, (4, 4), 0)
    with pytest.raises(evd.EVDError):
        evd.evd_create(g2, bad)
    arr = (evd.evd_member * 1)(evd.evd_member(4, 4, 1, 0, evd.SpeciesTable([1.0, 2.0], np.full((2, 2), 0.05), 1.0,
                                                                           flags=evd.EVD_FORCE_S_DIFF).struct))
    with pytest.raises(evd.EVDError):
        evd.evd_batch_create(evd.EVD_D2Q9, evd.EVD_FP64, arr)


def test_species_limits_per_lattice(evd):
    """Up to six species on D2Q9 (dense solve of the tau_ij system), three on
    D3Q19; the corrective terms take three at most."""
    for ns in range(1, 7):
        M = [1.0 + k for k in range(ns)]
        sp = evd.SpeciesTable(M, np.full((ns, ns), 0.05), 1.0)
        g2 = evd.make_grid(evd.EVD_D2Q9, evd.EVD_FP64, (6, 8), 0)
        assert evd.evd_required_bytes(g2, sp) == 64 * ns * 9 * 8
        g3 = evd.make_grid(evd.EVD_D3Q19, evd.EVD_FP32, (4, 4, 4), 0)
        assert (evd.evd_required_bytes(g3, sp) > 0) == (ns <= 3)
    M = [1.0, 2.0, 3.0, 4.0]
    sp = evd.SpeciesTable(M, np.full((4, 4), 0.05), 1.0, flags=evd.EVD_FORCE_S_DIFF)
    assert evd.evd_required_bytes(evd.make_grid(evd.EVD_D2Q9, evd.EVD_FP64, (6, 8), 0), sp) == 0


def test_fma_rate_validates_its_arguments_before_any_cuda_call(evd):
    """The arithmetic-roof microbenchmark rejects an unknown kind and an
    iteration count out of range with EVD_ERR_ARG (no device needed)."""
    for kind, iters in ((3, 16), (-1, 16), (0, 0), (1, 1 << 25)):
        with pytest.raises(evd.EVDError) as ei:
            evd.evd_fma_rate(kind, iters)
        assert ei.value.status == evd.EVD_ERR_ARG
