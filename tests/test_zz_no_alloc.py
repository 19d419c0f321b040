"""The allocation-free species-mass entry point, for callers that cannot call
cudaMalloc (their device memory belongs to another allocator, or they must
avoid the synchronisation an allocation can cause).  It must agree with the
context's own mass readout, call after call, while sharing one static device
scratch array.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2504_07059_gb300 import workloads as W
from parity_utils import max_rel

pytestmark = pytest.mark.gpu


def test_no_alloc_mass_matches_the_context_mass_on_consecutive_calls(evd):
    torch = pytest.importorskip("torch")
    wl = W.random_mixture(W.D3Q19, (13, 11, 9), W.WALL_X | W.WALL_Y | W.WALL_Z, (16.0, 28.0, 44.0),
                          g=(0.0, -2e-5, 1e-5), stream=400)
    sim = evd.Simulation.from_workload(wl, "fp64")
    L = evd.lib()
    m_dev = torch.empty(3, dtype=torch.float64, device="cuda")
    for steps in (5, 7):                       # two calls in a row, different states
        sim.step(steps)
        f_dev = torch.from_numpy(sim.populations()).to("cuda")
        m_dev.fill_(-1.0)
        torch.cuda.synchronize()
        status = L.evd_population_mass_noalloc(f_dev.data_ptr(), 3, 19, wl.nsites, m_dev.data_ptr(), None)
        torch.cuda.synchronize()
        assert status == evd.EVD_OK, evd.evd_last_error(None)
        assert max_rel(m_dev.cpu().numpy(), sim.species_mass()) < 1e-12
    sim.close()


def test_no_alloc_mass_rejects_sizes_beyond_its_scratch(evd):
    torch = pytest.importorskip("torch")
    f = torch.ones(4 * 9 * 8, dtype=torch.float64, device="cuda")
    m = torch.empty(4, dtype=torch.float64, device="cuda")
    L = evd.lib()
    assert L.evd_population_mass_noalloc(f.data_ptr(), 4, 9, 8, m.data_ptr(), None) == evd.EVD_ERR_ARG
    assert "n_species" in evd.evd_last_error(None)
    assert L.evd_population_mass_noalloc(f.data_ptr(), 2, 7, 8, m.data_ptr(), None) == evd.EVD_ERR_ARG
    # a valid call on the same inputs still works afterwards
    evd.evd_population_mass_noalloc(f, 2, 9, 8, m)
    torch.cuda.synchronize()
    assert np.allclose(m[:2].cpu().numpy(), 72.0)
