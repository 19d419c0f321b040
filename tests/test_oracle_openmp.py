"""The OpenMP build of the oracle (used to time it on every host core) runs
the same arithmetic as the serial build: the streaming tasks are the
direction pairs of a species, each summed in the serial order, and the node
collisions are independent.  Its populations are therefore bitwise the serial
ones, walls and periodic, D2Q9 and D3Q19."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2504_07059_gb300 import workloads as W

CASES = [
    W.random_mixture(W.D2Q9, (13, 17), W.WALL_Y, (2.0, 28.0, 44.0), g=(1e-5, -3e-5), stream=900),
    W.random_mixture(W.D2Q9, (9, 7), 0, (1.0, 3.0), g=(2e-5, 0.0), stream=901),
    W.random_mixture(W.D3Q19, (7, 6, 5), W.WALL_X | W.WALL_Y | W.WALL_Z, (16.0, 28.0, 44.0),
                     g=(1e-5, -2e-5, 3e-5), stream=902),
]


def _run(wl, steps):
    o = O.Oracle(wl.lattice, wl.shape, wl.wall_mask, wl.M, wl.D, wl.tau1, wl.g)
    o.init(wl.x, wl.n)
    o.step(steps)
    return o.get_f(), o.mass()


@pytest.mark.parametrize("k", range(len(CASES)))
def test_openmp_build_is_bitwise_the_serial_oracle(k):
    so = O.build_omp()
    if so is None:
        pytest.skip("no OpenMP in this compiler")
    wl = CASES[k]
    f_serial, m_serial = _run(wl, 12)
    assert O.threads() == 1
    with O.swapped_library(so):
        f_omp, m_omp = _run(wl, 12)
        assert O.threads() >= 1
    assert np.array_equal(f_serial, f_omp)
    assert np.array_equal(m_serial, m_omp)
