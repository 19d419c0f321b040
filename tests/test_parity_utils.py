"""The sampled-window construction used for full-size parity is exact: the
oracle on a window reproduces the oracle on the full grid at the centre."""
import numpy as np
import pytest

from paper_2504_07059_gb300 import workloads as W
from parity_utils import oracle_run, window


@pytest.mark.parametrize("lattice,shape,mask", [
    (W.D3Q19, (12, 11, 10), W.WALL_X | W.WALL_Y | W.WALL_Z),
    (W.D3Q19, (12, 11, 10), W.WALL_Y),
    (W.D2Q9, (15, 14, 1), W.WALL_Y)])
def test_window_reproduces_full_grid(lattice, shape, mask):
    M = (16.0, 28.0, 44.0)
    wl = W.random_mixture(lattice, shape, mask, M, g=(1e-5, -2e-5, 1e-5 if lattice else 0.0))
    k = 2
    full = oracle_run(wl, k).observables()["x"]
    nz = shape[2]
    for c in [(0, 0, 0), (11, 10, nz - 1), (5, 0, nz // 2), (6, 5, min(4, nz - 1)), (11, 3, 0)]:
        c = (min(c[0], shape[0] - 1), min(c[1], shape[1] - 1), min(c[2], nz - 1))
        sub, loc = window(wl, c, k)
        xs = oracle_run(sub, k).observables()["x"]
        np.testing.assert_allclose(xs[:, loc[2], loc[1], loc[0]], full[:, c[2], c[1], c[0]], rtol=1e-13)
