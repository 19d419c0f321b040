"""The seeded input generators shared by the oracle and the CUDA path."""
import os

import numpy as np

from paper_2504_07059_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_vectors.txt")


def test_splitmix64_reference_vectors():
    rows = [ln.split() for ln in open(GOLDEN) if ln.strip() and not ln.startswith("#")]
    assert rows
    for seed, k, hexval in rows:
        got = W.splitmix64(0, int(k) + 1, seed=int(seed))[int(k)]
        assert int(got) == int(hexval, 16)


def test_generators_are_deterministic_and_valid():
    a = W.loschmidt_ternary_gravity(nx=8, ny=32)
    b = W.loschmidt_ternary_gravity(nx=8, ny=32)
    assert np.array_equal(a.x, b.x) and np.array_equal(a.D, b.D)
    for wl in (a, W.loschmidt_binary(), W.stratification_3d(n=8),
               W.random_mixture(1, (5, 4, 3), W.WALL_Z, (1.0, 2.0, 3.0), n_amp=0.1)):
        assert wl.x.shape == (wl.ns,) + tuple(reversed(wl.shape))
        assert np.allclose(wl.x.sum(axis=0), 1.0, atol=1e-15)
        assert np.all(wl.x > 0)
        assert np.allclose(wl.D, wl.D.T) and np.all(np.diag(wl.D) == 0)
        assert list(wl.M) == sorted(wl.M)


def test_paper_gases_fill_the_tube_halves():
    wl = W.loschmidt_ternary_gravity(nx=4, ny=64)
    # gas B (H2 rich) below, gas A (Ar rich) above, within the 1% noise, away
    # from the smoothed interface between rows 31 and 32
    assert np.all(np.abs(wl.x[0, 0, :16] / 0.8 - 1) < 0.011)
    assert np.all(np.abs(wl.x[2, 0, 48:] / 0.7 - 1) < 0.011)
    # the interface is monotone and centred
    assert np.all(np.diff(wl.x[2, 0, 26:38, 0]) > 0)
    assert abs(wl.x[2, 0, 31, 0] + wl.x[2, 0, 32, 0] - (0.7 + 0.001)) < 0.02
    assert np.all((wl.D[np.triu_indices(3, 1)] >= 0.02) & (wl.D[np.triu_indices(3, 1)] <= 0.1))


def test_batched_tube_sweep_draws_the_stated_ranges():
    tubes = W.batched_tubes()
    assert len(tubes) == 512
    again = W.batched_tubes(count=3)
    for a, b in zip(tubes[:3], again):
        assert a.shape == b.shape and a.M == b.M and np.array_equal(a.D, b.D) and a.g == b.g
    lengths = np.array([t.shape[1] for t in tubes])
    assert lengths.min() >= 128 and lengths.max() <= 4096
    # log-uniform: the median length is near sqrt(128 * 4096) = 724
    assert 550 < np.median(lengths) < 950
    ns = np.array([t.ns for t in tubes])
    assert set(ns) == {2, 3} and 0.4 < (ns == 3).mean() < 0.6
    for t in tubes:
        assert t.shape[0] == 32 and t.shape[2] == 1 and t.wall_mask == W.WALL_Y
        assert t.M[0] == 1.0 and list(t.M) == sorted(t.M) and t.M[-1] <= 10.0
        off = t.D[np.triu_indices(t.ns, 1)]
        assert off.min() >= (0.01 if t.ns == 2 else 0.06) and off.max() <= 0.1
        assert t.g[0] == 0.0 and -5e-6 <= t.g[1] <= 0.0 and t.g[2] == 0.0
        assert np.allclose(t.x.sum(axis=0), 1.0, atol=1e-15)
        L = t.shape[1]
        below, above = t.x[:, 0, L // 2 - 1, 0], t.x[:, 0, L // 2, 0]
        assert np.allclose(below, W.TUBE_BELOW[t.ns]) and np.allclose(above, W.TUBE_ABOVE[t.ns])
    # 19.3 M sites, 48.1 M species-site updates per step
    assert 18e6 < sum(t.nsites for t in tubes) < 21e6
