"""The standard test set's generators (Sec. 3.5, Table modelspace): placement with a
minimum distance, centre-out numbering, and the four connectivity classes at their
two densities -- checked by brute force and by counting."""
import math

import numpy as np
import pytest

from paper_0908_3934_b300 import netgen


def _brute_knn(pos, j, k):
    d = np.sum((pos - pos[j]) ** 2, axis=1)
    d[j] = np.inf
    return set(np.argsort(d, kind="stable")[:k].tolist())


@pytest.mark.parametrize("dim", [2, 3])
def test_placement_keeps_the_minimum_distance_and_numbers_from_the_centre(dim):
    n = 300
    d_min = 0.5 * n ** (-1.0 / dim)
    pos = netgen.min_distance_placement(np.random.default_rng(1), n, dim, 1.0, d_min)
    diff = pos[:, None, :] - pos[None, :, :]
    dist = np.sqrt(np.sum(diff ** 2, axis=2)) + np.eye(n) * 10.0
    assert dist.min() >= d_min
    r = np.sqrt(np.sum((pos - 0.5) ** 2, axis=1))
    assert np.all(np.diff(r) >= 0.0) and np.all((pos >= 0.0) & (pos < 1.0))


@pytest.mark.parametrize("density,k", [("low", 3), ("high", 8)])
def test_lattice_takes_the_k_nearest_vertices(density, k):
    sp = netgen.test_set_net(100, 2, "lattice", density, seed=3)
    assert sp.n_edges == 100 * k
    for j in range(100):
        assert set(sp.src[sp.dst == j].tolist()) == _brute_knn(sp.pos, j, k)


@pytest.mark.parametrize("density,p,k", [("low", 0.05, 3), ("high", 0.15, 8)])
def test_small_world_rewires_the_expected_share(density, p, k):
    sp = netgen.test_set_net(1000, 2, "small_world", density, seed=4)
    assert sp.n_edges == 1000 * k and np.all(np.bincount(sp.dst, minlength=1000) == k)
    assert np.all(sp.src != sp.dst)
    moved = sum(len(set(sp.src[sp.dst == j].tolist()) - _brute_knn(sp.pos, j, k)) for j in range(1000))
    E = 1000 * k
    sd = math.sqrt(E * p * (1 - p))
    assert abs(moved - E * p) < 5 * sd + 0.01 * E   # a re-drawn source may land on a near vertex


@pytest.mark.parametrize("density,m", [("low", 2), ("high", 4)])
def test_scale_free_grows_m_links_per_vertex(density, m):
    n = 1000
    sp = netgen.test_set_net(n, 3, "scale_free", density, seed=5)
    assert sp.n_edges == sum(min(m, v) for v in range(1, n))
    deg = np.bincount(sp.src, minlength=n) + np.bincount(sp.dst, minlength=n)
    assert deg.max() > 4 * deg.mean()    # heavy tail: hubs far above the mean
    assert np.all(sp.src != sp.dst)


@pytest.mark.parametrize("density,p", [("low", 0.10), ("high", 0.20)])
def test_random_graph_density(density, p):
    n = 300
    sp = netgen.test_set_net(n, 2, "random", density, seed=6)
    pairs = n * (n - 1)
    assert abs(sp.n_edges - p * pairs) < 5 * math.sqrt(pairs * p * (1 - p))
    assert np.all(sp.src != sp.dst) and len(set(zip(sp.src.tolist(), sp.dst.tolist()))) == sp.n_edges


def test_the_set_spans_the_table():
    nets = netgen.test_set()
    assert len(nets) == 80
    seen = {(sp.n_nodes, sp.dim, sp.name.split("_")[1] if "small" not in sp.name and "scale" not in sp.name else
             "_".join(sp.name.split("_")[1:3])) for sp in nets}
    assert {n for n, _, _ in seen} == set(netgen.TEST_SET_SIZES) and {d for _, d, _ in seen} == {2, 3}
    assert {c for _, _, c in seen} == set(netgen.TEST_SET_CLASSES)
    assert all(sp.dt_ms == 1.0 and sp.speed_scalar > 0 for sp in nets)
