"""The seeded synthetic workloads follow the recipes they stand in for: node and
edge counts, degree statistics, the weight, speed, stimulus and observation laws
(CPU; the radius and hub nets at reduced node counts, where the laws do not depend
on the size).  Statistical checks allow 4 standard errors."""
import math

import numpy as np
import pytest

from paper_0908_3934_b300 import netgen


def _dist(sp):
    return np.sqrt(((sp.pos[sp.src] - sp.pos[sp.dst]) ** 2).sum(1))


def _in_deg(sp):
    return np.bincount(sp.dst, minlength=sp.n_nodes)


def _no_duplicates_or_loops(sp):
    key = sp.src.astype(np.int64) * sp.n_nodes + sp.dst
    return np.unique(key).size == key.size and (sp.src != sp.dst).all()


def _within(x, mean, se):
    return abs(x - mean) <= 4.0 * se


def test_tiny_recipe():
    """64 nodes in a 1 x 1 mm square, ordered pairs closer than 0.2 mm kept with
    p = 0.5, w ~ U(0.1, 0.5), speed 0.1 m/s, dt 0.05 ms, +1 on node 0 over [10, 12) ms,
    readout tau 5 ms with noise sigma 0.05 sampled every 1 ms."""
    sp = netgen.tiny()
    assert sp.n_nodes == 64 and sp.dim == 2 and sp.pos.min() >= 0.0 and sp.pos.max() < 1.0
    assert (_dist(sp) < 0.2).all() and _no_duplicates_or_loops(sp)
    D = np.sqrt(((sp.pos[:, None, :] - sp.pos[None, :, :]) ** 2).sum(-1))
    pairs = int(((D < 0.2) & ~np.eye(64, dtype=bool)).sum())
    assert _within(sp.n_edges, 0.5 * pairs, math.sqrt(0.25 * pairs))
    assert sp.weight.dtype == np.float32 and sp.weight.min() >= 0.1 and sp.weight.max() < 0.5
    assert sp.speed is None and sp.speed_scalar == 0.1 and sp.dt_ms == 0.05
    assert sp.pulses == [(0, 10.0, 12.0, 1.0)] and sp.background is None
    assert sp.obs["tau_ms"] == 5.0 and sp.obs["sigma"] == 0.05 and sp.obs["sample_every"] * sp.dt_ms == 1.0


def _unscaled_weights(sp, k0=20.0):
    """The weight law before the in-degree scaling w * min(1, k0 / k_dst)."""
    k = _in_deg(sp).astype(np.float64)[sp.dst]
    return sp.weight.astype(np.float64) / np.minimum(1.0, k0 / np.maximum(k, 1.0))


def _check_signed_lognormal_and_speeds(sp):
    w = _unscaled_weights(sp)
    E = w.size
    neg = float((w < 0).mean())
    assert _within(neg, 0.2, math.sqrt(0.16 / E))
    lw = np.log(np.abs(w))
    assert _within(lw.mean(), -2.0, 0.5 / math.sqrt(E)) and abs(lw.std() - 0.5) < 0.01
    assert sp.speed.min() >= 0.05 and sp.speed.max() < 0.5
    assert _within(sp.speed.mean(), 0.275, 0.45 / math.sqrt(12 * E))
    # targets with more than 20 inputs keep the total |input| of a 20-input node
    k = _in_deg(sp)
    big = np.flatnonzero(k > 20)
    if big.size:
        j = big[0]
        assert np.abs(w[sp.dst == j]).sum() * 20.0 / k[j] == pytest.approx(np.abs(sp.weight[sp.dst == j]).sum(),
                                                                           rel=1e-5)


def test_large_recipe_at_20k_nodes():
    """A unit cube, every ordered pair within the radius that gives mean in-degree
    100 (border losses included), signed lognormal(-2, 0.5) weights with 20 %
    negated (in-degree scaled), speeds U(0.05, 0.5) m/s, 5 Hz background pulses of
    2 ms, a ring of 256 steps."""
    sp = netgen.large(n=20000, mean_deg=100.0)
    assert sp.n_nodes == 20000 and sp.dim == 3 and sp.pos.min() >= 0.0 and sp.pos.max() < 1.0
    assert _no_duplicates_or_loops(sp)
    assert abs(_in_deg(sp).mean() - 100.0) < 2.0
    r = _dist(sp).max()
    # a radius graph: every pair closer than the largest edge length is an edge
    from scipy.spatial import cKDTree
    probe = np.arange(0, 20000, 997)
    near = cKDTree(sp.pos).query_ball_point(sp.pos[probe], r * 0.999)
    for j, ns in zip(probe, near):
        assert set(ns) - {j} <= set(sp.src[sp.dst == j].tolist())
    _check_signed_lognormal_and_speeds(sp)
    assert sp.background["rate_hz"] == 5.0 and sp.background["dur_ms"] == 2.0 and sp.ring_depth == 256


def test_roofline_recipe_at_40k_nodes():
    """Mean in-degree 50 with 2.5 % hubs taking in-edges from their 1000 nearest
    nodes and the other targets a radius graph of the remaining mean (about 25.6);
    the weight, speed and background laws of the large net."""
    n = 40000
    sp = netgen.roofline(n=n)
    k = _in_deg(sp)
    assert sp.n_nodes == n and _no_duplicates_or_loops(sp)
    hubs = np.flatnonzero(k == 1000)
    assert hubs.size == round(0.025 * n)
    assert abs(k.mean() - 50.0) < 1.0
    rest = np.delete(k, hubs)
    assert abs(rest.mean() - (50.0 * n - 1000.0 * hubs.size) / (n - hubs.size)) < 0.6
    assert rest.max() < 1000
    # a hub's sources are exactly its 1000 nearest other nodes
    j = hubs[0]
    d = np.sqrt(((sp.pos - sp.pos[j]) ** 2).sum(1))
    d[j] = np.inf
    assert set(sp.src[sp.dst == j].tolist()) == set(np.argsort(d, kind="stable")[:1000].tolist())
    _check_signed_lognormal_and_speeds(sp)
    assert sp.background["rate_hz"] == 5.0 and sp.ring_depth == 256


def test_batch_members_recipe():
    """2D members with N log-uniform in [32, 4096], pairs within sqrt(40 / (pi N))
    kept with p = 0.5 (kept in-degree about 20 away from the border), unscaled
    signed lognormal weights, speeds U(0.05, 0.5), 1-8 distinct nodes pulsed with
    amplitude 1 for 2 ms from an onset in [5, 50) ms; N = 512 on request (the
    estimator nets)."""
    members = netgen.batch(300, seed0=1000)
    N = np.array([m.n_nodes for m in members])
    assert N.min() >= 32 and N.max() <= 4096
    lo, hi = math.log(32), math.log(4096)
    assert _within(np.log(N).mean(), 0.5 * (lo + hi), (hi - lo) / math.sqrt(12 * N.size))
    for m in members:
        assert m.dim == 2 and _no_duplicates_or_loops(m)
        assert m.radius == pytest.approx(math.sqrt(40.0 / (math.pi * m.n_nodes)))
        assert (_dist(m) < m.radius).all()
        assert 1 <= len(m.pulses) <= 8 and len({p[0] for p in m.pulses}) == len(m.pulses)
        for node, t0, t1, amp in m.pulses:
            assert 0 <= node < m.n_nodes and 5.0 <= t0 < 50.0 and t1 - t0 == pytest.approx(2.0) and amp == 1.0
        assert m.speed.min() >= 0.05 and m.speed.max() < 0.5
    big = [m for m in members if m.n_nodes >= 2000]
    assert big and all(15.0 < _in_deg(m).mean() < 20.5 for m in big)
    w = np.concatenate([m.weight for m in members]).astype(np.float64)
    assert _within(float((w < 0).mean()), 0.2, math.sqrt(0.16 / w.size))
    assert _within(np.log(np.abs(w)).mean(), -2.0, 0.5 / math.sqrt(w.size))
    assert netgen.batch_member(7, n=512).n_nodes == 512


def test_candidate_pairs_and_labels_by_brute_force():
    """The estimator's candidates are every ordered pair closer than the member's
    radius, labelled 1 exactly where the pair is an edge (every edge is a candidate,
    about half the candidates are edges); a table of several members numbers the
    nodes globally in member order."""
    from paper_0908_3934_b300 import pipeline
    members = [netgen.batch_member(40 + i, n=n) for i, n in enumerate((60, 200, 512))]
    for m in members:
        src, dst, lab = netgen.candidates(m)
        D = np.sqrt(((m.pos[:, None, :] - m.pos[None, :, :]) ** 2).sum(-1))
        want = {(int(i), int(j)) for i, j in zip(*np.nonzero((D < m.radius) & ~np.eye(m.n_nodes, dtype=bool)))}
        got = list(zip(src.tolist(), dst.tolist()))
        assert len(got) == len(set(got)) and set(got) == want
        edges = set(zip(m.src.tolist(), m.dst.tolist()))
        assert [int(x) for x in lab] == [1 if p in edges else 0 for p in got]
        assert int(lab.sum()) == m.n_edges
        assert _within(lab.mean(), 0.5, math.sqrt(0.25 / lab.size))
    tab = pipeline.candidate_table(members)
    off = np.cumsum([0] + [m.n_nodes for m in members])
    assert tab["n_nodes"] == off[-1] and np.array_equal(tab["pos"], np.concatenate([m.pos for m in members]))
    for i, m in enumerate(members):
        sel = tab["net"] == i
        src, dst, lab = netgen.candidates(m)
        assert np.array_equal(tab["src"][sel], src + off[i]) and np.array_equal(tab["dst"][sel], dst + off[i])
        assert np.array_equal(tab["label"][sel], lab) and np.all(tab["radius"][sel] == m.radius)
    assert tab["src"].dtype == np.int32 and tab["radius"].dtype == np.float64


def test_secondary_roofline_variants():
    """The literal 5 % hub variant (5 % of the nodes with 1000 inputs beside a radius
    graph of mean in-degree 50: about 97.5 overall) and the delay-stress variant
    (every speed x 0.1, ring sized afresh)."""
    n = 40000
    sp = netgen.roofline(n=n, hub_frac=0.05, mean_deg=97.5)
    k = _in_deg(sp)
    hubs = k == 1000
    assert hubs.sum() == round(0.05 * n) and abs(k.mean() - 97.5) < 2.0 and abs(k[~hubs].mean() - 50.0) < 1.0
    base = netgen.roofline(n=n)
    slow = netgen.delay_stress(base)
    assert np.array_equal(slow.src, base.src) and np.array_equal(slow.weight, base.weight)
    assert np.allclose(slow.speed, base.speed * 0.1) and slow.ring_depth == 0
    with pytest.raises(ValueError):
        netgen.delay_stress(netgen.tiny())
