"""Pins of the FP64 oracle to facts outside itself (closed forms, textbook
results, library routines, brute force, the paper's worked example).

Each test names the passage of Buibas & Silva (arXiv:0908.3934) or the outside
source it pins against.  None of them re-types the oracle's own formulas.
"""
import math
import os

import numpy as np
import pytest
from scipy import signal, stats
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import dijkstra

import oracle
from paper_0908_3934_b300 import netgen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# classic FHN, dv/dt = v - v^3/3 - w + I, dw/dt = eps (v + a - b w)  (textbook form)
A_CL, B_CL, EPS = 0.7, 0.8, 0.08


def cardano_rest(a=A_CL, b=B_CL, i_ext=0.0):
    """Rest point of the classic FHN from Cardano's formula.  The nullclines
    w = v - v^3/3 + I and w = (v + a)/b meet where v^3 + p v + q = 0 with
    p = 3/b - 3 and q = 3a/b - 3I (one real root when (q/2)^2 + (p/3)^3 > 0)."""
    p = 3.0 / b - 3.0
    q = 3.0 * a / b - 3.0 * i_ext
    disc = (q / 2.0) ** 2 + (p / 3.0) ** 3
    assert disc > 0
    r = math.sqrt(disc)
    v = np.cbrt(-q / 2.0 + r) + np.cbrt(-q / 2.0 - r)
    return float(v), float((v + a) / b)


def iso_spec(n, fhn=None, pulses=(), dt=0.05, sample_every=1000):
    """n unconnected nodes."""
    return netgen.NetSpec(pos=np.zeros((n, 2)), src=np.zeros(0, np.int32), dst=np.zeros(0, np.int32),
                          weight=np.zeros(0, np.float32), speed=None, speed_scalar=1.0, dt_ms=dt,
                          fhn=dict(fhn or netgen.FHN_CLASSIC),
                          obs=dict(netgen.OBS_DEFAULT, sample_every=sample_every),
                          pulses=list(pulses))


def one_step(spec, v0, w0):
    """One oracle step of isolated nodes from the state (v0, w0) (relative to rest)."""
    n = len(v0)
    hist = np.zeros((2, n))
    hist[0] = v0
    r = oracle.simulate(spec, 1, init=dict(n0=1, v=v0, w=w0, c=np.zeros(n), hist=hist), want_y=False)
    return r["v"], r["w"]


# --------------------------------------------------------------------------- RNG
def test_philox_known_answers():
    """Philox4x32-10 against the published known-answer vectors (Salmon et al., SC'11)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert out.tolist() == v[6:10]


def test_gaussian_noise_statistics():
    """The readout noise N(0, gamma^2) of Sec. 3.3: xi is standard normal
    (mean, variance and a Kolmogorov-Smirnov test against scipy's normal)."""
    xs = np.array([oracle.gauss(7, j, k) for j in range(40) for k in range(1000)])
    M = xs.size
    assert abs(xs.mean()) < 4.0 / math.sqrt(M)
    assert abs(xs.std() - 1.0) < 4.0 * math.sqrt(0.5 / M)
    assert stats.kstest(xs, "norm").pvalue > 1e-3


def test_background_threshold_and_rate():
    """5 Hz onsets at dt = 0.05 ms: p = 2.5e-4 per step, threshold floor(p 2^32)."""
    thr = oracle.bg_threshold(5.0, 0.05)
    assert thr == math.floor(2.5e-4 * 2 ** 32) == 1073741
    assert oracle.bg_threshold(0.0, 0.05) == 0
    n = sum(oracle.bg_onset(11, j, k, thr) for j in range(100) for k in range(4000))
    # binomial(400000, 2.5e-4): mean 100, sd 10
    assert 50 <= n <= 150


# --------------------------------------------------------------------------- FHN
@pytest.mark.parametrize("i_ext", [0.0, 0.1, -0.2])
def test_rest_point_matches_cardano(i_ext):
    """The rest point (Sec. 3.1 FHN with S = U = 0) equals Cardano's closed form."""
    fhn = dict(netgen.FHN_CLASSIC, i_ext=i_ext)
    v, w = oracle.rest_point(fhn)
    vc, wc = cardano_rest(i_ext=i_ext)
    assert abs(v - vc) < 1e-14 and abs(w - wc) < 1e-14


def test_nullclines_are_stationary():
    """On the textbook V-nullcline w = v - v^3/3 + I one Euler step leaves V
    unchanged; on the W-nullcline w = (v + a)/b it leaves W unchanged.  This pins
    the whole FHN vector field of the transition (Sec. 3.1) at arbitrary points."""
    spec = iso_spec(7)
    vr, wr = cardano_rest()
    V = np.array([-2.1, -1.5, -0.7, 0.0, 0.4, 1.3, 2.2])
    Wv = V - V ** 3 / 3.0
    v1, _ = one_step(spec, V - vr, Wv - wr)
    assert np.max(np.abs(v1 - (V - vr))) < 1e-13
    Ww = (V + A_CL) / B_CL
    _, w1 = one_step(spec, V - vr, Ww - wr)
    assert np.max(np.abs(w1 - (Ww - wr))) < 1e-13


def test_euler_step_size():
    """Off the nullclines the Euler increment is dt * h(y) (Sec. 3.1, Euler form):
    halving dt halves the increment of the same state (the vector field is pinned
    by the nullcline test, its scale by this one)."""
    vr, wr = cardano_rest()
    V = np.array([-1.0, 0.5, 1.7])
    W = np.array([0.2, -0.3, 0.9])
    v1, w1 = one_step(iso_spec(3, dt=0.05), V - vr, W - wr)
    v2, w2 = one_step(iso_spec(3, dt=0.025), V - vr, W - wr)
    assert np.allclose((v1 - (V - vr)), 2.0 * (v2 - (V - vr)), rtol=1e-12, atol=1e-15)
    assert np.allclose((w1 - (W - wr)), 2.0 * (w2 - (W - wr)), rtol=1e-12, atol=1e-15)
    # and the rate equals the textbook right-hand side at the sampled points
    dv = V - V ** 3 / 3.0 - W
    dw = EPS * (V + A_CL - B_CL * W)
    assert np.allclose(v1 - (V - vr), 0.05 * dv, rtol=1e-12, atol=1e-14)
    assert np.allclose(w1 - (W - wr), 0.05 * dw, rtol=1e-12, atol=1e-14)


def test_small_perturbation_follows_linearisation():
    """A perturbation of 1e-9 evolves as (I + dt J)^n x0 with J the Jacobian of
    the classic FHN at rest, [[1 - v*^2, -1], [eps, -eps b]] (textbook linear
    stability); matrix powers from numpy."""
    vr, _ = cardano_rest()
    dt = 0.05
    J = np.array([[1.0 - vr * vr, -1.0], [EPS, -EPS * B_CL]])
    M = np.eye(2) + dt * J
    x0 = np.array([1e-9, -3e-10])
    spec = iso_spec(1)
    n = 2000
    hist = np.zeros((2, 1))
    hist[0] = x0[0]
    r = oracle.simulate(spec, n, init=dict(n0=1, v=x0[:1], w=x0[1:], c=np.zeros(1), hist=hist), want_y=False)
    want = np.linalg.matrix_power(M, n) @ x0
    got = np.array([r["v"][0], r["w"][0]])
    assert np.allclose(got, want, rtol=1e-5, atol=1e-24)


def test_relaxation_oscillation_amplitude():
    """Above the Hopf point the classic FHN relaxes between the outer branches of
    the cubic nullcline; in the singular limit V swings between about -2 and 2
    (the branches through the knees at w = -+2/3).  eps = 0.08 overshoots a little."""
    spec = iso_spec(1, fhn=dict(netgen.FHN_CLASSIC, i_ext=0.5))
    vr, _ = oracle.rest_point(spec.fhn)
    hist = np.zeros((2, 1))
    hist[0] = 0.1
    r = oracle.simulate(spec, 16000, snap_every=1, want_y=False,
                        init=dict(n0=1, v=[0.1], w=[0.0], c=[0.0], hist=hist))
    V = vr + r["snap_v"][8000:, 0]
    assert 1.8 < V.max() < 2.2
    assert -2.2 < V.min() < -1.8


# --------------------------------------------------------------------------- delays
def test_delay_closed_forms():
    """tau = |x_i - x_j| / s (Eq. delaydist, Sec. 3.2.1) on distances that are exact."""
    pos = np.array([[0.0, 0.0], [0.3, 0.4], [0.625, 0.0], [0.375, 0.0], [1e-4, 0.0]])
    src = np.array([0, 1, 0, 0, 0, 4], np.int32)
    dst = np.array([1, 0, 2, 3, 4, 0], np.int32)
    D, cl = oracle.delays(pos, src, dst, None, 0.1, 0.05)
    assert D[0] == D[1] == 100  # 0.5 mm at 0.1 mm/ms, dt 0.05 ms
    assert not cl[0]
    # exact halves (s dt = 0.25): 2.5 -> 3, 1.5 -> 2 (half away from zero)
    D2, _ = oracle.delays(pos, src, dst, None, 1.0, 0.25)
    assert D2[2] == 3 and D2[3] == 2
    # a delay below half a step is clamped to one step and flagged
    assert D[4] == 1 and D[5] == 1 and cl[4] and cl[5]
    # 3D: (1, 2, 2) has length 3
    p3 = np.array([[0.0, 0.0, 0.0], [0.1, 0.2, 0.2]])
    D3, _ = oracle.delays(p3, np.array([0], np.int32), np.array([1], np.int32), None, 0.1, 0.05)
    assert D3[0] == 60


def test_delays_per_edge_speed():
    """Per-edge speeds: tau_ij = d_ij / s_ij, Gamma_ij = {s} (Sec. 3.2.1)."""
    pos = np.array([[0.0, 0.0], [0.3, 0.4]])
    src = np.array([0, 1], np.int32)
    dst = np.array([1, 0], np.int32)
    D, _ = oracle.delays(pos, src, dst, np.array([0.1, 0.25]), 0.0, 0.05)
    assert D.tolist() == [100, 40]


# --------------------------------------------------------------------------- network
def test_fig2_worked_example_arrivals():
    """Figs. 1-2 (Sec. 3): the printed delays are whole multiples of dt = 0.05 ms;
    after a pulse on vertex 1 every vertex first leaves rest one step after the
    earliest delayed arrival along the network -- the shortest path with edge
    length D + 1 (scipy's Dijkstra)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "fig2_network.txt")) if l[0] != "#"]
    delay_ms = [float(r[2]) for r in rows]
    steps = [oracle.ms_to_step(d, 0.05) for d in delay_ms]
    assert steps == [72, 148, 76, 52, 96, 68, 72, 88]
    for d, s in zip(delay_ms, steps):
        assert abs(d / 0.05 - s) < 1e-9
    spec = netgen.fig2(steps)
    assert spec.weight.tolist() == [float(np.float32(r[3])) for r in rows]
    r = oracle.simulate(spec, 1000)
    n_on = 200
    G = csr_matrix((np.array(steps, float) + 1.0, (spec.src, spec.dst)), shape=(5, 5))
    dist = dijkstra(G, indices=0)
    want = (n_on + 1 + dist).astype(np.int64)
    assert r["first_arrival"].tolist() == want.tolist()
    assert want.tolist() == [201, 274, 350, 327, 423]  # vertex 5 via 1 -> 3 -> 5


def test_two_node_chain_first_arrival():
    """A two-node chain delivers the first change of node 0 to node 1's input
    exactly round(d / (s dt)) steps later; node 1 itself moves one step after."""
    for d, s in [(0.5, 0.1), (0.25, 0.05), (0.013, 0.5)]:
        spec = netgen.chain2(dist_mm=d, speed=s)
        D = int(round(d / (s * 0.05)))
        r = oracle.simulate(spec, 1000)
        assert r["delay"][0] == max(1, D)
        f0, f1 = r["first_arrival"]
        assert f0 == 101  # pulse starts at 5 ms = step 100
        assert f1 == f0 + max(1, D) + 1


def test_two_node_chain_first_arrival_at_a_deep_delay():
    """The same at a delay of 5000 steps, deeper than any ring the benchmark sizes
    (slow conduction, 0.002 mm/ms over 0.5 mm)."""
    d, s = 0.5, 0.002
    spec = netgen.chain2(dist_mm=d, speed=s)
    D = int(round(d / (s * 0.05)))
    assert D == 5000
    r = oracle.simulate(spec, 5200)
    assert r["delay"][0] == D
    f0, f1 = r["first_arrival"]
    assert f0 == 101 and f1 == f0 + D + 1


def test_tiny_arrivals_match_dijkstra():
    """Config 'tiny': all first arrivals equal the shortest-path schedule."""
    spec = netgen.tiny()
    r = oracle.simulate(spec, 4000)
    D = r["delay"]
    G = csr_matrix((D.astype(float) + 1.0, (spec.src, spec.dst)), shape=(spec.n_nodes,) * 2)
    dist = dijkstra(G, indices=0)
    want = np.where(np.isfinite(dist), 201 + np.nan_to_num(dist, posinf=0), -1).astype(np.int64)
    want[want > 4000] = -1
    assert np.array_equal(r["first_arrival"], want)
    assert (want > 0).sum() > 40


def test_unstimulated_network_stays_at_rest():
    """With u = 0 the rest point is an exact fixed point of the coupled network."""
    spec = netgen.tiny()
    spec.pulses = []
    r = oracle.simulate(spec, 3000)
    assert not r["v"].any() and not r["w"].any() and not r["c"].any()
    assert (r["first_arrival"] == -1).all() and r["ev_count"] == 0


def test_zero_weights_decouple_nodes():
    """Eq. basicstate (Sec. 3.1): with all weights zero each vertex evolves as an
    isolated vertex -- node 0 equals a one-node run, all others stay at rest."""
    spec = netgen.tiny()
    spec.weight = np.zeros_like(spec.weight)
    r = oracle.simulate(spec, 3000)
    one = iso_spec(1, pulses=[(0, 10.0, 12.0, 1.0)], sample_every=20)
    r1 = oracle.simulate(one, 3000)
    assert r["v"][0] == r1["v"][0] and r["w"][0] == r1["w"][0] and r["c"][0] == r1["c"][0]
    assert np.array_equal(r["y_clean"][:, 0], r1["y_clean"][:, 0])
    assert not r["v"][1:].any()


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_ring_history_equals_dense_brute_force(seed):
    """The circular history equals the brute force that keeps every past state
    and reads v_i(t - tau_ij) by its time index (Eq. Yjset, Sec. 2), bit for bit."""
    spec = netgen.random_small(seed)
    a = oracle.simulate(spec, 1500, dense=True)
    b = oracle.simulate(spec, 1500)
    for k in ("v", "w", "c", "y", "first_arrival", "ev_node", "ev_step"):
        assert np.array_equal(a[k], b[k]), k


def test_readout_is_a_first_order_lowpass():
    """The readout follows the linear calcium-style filter of Sec. 3.3: the
    sampled c equals scipy's lfilter of the V trace with pole 1 - dt/tau."""
    spec = netgen.tiny()
    r = oracle.simulate(spec, 3000, snap_every=1)
    alpha = spec.dt_ms / spec.obs["tau_ms"]
    c = signal.lfilter([alpha], [1.0, alpha - 1.0], r["snap_v"], axis=0)
    assert np.allclose(c, r["snap_c"], rtol=1e-11, atol=1e-14)
    vr, _ = r["rest"]
    assert np.allclose(r["y_clean"], vr + r["snap_c"][19::20], rtol=0, atol=1e-15)


def test_observation_noise_is_gaussian():
    """y = n c + b + N(0, gamma^2) (Sec. 3.3): the residual y - y_clean is
    gamma times a standard normal."""
    spec = netgen.tiny()
    r = oracle.simulate(spec, 20000)
    xi = (r["y"] - r["y_clean"]).ravel() / np.float32(spec.obs["sigma"])
    assert abs(xi.mean()) < 4.0 / math.sqrt(xi.size)
    assert stats.kstest(xi, "norm").pvalue > 1e-3


def test_events_are_upward_zero_crossings():
    """Events are the upward crossings of V through 0, found here by brute force on
    the recorded trajectory."""
    spec = netgen.tiny()
    r = oracle.simulate(spec, 4000, snap_every=1)
    vr, _ = r["rest"]
    V = vr + np.vstack([np.zeros((1, spec.n_nodes)), r["snap_v"]])
    up = (V[:-1] < 0) & (V[1:] >= 0)
    steps, nodes = np.nonzero(up)
    want = sorted(zip(nodes.tolist(), (steps + 1).tolist()))
    got = sorted(zip(r["ev_node"].tolist(), r["ev_step"].tolist()))
    assert got == want and len(want) > 20


def test_background_pulses_start_at_onsets():
    """An isolated node driven only by background pulses leaves rest one step after
    its first onset."""
    spec = iso_spec(30)
    spec.background = dict(rate_hz=500.0, amp=1.0, dur_ms=2.0, seed=5)
    thr = oracle.bg_threshold(500.0, spec.dt_ms)
    r = oracle.simulate(spec, 400, want_y=False)
    for j in range(30):
        onsets = [n for n in range(400) if oracle.bg_onset(5, j, n, thr)]
        want = onsets[0] + 1 if onsets else -1
        assert r["first_arrival"][j] == want


def test_raw_coupling_uses_absolute_voltage():
    """RAW coupling passes V itself: a node whose two inputs carry +w and -w from
    sources at rest receives exactly zero and stays at rest, while a node with one
    input of weight w is driven by w V*."""
    pos = np.zeros((4, 2))
    src = np.array([0, 1, 0], np.int32)
    dst = np.array([2, 2, 3], np.int32)
    w = np.array([0.25, -0.25, 0.25], np.float32)
    spec = netgen.NetSpec(pos=pos, src=src, dst=dst, weight=w, speed=None, speed_scalar=1.0,
                          delay=np.array([3, 3, 3], np.int32), coupling="raw")
    r = oracle.simulate(spec, 1, want_y=False)
    vr, _ = r["rest"]
    assert r["v"][2] == 0.0
    assert r["v"][3] == pytest.approx(0.05 * 0.25 * vr, rel=1e-15)
