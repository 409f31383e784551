"""Pins of the oracle's third node model -- Hodgkin-Huxley nodes (the paper's
second benchmark model, Sec. 3.1 and 3.4: state {v, m, n, h}, dt = 0.03 ms) with
the alpha-function PSC and calcium readout of Eq. alphapsc / spd / casimple --
against the model's published rest state and firing behaviour, closed forms of
the Euler recurrences, and brute force."""
import numpy as np
import pytest

import oracle
from paper_0908_3934_b300 import netgen

HH = netgen.HH_CLASSIC
DT = 0.03


def _lone(i_ext=0.0, dt=DT, n=1, src=(), dst=(), w=(), delay=None, pulses=(), **hh):
    return netgen.NetSpec(pos=np.zeros((n, 2)), src=np.array(src, np.int32), dst=np.array(dst, np.int32),
                          weight=np.array(w, np.float32), speed=None, speed_scalar=1.0,
                          delay=None if delay is None else np.array(delay, np.int32), dt_ms=dt,
                          pulses=list(pulses), model="hh", hh=dict(HH, i_ext=i_ext, **hh),
                          obs=dict(netgen.OBS_DEFAULT))


def _clamped(v0, n_steps, gates=None):
    """A node whose capacitance is so large that dt / C times any current is below
    half an ulp of V: V stays exactly v0 and only the gates move."""
    sp = _lone(C=1e30)
    g = oracle.hh_rest_gates() if gates is None else gates
    r = oracle.simulate(sp, n_steps, want_y=False,
                        init=dict(n0=0, v=[v0], w=[0.0], c=[0.0], r=[0.0], p=[0.0], m=[g[0]], n=[g[1]], h=[g[2]],
                                  hist=np.zeros((1, 1))))
    assert r["v"][0] == v0
    return np.array([r["m"][0], r["n"][0], r["h"][0]])


def test_rest_gates_are_the_published_values():
    """The classic squid-axon gates at -65 mV: m = 0.0529, n = 0.3177, h = 0.5961."""
    m, n, h = oracle.hh_rest_gates()
    assert (m, n, h) == pytest.approx((0.0529, 0.3177, 0.5961), abs=6e-5)


def test_a_lone_node_stays_at_rest():
    """E_L = -54.387 mV balances the currents at -65 mV: without input V stays
    within 0.01 mV of -65 and never crosses 0 mV, and the gates stay at rest."""
    r = oracle.simulate(_lone(), int(300 / DT), want_y=False, snap_every=1)
    V = r["snap_v"][:, 0]
    assert np.abs(V + 65.0).max() < 0.01 and r["ev_count"] == 0
    assert [r["m"][0], r["n"][0], r["h"][0]] == pytest.approx(list(oracle.hh_rest_gates()), abs=2e-4)
    assert r["p"][0] == 0.0 and r["r"][0] == 0.0


def test_type_ii_repetitive_firing():
    """Below ~6.2 uA/cm^2 a current step gives at most a transient; above it the
    model fires repetitively and starts at a non-zero rate (class II onset, ~50 Hz);
    at 10 uA/cm^2 it fires near 68 Hz, the first spike from rest peaking near
    +40 mV (later ones lower, h not having recovered) and an after-hyperpolarisation
    near -75 mV."""
    T = 1000.0

    def run(I):
        r = oracle.simulate(_lone(I), int(T / DT), want_y=False, ev_cap=10000, snap_every=1)
        ev = r["ev_step"][:r["ev_count"]] * DT
        late = ev[ev > 500.0]
        f = (late.size - 1) / (late[-1] - late[0]) * 1000.0 if late.size > 1 else 0.0
        return r, f

    r6, f6 = run(6.0)
    assert r6["ev_count"] <= 2 and f6 == 0.0
    _, f65 = run(6.5)
    assert 48.0 < f65 < 60.0
    r10, f10 = run(10.0)
    assert 65.0 < f10 < 71.0
    V = r10["snap_v"][:, 0]
    late = V[int(100 / DT):]
    assert 37.0 < V.max() < 44.0 and 20.0 < late.max() < V.max() and -77.0 < late.min() < -73.0


@pytest.mark.parametrize("v0", [-20.0, -50.0, -80.0])
def test_gates_relax_geometrically_under_a_clamp(v0):
    """With V held fixed each gate obeys x' = x + dt (alpha (1 - x) - beta x), a
    linear recurrence: the successive differences shrink by one constant factor
    q = 1 - dt (alpha + beta) in (0, 1), and x approaches alpha / (alpha + beta).
    Depolarisation opens m and n and closes h; hyperpolarisation the reverse."""
    xs = np.array([_clamped(v0, k) for k in range(0, 6)])
    d = np.diff(xs, axis=0)
    q = d[1:] / d[:-1]
    assert np.all(q > 0.0) and np.all(q < 1.0)
    assert np.allclose(q, q[0], rtol=1e-9, atol=0)
    x_inf = xs[0] + d[0] / (1.0 - q[0])
    far = _clamped(v0, 20000)   # 600 ms, many times the slowest time constant
    assert far == pytest.approx(x_inf, abs=1e-5)
    rest = np.array(oracle.hh_rest_gates())
    if v0 > -65.0:
        assert x_inf[0] > rest[0] and x_inf[1] > rest[1] and x_inf[2] < rest[2]
    else:
        assert x_inf[0] < rest[0] and x_inf[1] < rest[1] and x_inf[2] > rest[2]


@pytest.mark.parametrize("v_sing", [-40.0, -55.0])
def test_the_removable_singularities_are_continuous(v_sing):
    """alpha_m has 0/0 at -40 mV and alpha_n at -55 mV; the gates after a step at
    exactly that voltage agree with those a hair either side of it."""
    at = _clamped(v_sing, 50)
    assert np.all(np.isfinite(at))
    for eps in (1e-6, -1e-6):
        assert _clamped(v_sing + eps, 50) == pytest.approx(at, abs=1e-6)


def test_events_are_upward_crossings_and_calcium_counts_the_time_above_peak():
    """Events are the steps n + 1 with V(n) < V_peak <= V(n + 1); spd(V) stays 1 for
    every step spent above V_peak, and c(n + 1) = c(n)(1 - dt / tau_c) + dt spd(V(n))
    sums to dt sum_n q^(n_end - 1 - n) spd(V(n)) (Eq. casimple)."""
    sp = _lone(10.0)
    n_end = int(200 / DT)
    r = oracle.simulate(sp, n_end, ev_cap=1000, snap_every=1, want_y=False)
    V = np.concatenate([[-65.0], r["snap_v"][:, 0]])
    cross = np.nonzero((V[:-1] < 0.0) & (V[1:] >= 0.0))[0] + 1
    assert cross.size >= 10 and np.array_equal(r["ev_step"][:r["ev_count"]], cross)
    above = V[:-1] >= 0.0
    assert above.sum() > 3 * cross.size            # a spike is wider than one step
    q = 1.0 - DT / HH["tau_c"]
    c_ref = sum(DT * q ** (n_end - 1 - n) for n in np.nonzero(above)[0])
    assert r["c"][0] == pytest.approx(c_ref, rel=1e-12)


def test_one_spike_reaches_its_target_after_the_delay():
    """Edge 0 -> 1 with D = 100 steps: node 0 first reaches 0 mV at step s0, and
    p_1 stays exactly 0 through step s0 + D, then equals dt w at s0 + D + 1."""
    D, w = 100, 12.0
    sp = _lone(0.0, n=2, src=[0], dst=[1], w=[w], delay=[D], pulses=[(0, 1.0, 3.0, 20.0)])
    r = oracle.simulate(sp, 1000, want_y=False)
    s0 = int(r["ev_step"][0])
    assert r["ev_node"][0] == 0 and r["first_arrival"][0] == s0
    before = oracle.simulate(sp, s0 + D, want_y=False)
    after = oracle.simulate(sp, s0 + D + 1, want_y=False)
    assert before["p"][1] == 0.0 and before["r"][1] == 0.0
    assert after["p"][1] == DT * float(np.float32(w))


def test_hh_ring_equals_dense_history():
    """The circular history and the full [T][N] history give bit-identical runs on
    a spiking Hodgkin-Huxley network."""
    sp = netgen.hodgkin_huxley(netgen.tiny(), w_scale=10.0)
    a = oracle.simulate(sp, 3000, ev_cap=100000)
    b = oracle.simulate(sp, 3000, dense=True, ev_cap=100000)
    assert a["ev_count"] > 20
    for k in ("v", "m", "n", "h", "c", "r", "p", "y", "first_arrival", "ev_node", "ev_step"):
        assert np.array_equal(a[k], b[k]), k


def test_fig2_cascade_follows_the_printed_delays():
    """Fig. 2 (Sec. 3): the five-vertex network with Hodgkin-Huxley nodes, its printed
    delays and weights (x 10), a pulse on each vertex in turn.  The pulse on vertex 1
    sets off the cascade 1 -> 3 -> 5, 3 -> 2 -> 4 along the excitatory edges, each
    spike later than its source's by more than the printed delay; the synaptic input
    p of a vertex whose only earlier input is one edge leaves 0 exactly D + 1 steps
    after its source's first spike (Eq. izpsc, with D = round(delay / dt))."""
    spec = netgen.fig2_hh()
    assert spec.delay.tolist() == [120, 247, 127, 87, 160, 113, 120, 147]
    r = oracle.simulate(spec, 33334, ev_cap=10000, want_y=False)
    first = {}
    for n, j in sorted(zip(r["ev_step"].tolist(), r["ev_node"].tolist())):
        first.setdefault(j + 1, n)
    order = sorted(first, key=first.get)
    assert order == [1, 3, 5, 2, 4]
    dt = spec.dt_ms
    for a, b, d_ms in ((1, 3, 7.4), (3, 5, 3.6), (3, 2, 3.8), (2, 4, 2.6)):
        assert (first[b] - first[a]) * dt > d_ms
    D = dict(((e[0], e[1]), int(spec.delay[k])) for k, e in enumerate(netgen.FIG2_EDGES))
    for a, b in ((1, 3), (1, 2), (3, 5), (2, 4)):
        n = first[a] + D[(a, b)]
        before = oracle.simulate(spec, n, want_y=False)
        after = oracle.simulate(spec, n + 1, want_y=False)
        assert before["p"][b - 1] == 0.0 and after["p"][b - 1] != 0.0, (a, b)
