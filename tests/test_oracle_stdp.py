"""Pins of the oracle's spike-time-dependent plasticity (Sec. 3.2, the plasticity
transition G_ij of Eq. omegatrans with the spike-time state s_j): against the run
without plasticity, closed forms of s and of one pre/post pairing evaluated by hand,
and a brute-force replay of every weight from the spike trains alone."""
import math

import numpy as np
import pytest

import oracle
from paper_0908_3934_b300 import netgen

IZ = netgen.IZH_RS


def _spiking_tiny(model="izh", stdp=None):
    base = netgen.tiny()
    spec = netgen.izhikevich(base, w_scale=7000.0) if model == "izh" else netgen.hodgkin_huxley(base, w_scale=10.0)
    if stdp is not None:
        spec = netgen.dataclasses.replace(spec, stdp=stdp)
    return spec


def _spd_matrix(spec, n_end):
    """spd(V_j(n)) for n = 0 .. n_end (V(0) is the starting state) from snapshots."""
    r = oracle.simulate(spec, n_end, snap_every=1, want_y=False, ev_cap=1 << 20)
    v0 = IZ["vr"] if spec.model == "izh" else -65.0
    vpeak = IZ["vpeak"] if spec.model == "izh" else spec.hh["vpeak"]
    V = np.vstack([np.full((1, spec.n_nodes), v0), r["snap_v"]])
    return V >= vpeak


def _s_closed_form(spd, dt):
    """s_j(n) = dt (n - m - 1) for the last m < n with spd_j(m), else dt n."""
    T, N = spd.shape
    s = np.zeros((T, N))
    last = np.full(N, -1)
    for n in range(T):
        s[n] = np.where(last >= 0, dt * (n - last - 1), dt * n)
        last = np.where(spd[n], n, last)
    return s


def test_zero_rate_is_the_run_without_plasticity():
    plain = oracle.simulate(_spiking_tiny(), 3000, ev_cap=100000)
    zero = oracle.simulate(_spiking_tiny(stdp=dict(alpha=0.0, beta=0.1)), 3000, ev_cap=100000)
    assert plain["ev_count"] > 50
    for k in ("v", "w", "c", "r", "p", "y", "ev_node", "ev_step", "first_arrival"):
        assert np.array_equal(plain[k], zero[k]), k
    assert np.array_equal(zero["w_final"], np.asarray(_spiking_tiny().weight, np.float64))


@pytest.mark.parametrize("model", ["izh", "hh"])
def test_time_since_last_spike_is_the_closed_form(model):
    """s_j' = (1 - spd(V_j)) (s_j + dt) from s_j(0) = 0 sums to dt times the steps
    since the step after the last spike (every step above V_peak counts as spiking)."""
    spec = _spiking_tiny(model, stdp=dict(alpha=0.0, beta=0.1))
    n_end = 3000
    spd = _spd_matrix(spec, n_end)
    r = oracle.simulate(spec, n_end, want_y=False, ev_cap=100000, hist_depth=5)
    s_ref = _s_closed_form(spd, spec.dt_ms)
    assert spd[:-1].any(axis=0).sum() > 10
    assert r["s"] == pytest.approx(s_ref[n_end], rel=1e-12, abs=1e-12)
    for k in range(5):
        assert r["hist_s"][k] == pytest.approx(s_ref[n_end - k], rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("model", ["izh", "hh"])
def test_every_weight_replayed_from_the_spike_trains(model):
    """w_ij(n_end) - w_ij(0) = sum over the steps with max(spd_i(n - D), spd_j(n)) = 1 of
    dt alpha sign(q) exp(-beta |q|), q = s_i(n - D) - s_j(n), evaluated from the spike
    trains alone (spd and s before t = 0 are 0)."""
    alpha, beta = 0.5, 0.05
    spec = _spiking_tiny(model, stdp=dict(alpha=alpha, beta=beta))
    n_end = 2500
    dt = spec.dt_ms
    spd = _spd_matrix(spec, n_end)
    s = _s_closed_form(spd, dt)
    r = oracle.simulate(spec, n_end, want_y=False, ev_cap=100000)
    D = oracle.net_delays(spec)
    src, dst = np.asarray(spec.src), np.asarray(spec.dst)
    w = np.asarray(spec.weight, np.float64).copy()
    for n in range(n_end):
        past = n - D
        ok = past >= 0
        spd_i = np.where(ok, spd[np.maximum(past, 0), src], False)
        s_i = np.where(ok, s[np.maximum(past, 0), src], 0.0)
        gate = spd_i | spd[n, dst]
        q = (s_i - s[n, dst]) * gate
        w += dt * alpha * np.sign(q) * np.exp(-beta * np.abs(q))
    changed = np.abs(r["w_final"] - np.asarray(spec.weight, np.float64)) > 0
    assert changed.sum() > 0.15 * spec.n_edges
    assert r["w_final"] == pytest.approx(w, rel=1e-9, abs=1e-12)


def test_one_pairing_by_hand():
    """Edge 0 -> 1 (D = 10 steps); node 0 spikes once at step a, node 1 once at
    b > a + D.  The printed transition changes w twice: when the pre spike arrives
    (n = a + D: q = s_0(a) - s_1(a + D) = (a - a - D) dt) and when the post neuron
    spikes (n = b: q = s_0(b - D) - s_1(b) = ((b - D - a - 1) - b) dt)."""
    D, alpha, beta, w0 = 10, 0.3, 0.2, 1.0
    izh = dict(IZ)
    spec = netgen.NetSpec(pos=np.zeros((2, 2)), src=np.array([0], np.int32), dst=np.array([1], np.int32),
                          weight=np.array([w0], np.float32), speed=None, speed_scalar=1.0,
                          delay=np.array([D], np.int32), dt_ms=0.05,
                          pulses=[(0, 1.0, 3.0, 2500.0), (1, 6.0, 8.0, 2500.0)], model="izh", izh=izh,
                          obs=dict(netgen.OBS_DEFAULT), stdp=dict(alpha=alpha, beta=beta))
    r = oracle.simulate(spec, 400, want_y=False)
    ev = sorted(zip(r["ev_step"].tolist(), r["ev_node"].tolist()))
    assert [j for _, j in ev] == [0, 1]
    a, b = ev[0][0], ev[1][0]
    assert b > a + D
    dt = spec.dt_ms

    def dw(q):
        return dt * alpha * math.copysign(1.0, q) * math.exp(-beta * abs(q))
    want = w0 + dw(-D * dt) + dw(((b - D - a - 1) - b) * dt)
    assert r["w_final"][0] == pytest.approx(want, rel=1e-12)


def test_restart_from_a_saved_state_continues_the_same_run():
    """A run continued from its state at step 1000 (weights, s, and the spike and s
    histories) equals the uninterrupted run."""
    spec = _spiking_tiny("izh", stdp=dict(alpha=0.5, beta=0.05))
    D = oracle.net_delays(spec)
    depth = int(D.max()) + 1
    full = oracle.simulate(spec, 2000, ev_cap=100000, want_y=False)
    half = oracle.simulate(spec, 1000, ev_cap=100000, want_y=False, hist_depth=depth)
    rest = oracle.simulate(spec, 1000, ev_cap=100000, want_y=False,
                           init=dict(n0=1000, v=half["v"], w=half["w"], c=half["c"], r=half["r"], p=half["p"],
                                     bg_count=half["bg_count"], hist=half["hist"], hist_s=half["hist_s"],
                                     s=half["s"], w_edge=half["w_final"]))
    for k in ("v", "w", "c", "r", "p", "s", "w_final"):
        assert np.array_equal(full[k], rest[k]), k


def test_stdp_ring_equals_dense_history():
    spec = _spiking_tiny("izh", stdp=dict(alpha=0.5, beta=0.05))
    a = oracle.simulate(spec, 2500, ev_cap=100000)
    b = oracle.simulate(spec, 2500, dense=True, ev_cap=100000)
    for k in ("v", "w", "c", "r", "p", "y", "ev_node", "ev_step", "s", "w_final"):
        assert np.array_equal(a[k], b[k]), k


def test_plasticity_needs_a_spiking_model():
    spec = netgen.dataclasses.replace(netgen.tiny(), stdp=dict(alpha=0.1, beta=0.1))
    with pytest.raises(ValueError):
        oracle.simulate(spec, 10)
