"""Pins of the oracle's second node model -- Izhikevich simple model with an
alpha-function PSC and the calcium readout (Eq. izsimple, izpsc, alphapsc, spd,
casimple; Sec. 3.1-3.3) -- against closed forms, exact rules and brute force."""
import math

import numpy as np
import pytest

import oracle
from paper_0908_3934_b300 import netgen

IZ = netgen.IZH_RS


def _lone(i_ext=0.0, dt=0.05, n=1, src=(), dst=(), w=(), delay=None, pulses=()):
    izh = dict(IZ, i_ext=i_ext)
    return netgen.NetSpec(pos=np.zeros((n, 2)), src=np.array(src, np.int32), dst=np.array(dst, np.int32),
                          weight=np.array(w, np.float32), speed=None, speed_scalar=1.0,
                          delay=None if delay is None else np.array(delay, np.int32), dt_ms=dt,
                          pulses=list(pulses), model="izh", izh=izh, obs=dict(netgen.OBS_DEFAULT, gain=20.0))


def test_rheobase_and_the_subthreshold_fixed_point():
    """Below the saddle-node current I* = (k (Vt - Vr) + b)^2 / (4k) a lone node
    settles on the smaller root of k (V - Vr)(V - Vt) - b (V - Vr) + I = 0 with
    W = b (V - Vr); above it, it spikes."""
    k, vr, vt, b = IZ["k"], IZ["vr"], IZ["vt"], IZ["b"]
    i_star = (k * (vt - vr) + b) ** 2 / (4.0 * k)
    assert i_star == pytest.approx(51.4286, abs=1e-3)
    for I in (30.0, i_star - 1.5):
        r = oracle.simulate(_lone(I), 60000, want_y=False)
        A, B, Cq = k, -(k * (vr + vt) + b), k * vr * vt + b * vr + I
        v_star = (-B - math.sqrt(B * B - 4 * A * Cq)) / (2 * A)
        assert r["ev_count"] == 0
        assert r["v"][0] == pytest.approx(v_star, abs=1e-7)
        assert r["w"][0] == pytest.approx(b * (v_star - vr), abs=1e-6)
    assert oracle.simulate(_lone(i_star + 1.5), 60000, want_y=False)["ev_count"] > 0


def test_spike_resets_v_and_kicks_w():
    """The step after V(n) >= V_peak: V = V_reset and W = W(n) + d exactly."""
    r = oracle.simulate(_lone(200.0), 4000, snap_every=1, want_y=False, ev_cap=1000)
    V, W = r["snap_v"][:, 0], r["snap_w"][:, 0]   # snapshot i = state at step i + 1
    spikes = np.nonzero(V >= IZ["vpeak"])[0]
    assert spikes.size >= 5
    assert np.array_equal(r["ev_step"], spikes + 1)
    for i in spikes[spikes + 1 < V.size]:
        assert V[i + 1] == IZ["vreset"] and W[i + 1] == W[i] + IZ["d"]


@pytest.mark.parametrize("T_ms", [3.0, 5.0, 20.0])
def test_alpha_psc_converges_to_the_alpha_function(T_ms):
    """An impulse p(0) = p0 gives r(t) = p0 t exp(-a t) in the continuous model
    (Eq. alphapsc); forward Euler is first order, so halving dt halves the error
    (checked away from t ~ 2 / a, where the first-order error term changes sign)."""
    a, p0 = IZ["psc_a"], 10.0
    exact = p0 * T_ms * math.exp(-a * T_ms)
    errs = []
    for dt in (0.02, 0.01):
        sp = _lone(0.0, dt=dt)
        n = int(round(T_ms / dt))
        r = oracle.simulate(sp, n, want_y=False,
                            init=dict(n0=0, v=[IZ["vr"]], w=[0.0], c=[0.0], r=[0.0], p=[p0], hist=np.zeros((1, 1))))
        errs.append(abs(r["r"][0] - exact))
    assert errs[0] < 0.02 * exact
    assert errs[0] / errs[1] == pytest.approx(2.0, rel=0.05)


def test_calcium_follows_the_spike_train():
    """c(n + 1) = c(n)(1 - dt / tau_c) + dt spd(V(n)) (Eq. casimple): the final c is the
    sum over spike steps e of dt (1 - dt / tau_c)^(n_end - e - 1), and the noise-free
    readout is gain c + offset at every sample."""
    sp = _lone(120.0)
    n_end = 6000
    r = oracle.simulate(sp, n_end, ev_cap=1000)
    dt, tau = sp.dt_ms, IZ["tau_c"]
    q = 1.0 - dt / tau
    c_ref = sum(dt * q ** (n_end - e - 1) for e in r["ev_step"] if e < n_end)
    assert r["ev_count"] >= 3
    assert r["c"][0] == pytest.approx(c_ref, rel=1e-12)
    every = sp.obs["sample_every"]
    k_last = n_end // every - 1
    c_last = sum(dt * q ** ((k_last + 1) * every - e - 1) for e in r["ev_step"] if e < (k_last + 1) * every)
    assert r["y_clean"][k_last, 0] == pytest.approx(sp.obs["gain"] * c_last + sp.obs["offset"], rel=1e-12)


def test_one_spike_reaches_its_target_after_the_delay():
    """Edge 0 -> 1 with D = 37 steps: the first spike of node 0 at step s0 leaves p_1 at
    0 through step s0 + D and sets it to dt w at step s0 + D + 1 (Eq. izpsc: the input
    reads spd(V_0(n - D)))."""
    D, w = 37, 3000.0
    sp = _lone(0.0, n=2, src=[0], dst=[1], w=[w], delay=[D], pulses=[(0, 1.0, 3.0, 2500.0)])
    r = oracle.simulate(sp, 400, want_y=False)
    s0 = int(r["ev_step"][0])
    assert r["ev_node"][0] == 0 and r["first_arrival"][0] == s0
    before = oracle.simulate(sp, s0 + D, want_y=False)
    after = oracle.simulate(sp, s0 + D + 1, want_y=False)
    assert before["p"][1] == 0.0 and before["r"][1] == 0.0
    assert after["p"][1] == sp.dt_ms * float(np.float32(w))


def test_izh_ring_equals_dense_history():
    """The circular history of depth D_max + 1 and the full [T][N] history (Eq. izpsc
    read by time index) give bit-identical runs on a spiking network."""
    sp = netgen.izhikevich(netgen.tiny(), w_scale=7000.0)
    a = oracle.simulate(sp, 4000, ev_cap=100000)
    b = oracle.simulate(sp, 4000, dense=True, ev_cap=100000)
    assert a["ev_count"] > 20
    for k in ("v", "w", "c", "r", "p", "y", "first_arrival", "ev_node", "ev_step"):
        assert np.array_equal(a[k], b[k]), k
