"""Helpers shared by the GPU parity tests: run the CUDA path and the FP64 oracle
on the same seeded network and compare them.

Tolerance (floating point): |gpu - oracle| <= max(1e-4 |oracle|, 1e-6) elementwise
on v~, w~, c~ and y.  The oracle runs its own uninterrupted FP64 trajectory; at the
start of every window of `window` steps (default one observation interval,
20 steps = 1 ms) the GPU is loaded with the oracle's state rounded to FP32
(gn_set_state) and its next `window` steps are compared with the oracle's.  Data
flows only from the oracle to the GPU.  Windows are needed because the excitable
dynamics amplify rounding: an FP32 emulation that changes nothing but the
summation order of S drifts 3e-4 away from FP64 over 200 ms, so a comparison
without windows measures the conditioning of the network, not the arithmetic of
the step (the unwindowed drift is reported by its own test).

Integers (delays, arrivals, background counters, events) must match exactly; an
event may differ only where the oracle's V is within 1e-5 of the threshold at the
crossing, where FP32 cannot decide it.
"""
from __future__ import annotations

import numpy as np

import oracle

REL, ABS = 1e-4, 1e-6
EVENT_MARGIN = 1e-5


def ratio(gpu, ref):
    """Largest |gpu - ref| / max(REL |ref|, ABS); <= 1 passes."""
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    if gpu.size == 0:
        return 0.0
    return float(np.max(np.abs(gpu - ref) / np.maximum(REL * np.abs(ref), ABS)))


def windowed(spec, net, n_steps, window=20, start=0, coupling=None):
    """Compare `net` with the oracle over steps [start, start + n_steps) window by
    window.  Returns the worst ratio per quantity and the number of oracle events;
    raises AssertionError on an integer mismatch."""
    D = oracle.net_delays(spec)
    depth = int(D.max(initial=1)) + 1
    ref = oracle.simulate(spec, start, coupling=coupling, hist_depth=depth, want_y=False)
    vr = ref["rest"][0]
    worst = dict(v=0.0, w=0.0, c=0.0, y=0.0)
    n_events = 0
    n0 = start
    end = start + n_steps
    while n0 < end:
        K = min(window, end - n0)
        net.gn_set_state(ref["hist"].astype(np.float32), ref["w"].astype(np.float32),
                         ref["c"].astype(np.float32), ref["bg_count"], n0)
        nxt = oracle.simulate(spec, K, coupling=coupling, hist_depth=depth, snap_every=1,
                              ev_cap=spec.n_nodes * (K // 2 + 1) + 1024,
                              init=dict(n0=n0, v=ref["v"], w=ref["w"], c=ref["c"], bg_count=ref["bg_count"],
                                        hist=ref["hist"]))
        net.gn_step(K)
        g = net.gn_get_state()
        y, _, _ = net.gn_observe()
        for k in ("v", "w", "c"):
            worst[k] = max(worst[k], ratio(g[k], nxt[k]))
        if nxt["y"].shape[0]:
            assert y.shape == nxt["y"].shape
            worst["y"] = max(worst["y"], ratio(y, nxt["y"]))
        assert np.array_equal(g["bg_count"], nxt["bg_count"]), f"background counters differ in [{n0}, {n0 + K})"
        # events of the window; mismatches only where V sits on the threshold
        V = vr + np.vstack([ref["v"][None, :], nxt["snap_v"]])
        near = (np.abs(V[:-1]) < EVENT_MARGIN) | (np.abs(V[1:]) < EVENT_MARGIN)
        t, j = np.nonzero(near)
        excused = set(zip(j.tolist(), (n0 + t + 1).tolist()))
        node, step, _ = net.gn_get_events()
        got = set(zip(node.tolist(), step.tolist()))
        assert nxt["ev_count"] == nxt["ev_node"].size, "oracle event buffer too small"
        want = set(zip(nxt["ev_node"].tolist(), nxt["ev_step"].tolist()))
        bad = [e for e in got ^ want if e not in excused]
        assert not bad, f"events differ in [{n0}, {n0 + K}): {bad[:5]}"
        n_events += len(want)
        ref = nxt
        n0 += K
    return worst, n_events


def assert_windows(worst):
    for k, r in worst.items():
        assert r <= 1.0, f"{k}: {r:.3g} x tolerance"


PEAK_MARGIN = 1e-2   # mV: a spike decision this close to V_peak may go either way in FP32
# Hodgkin-Huxley windows: 8 steps (0.24 ms at dt = 0.03 ms).  The upswing amplifies a
# perturbation fast enough that over one 33-step observation interval the rounding of
# the starting state to FP32 alone -- the oracle run from the rounded state against
# the oracle run from the exact one -- takes up to 0.57 of the tolerance on V; over
# 8 steps it takes at most 0.12, leaving the rest for the step's own arithmetic.
HH_WINDOW = 8


def ratio_scaled(gpu, ref):
    """ratio() for dimensional state (mV, pA): the absolute floor is 1e-6 of the
    quantity's largest magnitude, |gpu - ref| <= max(REL |ref|, ABS max(1, max |ref|)).
    For O(1) quantities this is ratio(); for V in mV it keeps the floor above one
    FP32 ulp of the membrane potential (3.8e-6 mV at 60 mV), where the 0 mV crossing
    of an upswing would otherwise be held to 1e-6 mV."""
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    if gpu.size == 0:
        return 0.0
    floor = ABS * max(1.0, float(np.max(np.abs(ref))))
    return float(np.max(np.abs(gpu - ref) / np.maximum(REL * np.abs(ref), floor)))


def windowed_izh(spec, net, n_steps, window=None, start=0):
    """windowed() for the spiking models (Izhikevich or Hodgkin-Huxley + alpha PSC):
    the oracle's full state (V, W, calcium, r, p, the Hodgkin-Huxley gates, spike
    history, background counters; with plasticity the weights and the history of
    s) is loaded at every window start and the next
    `window` steps of V, W, c, r, p, m, n, h, y (ratio_scaled) and the spikes are
    compared.  A node is left out of a window's comparison only if the oracle's V
    came within PEAK_MARGIN of V_peak in it (the spike decision is not defined to
    FP32 there), or if such a node reaches it through an edge of delay below the
    window length (its input then depends on that decision); the count of such
    node-windows is returned with the worst ratios.  The window defaults to one
    observation interval (1 ms: 20 steps at dt = 0.05 ms, one step at dt = 1 ms,
    where a spike's upswing amplifies a perturbation more than twofold per step),
    and to HH_WINDOW steps for Hodgkin-Huxley."""
    hh = spec.model == "hh"
    window = window or (HH_WINDOW if hh else spec.obs["sample_every"])
    D = oracle.net_delays(spec)
    src, dst = np.asarray(spec.src), np.asarray(spec.dst)
    depth = int(D.max(initial=1)) + 1
    ref = oracle.simulate(spec, start, hist_depth=depth, want_y=False)
    worst = dict(v=0.0, w=0.0, c=0.0, r=0.0, p=0.0, y=0.0)
    if hh:
        worst.update(m=0.0, n=0.0, h=0.0)
    plastic = getattr(spec, "stdp", None) is not None
    if plastic:
        worst.update(weight=0.0, s=0.0)
    n_spikes = excused = 0
    n0 = start
    end = start + n_steps
    while n0 < end:
        K = min(window, end - n0)
        net.gn_set_state(ref["hist"].astype(np.float32), ref["w"].astype(np.float32),
                         ref["c"].astype(np.float32), ref["bg_count"], n0)
        net.gn_set_izh_state(V=ref["v"].astype(np.float32), r=ref["r"].astype(np.float32),
                             p=ref["p"].astype(np.float32))
        gates = {}
        if hh:
            gates = dict(m=ref["m"], n=ref["n"], h=ref["h"])
            net.gn_set_hh_gates(**{k: x.astype(np.float32) for k, x in gates.items()})
        if plastic:
            w_now = np.asarray(spec.weight, np.float64) if ref["w_final"] is None else ref["w_final"]
            net.gn_set_stdp_history(ref["hist_s"].astype(np.float32))
            net.gn_set_weights(w_now.astype(np.float32))
            gates.update(w_edge=w_now, s=ref["s"], hist_s=ref["hist_s"])
        nxt = oracle.simulate(spec, K, hist_depth=depth, ev_cap=spec.n_nodes * (K + 1) + 1024,
                              init=dict(n0=n0, v=ref["v"], w=ref["w"], c=ref["c"], r=ref["r"], p=ref["p"],
                                        bg_count=ref["bg_count"], hist=ref["hist"], **gates))
        net.gn_step(K)
        g = net.gn_get_state()
        gi = net.gn_get_izh_state()
        if hh:
            gg = net.gn_get_hh_gates()
        y, _, _ = net.gn_observe()
        ok = nxt["min_peak_gap"] > PEAK_MARGIN
        # a spike decision left open also changes, within the window, the input of
        # the targets it reaches in fewer than K steps
        reach = ~ok[src] & (D < K)
        ok[dst[reach]] = False
        excused += int((~ok).sum())
        for k, gv, rv in (("v", gi["V"], nxt["v"]), ("w", g["w"], nxt["w"]), ("c", g["c"], nxt["c"]),
                          ("r", gi["r"], nxt["r"]), ("p", gi["p"], nxt["p"])):
            worst[k] = max(worst[k], ratio_scaled(gv[ok], rv[ok]))
        if hh:
            for k in ("m", "n", "h"):
                worst[k] = max(worst[k], ratio_scaled(gg[k][ok], nxt[k][ok]))
        if plastic:
            ok_e = ok[src] & ok[dst]
            worst["weight"] = max(worst["weight"], ratio_scaled(net.gn_get_weights()[ok_e], nxt["w_final"][ok_e]))
            worst["s"] = max(worst["s"], ratio_scaled(net.gn_get_stdp_history(1)[0][ok], nxt["s"][ok]))
        if nxt["y"] is not None and nxt["y"].size:
            worst["y"] = max(worst["y"], ratio_scaled(y[:, ok], nxt["y"][:, ok]))
        assert np.array_equal(g["bg_count"], nxt["bg_count"]), "background counters differ"
        gn_nodes, gn_steps, _ = net.gn_get_events()
        ref_ev = {(int(a), int(b)) for a, b in zip(nxt["ev_node"], nxt["ev_step"]) if ok[a]}
        got_ev = {(int(a), int(b)) for a, b in zip(gn_nodes, gn_steps) if ok[a]}
        assert got_ev == ref_ev, f"spikes differ in window starting at {n0}: {sorted(got_ev ^ ref_ev)[:10]}"
        n_spikes += len(ref_ev)
        ref = nxt
        n0 += K
    return worst, n_spikes, excused
