"""FP32 emulation of the FitzHugh-Nagumo network step -- TEST INFRASTRUCTURE.

A second, plain numpy implementation of the step the FP64 oracle evaluates
(Sec. 2 Eq. Yjset for the delayed input; Sec. 3.1 Euler form of the FHN pair about
the rest point; Sec. 3.3 the Euler form of the readout), in a dtype of the
caller's choice and with the delayed input summed in a chosen order.  It exists to
measure how far the same arithmetic drifts from FP64 when it is carried out in
FP32, independently of the CUDA library:

  * in float64 with the oracle's summation order it reproduces the oracle (every
    operation in the oracle's order, no contraction), which pins the emulation;
  * in float32 it shows how much of the difference between an FP32 trajectory and
    the FP64 one is the network's conditioning (the same step, only rounded
    differently) rather than the arithmetic of any one implementation.

Only explicit pulses are emulated (no background pulses).  Every operation is
rounded to the dtype, each product before it is added, as the GPU kernels do.
"""
from __future__ import annotations

import numpy as np

import oracle

ORDERS = ("oracle", "random", "reversed")


def _row_order(spec, order: str, seed: int):
    """[N, maxdeg] edge indices of each target's row in summation order (-1 pads).
    'oracle': the caller's edge order (the oracle's loop), 'reversed': that order
    backwards, 'random': a seeded permutation of each row."""
    dst = np.asarray(spec.dst)
    N = spec.n_nodes
    deg = np.bincount(dst, minlength=N)
    width = int(deg.max(initial=0))
    idx = -np.ones((N, max(1, width)), np.int64)
    rng = np.random.default_rng(seed)
    for j in range(N):
        e = np.nonzero(dst == j)[0]
        if order == "reversed":
            e = e[::-1]
        elif order == "random":
            e = rng.permutation(e)
        elif order != "oracle":
            raise ValueError(order)
        idx[j, :e.size] = e
    return idx


def oracle_trajectory(spec, n_steps: int):
    """The FP64 oracle's v~, w~, c~ at steps 0..n_steps ([n_steps + 1, N] each)."""
    ref = oracle.simulate(spec, n_steps, snap_every=1, want_y=False, ev_cap=1)
    z = np.zeros((1, spec.n_nodes))
    return {k: np.vstack([z, ref[f"snap_{k}"]]) for k in ("v", "w", "c")}


def emulate(spec, n_steps: int, dtype=np.float32, order: str = "oracle", seed: int = 0,
            window: int = 0, ref: dict | None = None):
    """Run the step n_steps times from rest in `dtype`; returns v~, w~, c~ at steps
    0..n_steps.  With `window` > 0 the state and the whole history are reloaded from
    the oracle's trajectory `ref` (rounded to `dtype`) at every multiple of
    `window`, as the windowed GPU parity tests reload the device."""
    if spec.background:
        raise ValueError("the emulation covers explicit pulses only")
    if spec.coupling != "rest":
        raise ValueError("the emulation covers the REST coupling only")
    dt = np.dtype(dtype).type
    N = spec.n_nodes
    D = oracle.net_delays(spec).astype(np.int64)
    src = np.asarray(spec.src, np.int64)
    wgt = np.asarray(spec.weight, np.float64).astype(dtype)
    idx = _row_order(spec, order, seed)
    fhn, obs = spec.fhn, spec.obs
    v_rest, _ = oracle.rest_point(fhn)
    a, b, c_, e, g = (dt(fhn[k]) for k in ("a", "b", "c", "e", "g"))
    h = dt(spec.dt_ms)
    k_obs = dt(spec.dt_ms / obs["tau_ms"])
    vr = dt(v_rest)
    three = dt(3.0)
    on = [oracle.ms_to_step(p[1], spec.dt_ms) for p in spec.pulses]
    off = [oracle.ms_to_step(p[2], spec.dt_ms) for p in spec.pulses]
    amp = [dt(float(np.float32(p[3]))) for p in spec.pulses]
    node = [int(p[0]) for p in spec.pulses]

    H = np.zeros((n_steps + 1, N), dtype)   # v~(t), t = 0 .. n_steps
    v = np.zeros(N, dtype)
    w = np.zeros(N, dtype)
    c = np.zeros(N, dtype)
    out = {k: np.zeros((n_steps + 1, N), dtype) for k in ("v", "w", "c")}
    for n in range(n_steps):
        if window and n % window == 0 and n > 0:
            v, w, c = (ref[k][n].astype(dtype) for k in ("v", "w", "c"))
            H[:n + 1] = ref["v"][:n + 1].astype(dtype)
        H[n] = v
        t = n - D
        past = np.where(t >= 0, H[np.maximum(t, 0), src], dt(0.0)).astype(dtype)
        prod = (wgt * past).astype(dtype)
        S = np.zeros(N, dtype)
        for k in range(idx.shape[1]):
            m = idx[:, k] >= 0
            S[m] = S[m] + prod[idx[m, k]]
        U = np.zeros(N, dtype)
        for j, n_on, n_off, A in zip(node, on, off, amp):
            if n_on <= n < n_off:
                U[j] = U[j] + A
        cubic = ((three * vr) * vr) * v + ((three * vr) * v) * v + (v * v) * v
        dv = a * v - b * cubic - c_ * w + S + U
        dw = e * (v - g * w)
        v1 = v + h * dv
        w1 = w + h * dw
        c1 = c + k_obs * (v1 - c)
        v, w, c = v1.astype(dtype), w1.astype(dtype), c1.astype(dtype)
        out["v"][n + 1], out["w"][n + 1], out["c"][n + 1] = v, w, c
    return out


def elementwise_ratio(x, ref, rel=1e-4, floor=1e-6):
    """Largest |x - ref| / max(rel |ref|, floor) (the parity tolerance; <= 1 passes)."""
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.max(np.abs(x - ref) / np.maximum(rel * np.abs(ref), floor)))


def trace_maxnorm(x, ref):
    """Per-trace max-norm relative error, max over traces: for node j,
    max_t |x_j(t) - ref_j(t)| / max_t |ref_j(t)|, over the traces that move."""
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    scale = np.abs(ref).max(0)
    moving = scale > 0
    if not moving.any():
        return 0.0
    return float((np.abs(x - ref).max(0)[moving] / scale[moving]).max())
