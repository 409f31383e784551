"""FP64 oracle of the delayed geometric-network simulation (Buibas & Silva,
arXiv:0908.3934) -- TEST INFRASTRUCTURE.

Only the test-suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product library (``paper_0908_3934_b300``) never imports it, and it never
imports the product: the two sides share only the seeded input generators
(``paper_0908_3934_b300.netgen``), which hold none of the method's arithmetic.

The simulator itself is plain C in ``oracle.c`` (FP64, no FMA contraction),
loaded with ctypes; the connectivity estimator's oracle is plain numpy in
``estimator.py``.  See the header of ``oracle.c`` for what is computed and
which passage of the paper each part follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` with gcc (FP64, no FMA contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math",
             "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Net(C.Structure):
    _fields_ = [
        ("n_nodes", C.c_int32), ("n_edges", C.c_int64),
        ("src", C.c_void_p), ("dst", C.c_void_p), ("weight", C.c_void_p), ("delay", C.c_void_p),
        ("dt_ms", C.c_double),
        ("a", C.c_double), ("b", C.c_double), ("c", C.c_double), ("e", C.c_double),
        ("f", C.c_double), ("g", C.c_double), ("i_ext", C.c_double),
        ("coupling", C.c_int32), ("theta", C.c_double),
        ("tau_ms", C.c_double), ("sample_every", C.c_int32),
        ("gain", C.c_double), ("offset", C.c_double), ("sigma", C.c_double), ("obs_seed", C.c_uint64),
        ("n_pulses", C.c_int32), ("p_node", C.c_void_p), ("p_on", C.c_void_p), ("p_off", C.c_void_p),
        ("p_amp", C.c_void_p),
        ("bg_threshold", C.c_uint32), ("bg_amp", C.c_double), ("bg_width", C.c_int32),
        ("bg_seed", C.c_uint64),
        ("model", C.c_int32),
        ("iz_C", C.c_double), ("iz_k", C.c_double), ("iz_vr", C.c_double), ("iz_vt", C.c_double),
        ("iz_vpeak", C.c_double), ("iz_vreset", C.c_double), ("iz_a", C.c_double), ("iz_b", C.c_double),
        ("iz_d", C.c_double), ("iz_iext", C.c_double), ("psc_a", C.c_double), ("tau_c", C.c_double),
        ("hh_C", C.c_double), ("hh_gna", C.c_double), ("hh_gk", C.c_double), ("hh_gl", C.c_double),
        ("hh_ena", C.c_double), ("hh_ek", C.c_double), ("hh_el", C.c_double), ("hh_vpeak", C.c_double),
        ("hh_iext", C.c_double),
        ("stdp", C.c_int32), ("stdp_alpha", C.c_double), ("stdp_beta", C.c_double),
        ("frame_average", C.c_int32),
        ("n_types", C.c_int32), ("types", C.c_void_p), ("cell_type", C.c_void_p),
    ]


class _Init(C.Structure):
    _fields_ = [
        ("n0", C.c_int64), ("v", C.c_void_p), ("w", C.c_void_p), ("c", C.c_void_p),
        ("bg_count", C.c_void_p), ("hist", C.c_void_p), ("hist_depth", C.c_int32),
        ("r", C.c_void_p), ("p", C.c_void_p),
        ("m", C.c_void_p), ("n", C.c_void_p), ("h", C.c_void_p),
        ("w_edge", C.c_void_p), ("s", C.c_void_p), ("hist_s", C.c_void_p),
    ]


class _Out(C.Structure):
    _fields_ = [
        ("v", C.c_void_p), ("w", C.c_void_p), ("c", C.c_void_p),
        ("y", C.c_void_p), ("y_clean", C.c_void_p),
        ("first_arrival", C.c_void_p), ("first_value", C.c_void_p),
        ("ev_node", C.c_void_p), ("ev_step", C.c_void_p), ("ev_cap", C.c_int64), ("ev_count", C.c_int64),
        ("snap_every", C.c_int32),
        ("snap_v", C.c_void_p), ("snap_w", C.c_void_p), ("snap_c", C.c_void_p), ("bg_count", C.c_void_p),
        ("hist_out", C.c_void_p), ("hist_out_depth", C.c_int32),
        ("r", C.c_void_p), ("p", C.c_void_p),
        ("m", C.c_void_p), ("n", C.c_void_p), ("h", C.c_void_p), ("min_peak_gap", C.c_void_p),
        ("w_final", C.c_void_p), ("s", C.c_void_p), ("hist_s_out", C.c_void_p),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            L.orc_philox4x32_10.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
            L.orc_gauss.argtypes = [C.c_uint64, C.c_uint32, C.c_int64]
            L.orc_gauss.restype = C.c_double
            L.orc_bg_threshold.argtypes = [C.c_double, C.c_double]
            L.orc_bg_threshold.restype = C.c_uint32
            L.orc_bg_onset.argtypes = [C.c_uint64, C.c_uint32, C.c_int64, C.c_uint32]
            L.orc_rest_point.argtypes = [C.c_double] * 6 + [C.POINTER(C.c_double)] * 2
            L.orc_delays.argtypes = [C.c_int32, C.c_int32, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                     C.c_void_p, C.c_double, C.c_double, C.c_void_p, C.c_void_p]
            L.orc_ms_to_step.argtypes = [C.c_double, C.c_double]
            L.orc_ms_to_step.restype = C.c_int64
            L.orc_simulate.argtypes = [C.POINTER(_Net), C.c_int64, C.POINTER(_Out)]
            L.orc_simulate_dense.argtypes = [C.POINTER(_Net), C.c_int64, C.POINTER(_Out)]
            L.orc_simulate_from.argtypes = [C.POINTER(_Net), C.POINTER(_Init), C.c_int64, C.POINTER(_Out)]
            L.orc_hh_rest_gates.argtypes = [C.POINTER(C.c_double)] * 3
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def philox4x32_10(ctr, key):
    """Philox4x32-10 block function (Salmon et al., SC'11) on one counter."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return o


def gauss(seed: int, node: int, sample: int) -> float:
    """The observation noise xi(seed, node, sample) ~ N(0, 1)."""
    return lib().orc_gauss(seed, node, sample)


def bg_threshold(rate_hz: float, dt_ms: float) -> int:
    return int(lib().orc_bg_threshold(rate_hz, dt_ms))


def bg_onset(seed: int, node: int, step: int, threshold: int) -> bool:
    return bool(lib().orc_bg_onset(seed, node, step, threshold))


def rest_point(fhn: dict):
    """(V*, W*) of the isolated FHN node in the paper's notation (Sec. 3.1)."""
    v = C.c_double()
    w = C.c_double()
    rc = lib().orc_rest_point(fhn["a"], fhn["b"], fhn["c"], fhn["f"], fhn["g"], fhn["i_ext"],
                              C.byref(v), C.byref(w))
    if rc != 0:
        raise ValueError("FHN parameters have no unique rest point (need a < c/g)")
    return v.value, w.value


def delays(pos, src, dst, speed, speed_scalar, dt_ms):
    """Whole-step delays D = max(1, llround(|x_i - x_j| / (s dt))) per edge and the clamp flags."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    n, dim = pos.shape
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    sp = None if speed is None else np.ascontiguousarray(speed, dtype=np.float64)
    E = src.shape[0]
    D = np.zeros(E, np.int32)
    cl = np.zeros(E, np.uint8)
    rc = lib().orc_delays(n, dim, _ptr(pos), E, _ptr(src), _ptr(dst), _ptr(sp),
                          float(speed_scalar or 0.0), dt_ms, _ptr(D), _ptr(cl))
    if rc != 0:
        raise ValueError("invalid delay inputs")
    return D, cl.astype(bool)


def ms_to_step(t_ms: float, dt_ms: float) -> int:
    """Whole step of a time in ms: llround(t/dt), half away from zero."""
    return int(lib().orc_ms_to_step(t_ms, dt_ms))


def hh_rest_gates():
    """Hodgkin-Huxley gates m, n, h at rest (-65 mV): alpha / (alpha + beta)."""
    m, n, h = C.c_double(), C.c_double(), C.c_double()
    lib().orc_hh_rest_gates(C.byref(m), C.byref(n), C.byref(h))
    return m.value, n.value, h.value


def net_delays(spec) -> np.ndarray:
    """Delay table of a generated network: explicit if given, else geometric."""
    if spec.delay is not None:
        return np.ascontiguousarray(spec.delay, dtype=np.int32)
    D, _ = delays(spec.pos, spec.src, spec.dst, spec.speed, spec.speed_scalar, spec.dt_ms)
    return D


def simulate(spec, n_steps: int, *, dense: bool = False, snap_every: int = 0,
             ev_cap: int = 1 << 16, want_y: bool = True, coupling: str | None = None,
             init: dict | None = None, delay: np.ndarray | None = None, hist_depth: int = 0):
    """Run the FP64 oracle for ``n_steps`` steps of ``dt``.

    ``spec`` is a ``paper_0908_3934_b300.netgen.NetSpec``.  The run starts from
    rest at step 0, or, with ``init = dict(n0, v, w, c, bg_count, hist)``, from
    that state at step n0 (``hist[k, j]`` = v~_j(n0 - k)).  Returns a dict with
    the final state relative to rest (v, w, c), background counters, observations
    y / y_clean [n_samples, N] for the samples taken inside the run, first_arrival /
    first_value [N], events (node, step), if ``snap_every`` > 0 state snapshots
    [n_steps // snap_every, N], and if ``hist_depth`` > 0 the final history
    ``hist[k, j]`` = v~_j(n_end - k), k < hist_depth (at most D_max + 1).

    With ``spec.model == "izh"`` (Izhikevich + alpha PSC + calcium) the state is
    absolute (v = V, w = W, c = calcium, plus r, p returned and accepted in
    ``init``), the history holds spd(V) in {0, 1}, events are spikes, the arrival
    of a node is its first spike, and ``min_peak_gap`` [N] is the smallest
    |V - V_peak| seen during the run.  With ``spec.model == "hh"`` (Hodgkin-Huxley
    + alpha PSC + calcium) the same holds with W = 0, the gates m, n, h returned
    (and accepted in ``init``), and events the upward crossings of V_peak.

    With ``spec.stdp = dict(alpha, beta)`` (spiking models) the weights evolve by the
    plasticity transition: the result adds ``w_final`` [E] (caller edge order), ``s``
    [N] (time since the last spike) and, with ``hist_depth``, ``hist_s`` [k, j] =
    s_j(n_end - k); ``init`` accepts ``w_edge``, ``s`` and ``hist_s``.
    """
    L = lib()
    N = spec.n_nodes
    E = spec.n_edges
    D = net_delays(spec) if delay is None else np.ascontiguousarray(delay, np.int32)
    src = np.ascontiguousarray(spec.src, np.int32)
    dst = np.ascontiguousarray(spec.dst, np.int32)
    wgt = np.ascontiguousarray(spec.weight, np.float64)
    fhn = spec.fhn
    obs = spec.obs
    pulses = spec.pulses or []
    p_node = np.array([p[0] for p in pulses], np.int32)
    p_on = np.array([ms_to_step(p[1], spec.dt_ms) for p in pulses], np.int64)
    p_off = np.array([ms_to_step(p[2], spec.dt_ms) for p in pulses], np.int64)
    p_amp = np.array([float(np.float32(p[3])) for p in pulses], np.float64)
    bg = spec.background
    cpl = coupling or spec.coupling
    izh = spec.model == "izh"
    hh = spec.model == "hh"
    spiking = izh or hh
    iz = spec.izh
    hp = getattr(spec, "hh", None) or {}
    # the PSC rate and calcium time are shared by the spiking models
    psc = hp if hh else iz
    stdp = getattr(spec, "stdp", None)
    ctypes_ = getattr(spec, "cell_types", None)
    if ctypes_:
        keys = ("C", "gna", "gk", "gl", "ena", "ek", "el", "vpeak", "i_ext", "psc_a", "tau_c") if hh else \
               ("C", "k", "vr", "vt", "vpeak", "vreset", "a", "b", "d", "i_ext", "psc_a", "tau_c")
        type_tab = np.array([[t[k] for k in keys] for t in ctypes_], np.float64)
        cell_type = np.ascontiguousarray(spec.cell_type, np.uint8)
    else:
        type_tab = cell_type = None
    net = _Net(
        n_nodes=N, n_edges=E, src=_ptr(src), dst=_ptr(dst), weight=_ptr(wgt), delay=_ptr(D),
        dt_ms=spec.dt_ms, a=fhn["a"], b=fhn["b"], c=fhn["c"], e=fhn["e"], f=fhn["f"], g=fhn["g"],
        i_ext=fhn["i_ext"], coupling=1 if cpl == "raw" else 0, theta=spec.theta,
        tau_ms=obs["tau_ms"], sample_every=obs["sample_every"],
        gain=float(np.float32(obs["gain"])), offset=float(np.float32(obs["offset"])),
        sigma=float(np.float32(obs["sigma"])), obs_seed=obs["seed"],
        n_pulses=len(pulses), p_node=_ptr(p_node), p_on=_ptr(p_on), p_off=_ptr(p_off), p_amp=_ptr(p_amp),
        bg_threshold=bg_threshold(bg["rate_hz"], spec.dt_ms) if bg else 0,
        bg_amp=float(np.float32(bg["amp"])) if bg else 0.0,
        bg_width=ms_to_step(bg["dur_ms"], spec.dt_ms) if bg else 0,
        bg_seed=bg["seed"] if bg else 0,
        model=2 if hh else 1 if izh else 0,
        iz_C=iz["C"], iz_k=iz["k"], iz_vr=iz["vr"], iz_vt=iz["vt"], iz_vpeak=iz["vpeak"],
        iz_vreset=iz["vreset"], iz_a=iz["a"], iz_b=iz["b"], iz_d=iz["d"], iz_iext=iz["i_ext"],
        psc_a=psc["psc_a"], tau_c=psc["tau_c"],
        **({f"hh_{k}": hp[k] for k in ("C", "gna", "gk", "gl", "ena", "ek", "el", "vpeak")} if hh else {}),
        hh_iext=hp.get("i_ext", 0.0),
        stdp=1 if stdp else 0, stdp_alpha=stdp["alpha"] if stdp else 0.0, stdp_beta=stdp["beta"] if stdp else 0.0,
        frame_average=1 if obs.get("frame_average") else 0,
        n_types=len(ctypes_) if ctypes_ else 0, types=_ptr(type_tab), cell_type=_ptr(cell_type),
    )
    v = np.zeros(N)
    w = np.zeros(N)
    c = np.zeros(N)
    n0 = int(init["n0"]) if init else 0
    every = obs["sample_every"]
    n_samples = (n0 + n_steps) // every - n0 // every
    y = np.zeros((n_samples, N)) if want_y else None
    yc = np.zeros((n_samples, N)) if want_y else None
    fa = np.zeros(N, np.int32)
    fv = np.zeros(N)
    evn = np.zeros(ev_cap, np.int32)
    evs = np.zeros(ev_cap, np.int64)
    n_snap = n_steps // snap_every if snap_every > 0 else 0
    sv = np.zeros((n_snap, N)) if n_snap else None
    sw = np.zeros((n_snap, N)) if n_snap else None
    sc = np.zeros((n_snap, N)) if n_snap else None
    bgc = np.zeros(N, np.int32)
    hout = np.zeros((hist_depth, N)) if hist_depth > 0 else None
    r_out = np.zeros(N)
    p_out = np.zeros(N)
    gates = [np.zeros(N) for _ in range(3)]
    gap = np.zeros(N)
    w_fin = np.array(wgt) if stdp else None
    s_out = np.zeros(N) if stdp else None
    hs_out = np.zeros((hist_depth, N)) if stdp and hist_depth > 0 else None
    out = _Out(w_final=_ptr(w_fin), s=_ptr(s_out), hist_s_out=_ptr(hs_out),v=_ptr(v), w=_ptr(w), c=_ptr(c), y=_ptr(y), y_clean=_ptr(yc), bg_count=_ptr(bgc),
               r=_ptr(r_out), p=_ptr(p_out), min_peak_gap=_ptr(gap) if spiking else None,
               m=_ptr(gates[0]), n=_ptr(gates[1]), h=_ptr(gates[2]),
               hist_out=_ptr(hout), hist_out_depth=hist_depth,
               first_arrival=_ptr(fa), first_value=_ptr(fv), ev_node=_ptr(evn), ev_step=_ptr(evs),
               ev_cap=ev_cap, ev_count=0, snap_every=snap_every if n_snap else 0,
               snap_v=_ptr(sv), snap_w=_ptr(sw), snap_c=_ptr(sc))
    if init is not None:
        keep = []

        def arr(x, dt):
            a = None if x is None else np.ascontiguousarray(x, dt)
            keep.append(a)
            return _ptr(a)
        hist = np.ascontiguousarray(init["hist"], np.float64)
        ini = _Init(n0=n0, v=arr(init["v"], np.float64), w=arr(init["w"], np.float64),
                    c=arr(init["c"], np.float64), bg_count=arr(init.get("bg_count"), np.int32),
                    hist=_ptr(hist), hist_depth=hist.shape[0],
                    r=arr(init.get("r"), np.float64), p=arr(init.get("p"), np.float64),
                    m=arr(init.get("m"), np.float64), n=arr(init.get("n"), np.float64),
                    h=arr(init.get("h"), np.float64), w_edge=arr(init.get("w_edge"), np.float64),
                    s=arr(init.get("s"), np.float64), hist_s=arr(init.get("hist_s"), np.float64))
        rc = L.orc_simulate_from(C.byref(net), C.byref(ini), n_steps, C.byref(out))
    else:
        fn = L.orc_simulate_dense if dense else L.orc_simulate
        rc = fn(C.byref(net), n_steps, C.byref(out))
    if rc != 0:
        raise ValueError(f"oracle rejected the network (status {rc})")
    ne = min(out.ev_count, ev_cap)
    return dict(v=v, w=w, c=c, y=y, y_clean=yc, first_arrival=fa, first_value=fv,
                ev_node=evn[:ne].copy(), ev_step=evs[:ne].copy(), ev_count=out.ev_count,
                snap_v=sv, snap_w=sw, snap_c=sc, bg_count=bgc, hist=hout, n_end=n0 + n_steps,
                delay=D, rest=None if spiking else rest_point(fhn), r=r_out, p=p_out,
                min_peak_gap=gap if spiking else None, m=gates[0], n=gates[1], h=gates[2],
                w_final=w_fin, s=s_out, hist_s=hs_out)
