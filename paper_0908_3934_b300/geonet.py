"""ctypes binding of libgeonet.so (include/geonet.h): the same names, argument
marshalling only.  Every step of the simulation runs in the library's CUDA
kernels; nothing here computes.

The library is built in-tree by ``python -m paper_0908_3934_b300.build``;
loading raises ``RuntimeError`` if it is missing -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgeonet.so")

GN_OK, GN_EINVAL, GN_ENOMEM, GN_ERANGE, GN_ECUDA, GN_ESTATE, GN_ETIMEOUT, GN_EINTERNAL, GN_EOVERFLOW = (
    0, -1, -2, -3, -4, -5, -6, -7, -8)
STATUS_NAMES = {0: "GN_OK", -1: "GN_EINVAL", -2: "GN_ENOMEM", -3: "GN_ERANGE", -4: "GN_ECUDA", -5: "GN_ESTATE",
                -6: "GN_ETIMEOUT", -7: "GN_EINTERNAL", -8: "GN_EOVERFLOW"}
GN_COUPLE_REST, GN_COUPLE_RAW = 0, 1


class GeonetError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class gn_fhn_params(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("a", "b", "c", "e", "f", "g", "i_ext")]


class gn_obs_params(C.Structure):
    _fields_ = [("tau_ms", C.c_double), ("sample_every", C.c_int32), ("gain", C.c_float),
                ("offset", C.c_float), ("sigma", C.c_float), ("seed", C.c_uint64), ("frame_average", C.c_int32)]


class gn_izh_params(C.Structure):
    _fields_ = [(x, C.c_double) for x in ("C", "k", "v_r", "v_t", "v_peak", "v_reset", "a", "b", "d", "i_ext",
                                          "psc_a", "tau_c")]


class gn_hh_params(C.Structure):
    _fields_ = [(x, C.c_double) for x in ("C", "g_na", "g_k", "g_l", "e_na", "e_k", "e_l", "v_peak", "i_ext",
                                          "psc_a", "tau_c")]


class gn_stdp_params(C.Structure):
    _fields_ = [("enable", C.c_int32), ("alpha", C.c_double), ("beta", C.c_double)]


GN_MODEL_FHN, GN_MODEL_IZH, GN_MODEL_HH = 0, 1, 2
_MODELS = {"fhn": GN_MODEL_FHN, "izh": GN_MODEL_IZH, "hh": GN_MODEL_HH}


class gn_net_desc(C.Structure):
    _fields_ = [
        ("n_nodes", C.c_int32), ("dim", C.c_int32), ("pos", C.c_void_p), ("n_edges", C.c_int64),
        ("src", C.c_void_p), ("dst", C.c_void_p), ("weight", C.c_void_p), ("speed", C.c_void_p),
        ("speed_scalar", C.c_double), ("delay_steps", C.c_void_p), ("dt_ms", C.c_double),
        ("fhn", gn_fhn_params), ("obs", gn_obs_params), ("coupling", C.c_int32), ("theta", C.c_double),
        ("ring_depth", C.c_int32), ("obs_capacity", C.c_int64), ("event_capacity", C.c_int64),
        ("renumber", C.c_int32), ("edge_format", C.c_int32), ("step_kernel", C.c_int32),
        ("cuda_stream", C.c_void_p), ("device", C.c_int32),
        ("model", C.c_int32), ("izh", gn_izh_params), ("hh", gn_hh_params), ("stdp", gn_stdp_params),
        ("n_cell_types", C.c_int32), ("izh_types", C.c_void_p), ("hh_types", C.c_void_p), ("cell_type", C.c_void_p),
    ]


class gn_pulse(C.Structure):
    _fields_ = [("node", C.c_int32), ("t_on_ms", C.c_double), ("t_off_ms", C.c_double), ("amp", C.c_float)]


class gn_batch_info(C.Structure):
    _fields_ = [("n_nets", C.c_int32), ("n_nodes", C.c_int64), ("n_edges", C.c_int64), ("step", C.c_int64),
                ("cta_threads", C.c_int32), ("grid", C.c_int32), ("device_bytes", C.c_size_t),
                ("step_kernel", C.c_int32), ("step_groups", C.c_int32),
                ("step_lanes", C.c_int32)]


class gn_net_info(C.Structure):
    _fields_ = [
        ("n_nodes", C.c_int32), ("n_edges", C.c_int64), ("dim", C.c_int32), ("ring_depth", C.c_int32),
        ("max_delay", C.c_int32), ("min_delay", C.c_int32), ("n_clamped", C.c_int64),
        ("edge_format", C.c_int32), ("n_blocks", C.c_int32), ("step_kernel", C.c_int32),
        ("step_threads", C.c_int32), ("step_edges_per_thread", C.c_int32), ("grid", C.c_int32),
        ("step", C.c_int64), ("samples", C.c_int64),
        ("v_rest", C.c_double), ("w_rest", C.c_double), ("device_bytes", C.c_size_t),
        ("step_gathers", C.c_int64), ("step_entries", C.c_int64), ("step_lane_slots", C.c_int64),
        ("step_cluster", C.c_int32),
    ]


_P = C.c_void_p
_SIGS = {
    "gn_net_create": ([C.POINTER(gn_net_desc), C.POINTER(C.c_void_p)], C.c_int),
    "gn_net_destroy": ([_P], C.c_int),
    "gn_net_get_info": ([_P, C.POINTER(gn_net_info)], C.c_int),
    "gn_get_delays": ([_P, _P], C.c_int),
    "gn_get_rest": ([_P, C.POINTER(C.c_double), C.POINTER(C.c_double)], C.c_int),
    "gn_set_stimulus": ([_P, C.POINTER(gn_pulse), C.c_int32], C.c_int),
    "gn_set_background": ([_P, C.c_double, C.c_float, C.c_double, C.c_uint64], C.c_int),
    "gn_step": ([_P, C.c_int64], C.c_int),
    "gn_synchronize": ([_P], C.c_int),
    "gn_observe": ([_P, _P, C.c_int64, C.POINTER(C.c_int64), C.POINTER(C.c_int64)], C.c_int),
    "gn_observe_async": ([_P, _P, C.c_int64, C.POINTER(C.c_int64), C.POINTER(C.c_int64)], C.c_int),
    "gn_observe_wait": ([_P], C.c_int),
    "gn_get_state": ([_P, _P, _P, _P, _P, C.POINTER(C.c_int64)], C.c_int),
    "gn_get_history": ([_P, _P, C.c_int32], C.c_int),
    "gn_set_state": ([_P, _P, C.c_int32, _P, _P, _P, C.c_int64], C.c_int),
    "gn_get_izh_state": ([_P, _P, _P, _P], C.c_int),
    "gn_set_izh_state": ([_P, _P, _P, _P], C.c_int),
    "gn_get_hh_gates": ([_P, _P, _P, _P], C.c_int),
    "gn_get_weights": ([_P, _P], C.c_int),
    "gn_set_weights": ([_P, _P], C.c_int),
    "gn_get_stdp_history": ([_P, _P, C.c_int32], C.c_int),
    "gn_set_stdp_history": ([_P, _P, C.c_int32], C.c_int),
    "gn_set_hh_gates": ([_P, _P, _P, _P], C.c_int),
    "gn_get_arrivals": ([_P, _P], C.c_int),
    "gn_get_events": ([_P, _P, _P, C.c_int64, C.POINTER(C.c_int64)], C.c_int),
    "gn_save_state": ([_P, _P, C.c_size_t, C.POINTER(C.c_size_t)], C.c_int),
    "gn_load_state": ([_P, _P, C.c_size_t], C.c_int),
    "gn_last_error": ([], C.c_char_p),
    "gn_batch_create": ([C.POINTER(gn_net_desc), C.c_int32, C.POINTER(C.c_void_p)], C.c_int),
    "gn_batch_destroy": ([_P], C.c_int),
    "gn_batch_get_info": ([_P, _P], C.c_int),
    "gn_batch_get_net_info": ([_P, C.c_int32, C.POINTER(gn_net_info)], C.c_int),
    "gn_batch_get_delays": ([_P, C.c_int32, _P], C.c_int),
    "gn_batch_set_stimulus_all": ([_P, _P, _P], C.c_int),
    "gn_batch_set_background": ([_P, C.c_int32, C.c_double, C.c_float, C.c_double, C.c_uint64], C.c_int),
    "gn_batch_step": ([_P, C.c_int64], C.c_int),
    "gn_batch_step_static": ([_P, C.c_int64], C.c_int),
    "gn_batch_synchronize": ([_P], C.c_int),
    "gn_batch_observe": ([_P, C.c_int32, _P, C.c_int64, C.POINTER(C.c_int64), C.POINTER(C.c_int64)], C.c_int),
    "gn_batch_get_state": ([_P, C.c_int32, _P, _P, _P, _P, C.POINTER(C.c_int64)], C.c_int),
    "gn_batch_get_history": ([_P, C.c_int32, _P, C.c_int32], C.c_int),
    "gn_batch_get_izh_state": ([_P, C.c_int32, _P, _P, _P], C.c_int),
    "gn_batch_get_hh_gates": ([_P, C.c_int32, _P, _P, _P], C.c_int),
    "gn_batch_get_arrivals": ([_P, C.c_int32, _P], C.c_int),
    "gn_batch_get_events": ([_P, C.c_int32, _P, _P, C.c_int64, C.POINTER(C.c_int64)], C.c_int),
    "gn_batch_set_step": ([_P, C.c_int64], C.c_int),
    "gn_batch_set_state": ([_P, C.c_int32, _P, C.c_int32, _P, _P, _P], C.c_int),
    "gn_batch_export_traces": ([_P, C.c_int64, C.c_int32, _P], C.c_int),
    "gn_xcorr_features": ([_P, C.c_int64, C.c_int32, _P, C.c_int32, C.c_int64, _P, _P, _P, C.c_double, C.c_double,
                           _P, _P, _P], C.c_int),
    "gn_score_auroc": ([_P, _P, C.c_int64, C.POINTER(C.c_double)], C.c_int),
    "gn_score_f1": ([_P, _P, C.c_int64, C.c_double, C.POINTER(C.c_double)], C.c_int),
    "gn_score_best_f1": ([_P, _P, C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_double)], C.c_int),
    "gn_mlp_create": ([C.c_int32, C.c_int32, _P, C.c_int32, _P, C.POINTER(C.c_void_p)], C.c_int),
    "gn_mlp_destroy": ([_P], C.c_int),
    "gn_mlp_get_params": ([_P, _P], C.c_int),
    "gn_mlp_gradients": ([_P, _P, _P, _P, C.c_int32, _P, C.POINTER(C.c_float)], C.c_int),
    "gn_mlp_train_step": ([_P, _P, _P, _P, C.c_int32, C.c_float, C.c_float, C.POINTER(C.c_float)], C.c_int),
    "gn_mlp_train_epoch": ([_P, _P, _P, _P, C.c_int32, C.c_int32, C.c_float, C.c_float, _P], C.c_int),
    "gn_mlp_infer": ([_P, _P, C.c_int64, _P], C.c_int),
    "gn_mlp_synchronize": ([_P], C.c_int),
}

_lib = None


def lib() -> C.CDLL:
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_0908_3934_b300.build`")
        L = C.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def check(status: int, allow=()):
    if status != GN_OK and status not in allow:
        raise GeonetError(status, lib().gn_last_error().decode())
    return status


def _ptr(a):
    return None if a is None else a.ctypes.data


def _c(a, dt):
    return None if a is None else np.ascontiguousarray(a, dtype=dt)


def _vec(a, dt, n: int, name: str):
    """A caller's input of n values as a contiguous array of dtype dt (None stays
    None, the library's "leave unchanged"): checked before the library reads it."""
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=dt).reshape(-1)
    if a.size != n:
        raise ValueError(f"{name} has {a.size} values, {n} expected")
    return a


def _rows_in(a, n: int, name: str):
    """A caller's input of k >= 1 rows of n float32 values (history rows)."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.ndim != 2 or a.shape[0] < 1 or a.shape[1] != n:
        raise ValueError(f"{name} must have shape (k >= 1, {n}), got {a.shape}")
    return a


def _out_rows(out, rows: int, cols: int):
    """A caller's output buffer for `rows` rows of `cols` float32 values: checked
    before the library writes into it."""
    if not (isinstance(out, np.ndarray) and out.dtype == np.float32 and out.flags.c_contiguous
            and out.flags.writeable):
        raise ValueError("out must be a writable C-contiguous float32 array")
    if out.size < max(0, rows) * cols:
        raise ValueError(f"out holds {out.size} values, {max(0, rows)} rows of {cols} need more")
    return out


def make_desc(spec, keep: list, *, device: int = 0, stream=None, obs_capacity: int = 0, event_capacity: int = 0,
              renumber: bool = True, ring_depth: int | None = None, coupling: str | None = None,
              wide_edges: bool = False, step_kernel: int = 0) -> gn_net_desc:
    """Marshal a ``netgen.NetSpec``-like object into a gn_net_desc; the arrays it
    points to are appended to ``keep`` (they must live until the create call)."""
    k = dict(pos=_c(spec.pos, np.float64), src=_c(spec.src, np.int32), dst=_c(spec.dst, np.int32),
             weight=_c(spec.weight, np.float32), speed=_c(spec.speed, np.float64), delay=_c(spec.delay, np.int32))
    keep.append(k)
    fhn = spec.fhn
    obs = spec.obs
    cpl = coupling or spec.coupling
    return gn_net_desc(
        n_nodes=spec.n_nodes, dim=spec.dim, pos=_ptr(k["pos"]), n_edges=spec.n_edges,
        src=_ptr(k["src"]), dst=_ptr(k["dst"]), weight=_ptr(k["weight"]), speed=_ptr(k["speed"]),
        speed_scalar=float(spec.speed_scalar or 0.0), delay_steps=_ptr(k["delay"]), dt_ms=spec.dt_ms,
        fhn=gn_fhn_params(**{x: fhn[x] for x in ("a", "b", "c", "e", "f", "g", "i_ext")}),
        obs=gn_obs_params(tau_ms=obs["tau_ms"], sample_every=obs["sample_every"], gain=obs["gain"],
                          offset=obs["offset"], sigma=obs["sigma"], seed=obs["seed"],
                          frame_average=1 if obs.get("frame_average") else 0),
        coupling=GN_COUPLE_RAW if cpl == "raw" else GN_COUPLE_REST, theta=spec.theta,
        ring_depth=spec.ring_depth if ring_depth is None else ring_depth,
        obs_capacity=obs_capacity, event_capacity=event_capacity, renumber=0 if renumber else -1,
        edge_format=1 if wide_edges else 0, step_kernel=step_kernel,
        cuda_stream=stream, device=device, model=_MODELS[getattr(spec, "model", "fhn")],
        izh=_izh_params(getattr(spec, "izh", None)), hh=_hh_params(getattr(spec, "hh", None)),
        stdp=_stdp_params(getattr(spec, "stdp", None)), **_cell_types(spec, keep))


def _cell_types(spec, keep) -> dict:
    types = getattr(spec, "cell_types", None)
    if not types:
        return {}
    hh = getattr(spec, "model", "fhn") == "hh"
    tab = (gn_hh_params * len(types))(*[_hh_params(t) for t in types]) if hh else \
        (gn_izh_params * len(types))(*[_izh_params(t) for t in types])
    cell = np.ascontiguousarray(spec.cell_type, np.uint8)
    keep += [tab, cell]
    ptr = C.cast(tab, C.c_void_p)
    return dict(n_cell_types=len(types), izh_types=None if hh else ptr, hh_types=ptr if hh else None,
                cell_type=_ptr(cell))


def _izh_params(iz) -> gn_izh_params:
    if not iz:
        return gn_izh_params()
    return gn_izh_params(C=iz["C"], k=iz["k"], v_r=iz["vr"], v_t=iz["vt"], v_peak=iz["vpeak"], v_reset=iz["vreset"],
                         a=iz["a"], b=iz["b"], d=iz["d"], i_ext=iz["i_ext"], psc_a=iz["psc_a"], tau_c=iz["tau_c"])


def _stdp_params(sp) -> gn_stdp_params:
    if not sp:
        return gn_stdp_params()
    return gn_stdp_params(enable=1, alpha=sp["alpha"], beta=sp["beta"])


def _hh_params(hp) -> gn_hh_params:
    if not hp:
        return gn_hh_params()
    return gn_hh_params(C=hp["C"], g_na=hp["gna"], g_k=hp["gk"], g_l=hp["gl"], e_na=hp["ena"], e_k=hp["ek"],
                        e_l=hp["el"], v_peak=hp["vpeak"], i_ext=hp["i_ext"], psc_a=hp["psc_a"], tau_c=hp["tau_c"])


class Net:
    """One network on the GPU, created from a ``netgen.NetSpec``-like object."""

    def __init__(self, spec, *, device: int = 0, stream=None, obs_capacity: int = 0,
                 event_capacity: int = 0, renumber: bool = True, ring_depth: int | None = None,
                 coupling: str | None = None, wide_edges: bool = False, step_kernel: int = 0):
        L = lib()
        keep = []
        d = make_desc(spec, keep, device=device, stream=stream, obs_capacity=obs_capacity,
                      event_capacity=event_capacity, renumber=renumber, ring_depth=ring_depth, coupling=coupling,
                      wide_edges=wide_edges, step_kernel=step_kernel)
        h = C.c_void_p()
        check(L.gn_net_create(C.byref(d), C.byref(h)))
        self.h = h
        self.n_nodes = spec.n_nodes
        self.n_edges = spec.n_edges
        self.spec = spec
        if spec.pulses:
            self.gn_set_stimulus(spec.pulses)
        bg = spec.background
        if bg:
            self.gn_set_background(bg["rate_hz"], bg["amp"], bg["dur_ms"], bg["seed"])

    # ---- the C ABI, one method per call ----
    def gn_net_destroy(self):
        if getattr(self, "h", None):
            check(lib().gn_net_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.gn_net_destroy()
        except Exception:
            pass

    def gn_net_get_info(self) -> dict:
        i = gn_net_info()
        check(lib().gn_net_get_info(self.h, C.byref(i)))
        return {f: getattr(i, f) for f, _ in gn_net_info._fields_}

    def gn_get_delays(self) -> np.ndarray:
        out = np.zeros(self.n_edges, np.int32)
        check(lib().gn_get_delays(self.h, _ptr(out)))
        return out

    def gn_get_rest(self):
        v, w = C.c_double(), C.c_double()
        check(lib().gn_get_rest(self.h, C.byref(v), C.byref(w)))
        return v.value, w.value

    def gn_set_stimulus(self, pulses):
        arr = (gn_pulse * max(1, len(pulses)))()
        for i, (node, t_on, t_off, amp) in enumerate(pulses):
            arr[i] = gn_pulse(node=node, t_on_ms=t_on, t_off_ms=t_off, amp=amp)
        check(lib().gn_set_stimulus(self.h, arr, len(pulses)))

    def gn_set_background(self, rate_hz, amp, dur_ms, seed):
        check(lib().gn_set_background(self.h, rate_hz, amp, dur_ms, seed))

    def gn_step(self, n_steps: int):
        check(lib().gn_step(self.h, n_steps))

    def gn_synchronize(self):
        check(lib().gn_synchronize(self.h))

    def gn_observe(self, max_samples: int | None = None, out: np.ndarray | None = None,
                   discard: bool = False):
        """Unread observation rows [k, n_nodes] (caller order), the number of the
        first, and the status (GN_OK or GN_EOVERFLOW)."""
        info = self.gn_net_get_info()
        if max_samples is None:
            max_samples = info["samples"]
        if out is None and not discard:
            out = np.zeros((max(0, max_samples), self.n_nodes), np.float32)
        elif not discard:
            _out_rows(out, max_samples, self.n_nodes)
        first = C.c_int64()
        wr = C.c_int64()
        st = check(lib().gn_observe(self.h, None if discard else _ptr(out), max_samples, C.byref(first),
                                    C.byref(wr)), allow=(GN_EOVERFLOW,))
        return (None if discard else out[: wr.value]), first.value, st

    def gn_observe_async(self, out: np.ndarray, max_samples: int):
        """Queue the copy of up to max_samples unread rows into `out` (which must stay
        alive until gn_observe_wait); returns (rows written, first sample, status)."""
        _out_rows(out, max_samples, self.n_nodes)
        first = C.c_int64()
        wr = C.c_int64()
        st = check(lib().gn_observe_async(self.h, _ptr(out), max_samples, C.byref(first), C.byref(wr)),
                   allow=(GN_EOVERFLOW,))
        return wr.value, first.value, st

    def gn_observe_wait(self):
        check(lib().gn_observe_wait(self.h))

    def gn_get_state(self):
        N = self.n_nodes
        v, w, c = (np.zeros(N, np.float32) for _ in range(3))
        bg = np.zeros(N, np.int32)
        st = C.c_int64()
        check(lib().gn_get_state(self.h, _ptr(v), _ptr(w), _ptr(c), _ptr(bg), C.byref(st)))
        return dict(v=v, w=w, c=c, bg_count=bg, step=st.value)

    def gn_set_state(self, hist, w=None, c=None, bg_count=None, step: int = 0):
        N = self.n_nodes
        hist = _rows_in(hist, N, "hist")
        w, c = _vec(w, np.float32, N, "w"), _vec(c, np.float32, N, "c")
        bg = _vec(bg_count, np.int32, N, "bg_count")
        check(lib().gn_set_state(self.h, _ptr(hist), hist.shape[0], _ptr(w), _ptr(c), _ptr(bg), step))

    def gn_get_izh_state(self):
        N = self.n_nodes
        V, r, p = (np.zeros(N, np.float32) for _ in range(3))
        check(lib().gn_get_izh_state(self.h, _ptr(V), _ptr(r), _ptr(p)))
        return dict(V=V, r=r, p=p)

    def gn_set_izh_state(self, V=None, r=None, p=None):
        N = self.n_nodes
        V, r, p = _vec(V, np.float32, N, "V"), _vec(r, np.float32, N, "r"), _vec(p, np.float32, N, "p")
        check(lib().gn_set_izh_state(self.h, _ptr(V), _ptr(r), _ptr(p)))

    def gn_get_hh_gates(self):
        N = self.n_nodes
        m, n, h = (np.zeros(N, np.float32) for _ in range(3))
        check(lib().gn_get_hh_gates(self.h, _ptr(m), _ptr(n), _ptr(h)))
        return dict(m=m, n=n, h=h)

    def gn_set_hh_gates(self, m=None, n=None, h=None):
        N = self.n_nodes
        m, n, h = _vec(m, np.float32, N, "m"), _vec(n, np.float32, N, "n"), _vec(h, np.float32, N, "h")
        check(lib().gn_set_hh_gates(self.h, _ptr(m), _ptr(n), _ptr(h)))

    def gn_get_weights(self) -> np.ndarray:
        out = np.zeros(self.n_edges, np.float32)
        check(lib().gn_get_weights(self.h, _ptr(out)))
        return out

    def gn_set_weights(self, w):
        w = _vec(w, np.float32, self.n_edges, "w")
        if w is None:
            raise ValueError("w is required")
        check(lib().gn_set_weights(self.h, _ptr(w)))

    def gn_get_stdp_history(self, depth: int) -> np.ndarray:
        out = np.zeros((depth, self.n_nodes), np.float32)
        check(lib().gn_get_stdp_history(self.h, _ptr(out), depth))
        return out

    def gn_set_stdp_history(self, s_hist):
        s_hist = _rows_in(s_hist, self.n_nodes, "s_hist")
        check(lib().gn_set_stdp_history(self.h, _ptr(s_hist), s_hist.shape[0]))

    def gn_get_history(self, depth: int) -> np.ndarray:
        out = np.zeros((depth, self.n_nodes), np.float32)
        check(lib().gn_get_history(self.h, _ptr(out), depth))
        return out

    def gn_get_arrivals(self) -> np.ndarray:
        out = np.zeros(self.n_nodes, np.int64)
        check(lib().gn_get_arrivals(self.h, _ptr(out)))
        return out

    def gn_get_events(self, cap: int = 1 << 22):
        node = np.zeros(cap, np.int32)
        step = np.zeros(cap, np.int64)
        n = C.c_int64()
        st = check(lib().gn_get_events(self.h, _ptr(node), _ptr(step), cap, C.byref(n)), allow=(GN_EOVERFLOW,))
        m = min(cap, n.value)
        return node[:m], step[:m], st

    def gn_save_state(self) -> bytes:
        used = C.c_size_t()
        check(lib().gn_save_state(self.h, None, 0, C.byref(used)))
        buf = (C.c_uint8 * used.value)()
        check(lib().gn_save_state(self.h, buf, used.value, C.byref(used)))
        return bytes(buf)

    def gn_load_state(self, blob: bytes):
        buf = (C.c_uint8 * len(blob)).from_buffer_copy(blob)
        check(lib().gn_load_state(self.h, buf, len(blob)))


class Batch:
    """Many independent networks advanced together (gn_batch_*); ``specs`` are
    ``netgen.NetSpec``-like objects, their pulses and background are applied."""

    def __init__(self, specs, *, device: int = 0, stream=None, obs_capacity: int = 0):
        L = lib()
        keep = []
        n = len(specs)
        descs = (gn_net_desc * n)()
        for i, sp in enumerate(specs):
            descs[i] = make_desc(sp, keep, device=device, stream=stream, obs_capacity=obs_capacity)
        h = C.c_void_p()
        check(L.gn_batch_create(descs, n, C.byref(h)))
        self.h = h
        self.specs = list(specs)
        self.n_nets = n
        counts = np.array([len(sp.pulses or []) for sp in specs], np.int32)
        if counts.sum():
            allp = (gn_pulse * int(counts.sum()))()
            k = 0
            for sp in specs:
                for (node, t_on, t_off, amp) in sp.pulses or []:
                    allp[k] = gn_pulse(node=node, t_on_ms=t_on, t_off_ms=t_off, amp=amp)
                    k += 1
            check(L.gn_batch_set_stimulus_all(h, allp, _ptr(counts)))
        for i, sp in enumerate(specs):
            bg = sp.background
            if bg:
                check(L.gn_batch_set_background(h, i, bg["rate_hz"], bg["amp"], bg["dur_ms"], bg["seed"]))

    def gn_batch_destroy(self):
        if getattr(self, "h", None):
            check(lib().gn_batch_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.gn_batch_destroy()
        except Exception:
            pass

    def gn_batch_get_info(self) -> dict:
        i = gn_batch_info()
        check(lib().gn_batch_get_info(self.h, C.byref(i)))
        return {f: getattr(i, f) for f, _ in gn_batch_info._fields_}

    def gn_batch_get_net_info(self, net: int) -> dict:
        i = gn_net_info()
        check(lib().gn_batch_get_net_info(self.h, net, C.byref(i)))
        return {f: getattr(i, f) for f, _ in gn_net_info._fields_}

    def gn_batch_get_delays(self, net: int) -> np.ndarray:
        out = np.zeros(self.specs[net].n_edges, np.int32)
        check(lib().gn_batch_get_delays(self.h, net, _ptr(out)))
        return out

    def gn_batch_step(self, n_steps: int):
        check(lib().gn_batch_step(self.h, n_steps))

    def gn_batch_step_static(self, n_steps: int):
        check(lib().gn_batch_step_static(self.h, n_steps))

    def gn_batch_synchronize(self):
        check(lib().gn_batch_synchronize(self.h))

    def gn_batch_observe(self, net: int, max_samples: int | None = None):
        info = self.gn_batch_get_net_info(net)
        if max_samples is None:
            max_samples = info["samples"]
        out = np.zeros((max(0, max_samples), self.specs[net].n_nodes), np.float32)
        first = C.c_int64()
        wr = C.c_int64()
        st = check(lib().gn_batch_observe(self.h, net, _ptr(out), max_samples, C.byref(first), C.byref(wr)),
                   allow=(GN_EOVERFLOW,))
        return out[: wr.value], first.value, st

    def gn_batch_get_state(self, net: int):
        N = self.specs[net].n_nodes
        v, w, c = (np.zeros(N, np.float32) for _ in range(3))
        bg = np.zeros(N, np.int32)
        st = C.c_int64()
        check(lib().gn_batch_get_state(self.h, net, _ptr(v), _ptr(w), _ptr(c), _ptr(bg), C.byref(st)))
        return dict(v=v, w=w, c=c, bg_count=bg, step=st.value)

    def gn_batch_get_history(self, net: int, depth: int) -> np.ndarray:
        out = np.zeros((depth, self.specs[net].n_nodes), np.float32)
        check(lib().gn_batch_get_history(self.h, net, _ptr(out), depth))
        return out

    def gn_batch_get_izh_state(self, net: int):
        N = self.specs[net].n_nodes
        V, r, p = (np.zeros(N, np.float32) for _ in range(3))
        check(lib().gn_batch_get_izh_state(self.h, net, _ptr(V), _ptr(r), _ptr(p)))
        return dict(V=V, r=r, p=p)

    def gn_batch_get_hh_gates(self, net: int):
        N = self.specs[net].n_nodes
        m, n, h = (np.zeros(N, np.float32) for _ in range(3))
        check(lib().gn_batch_get_hh_gates(self.h, net, _ptr(m), _ptr(n), _ptr(h)))
        return dict(m=m, n=n, h=h)

    def gn_batch_get_arrivals(self, net: int) -> np.ndarray:
        out = np.zeros(self.specs[net].n_nodes, np.int64)
        check(lib().gn_batch_get_arrivals(self.h, net, _ptr(out)))
        return out

    def gn_batch_get_events(self, net: int, cap: int = 1 << 20):
        node = np.zeros(cap, np.int32)
        step = np.zeros(cap, np.int64)
        n = C.c_int64()
        st = check(lib().gn_batch_get_events(self.h, net, _ptr(node), _ptr(step), cap, C.byref(n)),
                   allow=(GN_EOVERFLOW,))
        m = min(cap, n.value)
        return node[:m], step[:m], st

    def gn_batch_set_step(self, step: int):
        check(lib().gn_batch_set_step(self.h, step))

    def gn_batch_set_state(self, net: int, hist, w=None, c=None, bg_count=None):
        N = self.specs[net].n_nodes
        hist = _rows_in(hist, N, "hist")
        w, c = _vec(w, np.float32, N, "w"), _vec(c, np.float32, N, "c")
        bg = _vec(bg_count, np.int32, N, "bg_count")
        check(lib().gn_batch_set_state(self.h, net, _ptr(hist), hist.shape[0], _ptr(w), _ptr(c), _ptr(bg)))


# --------------------------------------------------------------------------- estimator
def _dptr(t):
    """Device address of a torch CUDA tensor (or None)."""
    return None if t is None else C.c_void_p(t.data_ptr())


def _dev(t, dtype: str, name: str, shape=None, min_len: int | None = None):
    """A caller's device tensor, checked before its address goes to the library: a
    contiguous CUDA tensor of `dtype` ("float32", "float64", "int32", "int64"),
    of `shape` (None entries free) or 1-D with at least `min_len` entries."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()
            and t.dtype == getattr(torch, dtype)):
        raise ValueError(f"{name} must be a contiguous CUDA tensor of {dtype}")
    if shape is not None and (t.dim() != len(shape)
                              or any(want is not None and got != want for got, want in zip(t.shape, shape))):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, {tuple(shape)} expected")
    if min_len is not None and (t.dim() != 1 or t.shape[0] < min_len):
        raise ValueError(f"{name} must be 1-D with at least {min_len} entries, got {tuple(t.shape)}")
    return t


def gn_batch_export_traces(batch: "Batch", first_sample: int, n_samples: int, out):
    """Node-major traces [total nodes, n_samples] of every network of `batch` into
    the CUDA tensor `out`."""
    _dev(out, "float32", "out", shape=(sum(sp.n_nodes for sp in batch.specs), n_samples))
    check(lib().gn_batch_export_traces(batch.h, first_sample, n_samples, _dptr(out)))
    return out


def gn_xcorr_features(traces, pos, src, dst, radius, features, score, v_max: float = 0.5, sample_ms: float = 1.0,
                      stream=None):
    """Lagged normalised cross-correlation features of candidate pairs; every
    argument but v_max / sample_ms is a CUDA tensor (traces f32 [M, T], pos f64
    [M, dim], src / dst i32 [P], radius f64 [P], features f32 [P, 33], score f32 [P])."""
    _dev(traces, "float32", "traces", shape=(None, None))
    M, T = traces.shape
    _dev(pos, "float64", "pos", shape=(M, None))
    _dev(src, "int32", "src", shape=(None,))
    P = src.shape[0]
    _dev(dst, "int32", "dst", shape=(P,))
    _dev(radius, "float64", "radius", shape=(P,))
    _dev(features, "float32", "features", shape=(P, 33))
    _dev(score, "float32", "score", shape=(P,))
    check(lib().gn_xcorr_features(_dptr(traces), M, T, _dptr(pos), pos.shape[1], src.shape[0], _dptr(src),
                                  _dptr(dst), _dptr(radius), v_max, sample_ms, _dptr(features), _dptr(score),
                                  stream))


def _host_scores(scores, labels):
    s = np.ascontiguousarray(scores, np.float32)
    y = np.ascontiguousarray(labels, np.uint8)
    return s, y


def gn_score_auroc(scores, labels) -> float:
    s, y = _host_scores(scores, labels)
    out = C.c_double()
    check(lib().gn_score_auroc(_ptr(s), _ptr(y), s.size, C.byref(out)))
    return out.value


def gn_score_f1(scores, labels, threshold: float) -> float:
    s, y = _host_scores(scores, labels)
    out = C.c_double()
    check(lib().gn_score_f1(_ptr(s), _ptr(y), s.size, threshold, C.byref(out)))
    return out.value


def gn_score_best_f1(scores, labels):
    s, y = _host_scores(scores, labels)
    thr, f1 = C.c_double(), C.c_double()
    check(lib().gn_score_best_f1(_ptr(s), _ptr(y), s.size, C.byref(thr), C.byref(f1)))
    return thr.value, f1.value


MLP_HIDDEN = 256


def mlp_pack(params: dict) -> np.ndarray:
    """Packed parameter array [W1 | b1 | W2 | b2 | w3 | b3] (FP32)."""
    return np.concatenate([np.asarray(params[k], np.float32).reshape(-1)
                           for k in ("W1", "b1", "W2", "b2", "w3", "b3")])


def mlp_unpack(flat: np.ndarray, in_dim: int) -> dict:
    H = MLP_HIDDEN
    sizes = dict(W1=(in_dim, H), b1=(H,), W2=(H, H), b2=(H,), w3=(H,), b3=(1,))
    out, o = {}, 0
    for k, shp in sizes.items():
        n = int(np.prod(shp))
        out[k] = np.asarray(flat[o:o + n]).reshape(shp)
        o += n
    return out


class Mlp:
    """The learned estimator's network on the GPU (gn_mlp_*); batches are CUDA tensors."""

    def __init__(self, params: dict, max_batch: int, *, device: int = 0, stream=None):
        self.in_dim = int(np.asarray(params["W1"]).shape[0])
        flat = mlp_pack(params)
        self.n_params = flat.size
        h = C.c_void_p()
        check(lib().gn_mlp_create(self.in_dim, max_batch, _ptr(flat), device, stream, C.byref(h)))
        self.h = h

    def gn_mlp_destroy(self):
        if getattr(self, "h", None):
            check(lib().gn_mlp_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.gn_mlp_destroy()
        except Exception:
            pass

    def gn_mlp_get_params(self) -> dict:
        flat = np.zeros(self.n_params, np.float32)
        check(lib().gn_mlp_get_params(self.h, _ptr(flat)))
        return mlp_unpack(flat, self.in_dim)

    def _xy(self, X, y, idx, min_idx: int = 0):
        """Check a resident set X [rows, in_dim], y [rows] and an optional int64
        row index (device tensors)."""
        _dev(X, "float32", "X", shape=(None, self.in_dim))
        _dev(y, "float32", "y", shape=(X.shape[0],))
        if idx is not None:
            _dev(idx, "int64", "idx", min_len=min_idx)

    def gn_mlp_gradients(self, X, y, idx=None):
        self._xy(X, y, idx)
        flat = np.zeros(self.n_params, np.float32)
        loss = C.c_float()
        B = X.shape[0] if idx is None else idx.shape[0]
        check(lib().gn_mlp_gradients(self.h, _dptr(X), _dptr(y), _dptr(idx), B, _ptr(flat), C.byref(loss)))
        return mlp_unpack(flat, self.in_dim), loss.value

    def gn_mlp_train_step(self, X, y, idx=None, lr: float = 1e-3, weight_decay: float = 0.0,
                          want_loss: bool = True):
        self._xy(X, y, idx)
        loss = C.c_float()
        B = X.shape[0] if idx is None else idx.shape[0]
        check(lib().gn_mlp_train_step(self.h, _dptr(X), _dptr(y), _dptr(idx), B, lr, weight_decay,
                                      C.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def gn_mlp_train_epoch(self, X, y, idx, n_batches: int, B: int, lr: float = 1e-3, weight_decay: float = 0.0,
                           want_losses: bool = True):
        """n_batches AdamW steps on rows idx[j B .. (j + 1) B) (device int64), one
        replayed graph launch per step; returns the per-step losses (numpy) or None."""
        if idx is None:
            raise ValueError("idx is required")
        self._xy(X, y, idx, min_idx=n_batches * B)
        losses = np.zeros(n_batches, np.float32) if want_losses else None
        check(lib().gn_mlp_train_epoch(self.h, _dptr(X), _dptr(y), _dptr(idx), n_batches, B, lr, weight_decay,
                                       _ptr(losses) if want_losses else None))
        return losses

    def gn_mlp_infer(self, X, out):
        _dev(X, "float32", "X", shape=(None, self.in_dim))
        _dev(out, "float32", "out", min_len=X.shape[0])
        check(lib().gn_mlp_infer(self.h, _dptr(X), X.shape[0], _dptr(out)))
        return out

    def gn_mlp_synchronize(self):
        check(lib().gn_mlp_synchronize(self.h))


def exported_symbols() -> list:
    """Names of the gn_* functions declared in include/*.h."""
    import glob
    import re
    names = []
    for h in glob.glob(os.path.join(os.path.dirname(_HERE), "include", "*.h")):
        names += re.findall(r"^\s*GN_API\s+(?:gn_status|const char \*)\s*(gn_\w+)\s*\(", open(h).read(), re.M)
    return sorted(set(names))
