"""Seeded synthetic inputs: node positions, directed edges, weights, speeds and
stimulus schedules of geometric networks.

This module is the one place both the CUDA path and the FP64 oracle take their
inputs from.  It holds none of the method's arithmetic: no delays, no dynamics,
no readout -- only the random draws that define a network and its controls.

The paper's own test networks (Sec. 3.5, "available for download") are not
available, so these generators stand in for them.  The recipes:

* ``tiny``      N = 64 uniform in a 1 x 1 mm square; directed i -> j for every
                ordered pair closer than 0.2 mm, kept with p = 0.5; w ~ U(0.1, 0.5);
                one speed 0.1 m/s; +1.0 pulse on node 0 over [10, 12) ms.
* ``large``     N = 100,000 uniform in a 1 mm cube; every ordered pair within the
                radius that gives a mean in-degree of 100; w = lognormal(-2, 0.5)
                with 20 % negated, then the in-weights of a target with k > 20
                inputs scaled by 20 / k; speed U(0.05, 0.5) m/s per edge; 5 Hz
                background pulses (1.0, 2 ms).
* ``roofline``  N = 1,000,000 in a 1 mm cube, mean in-degree 50: 2.5 % hub nodes
                take in-edges from their 1000 nearest nodes, the rest take every
                node within the radius giving the remaining mean (about 25.6);
                weight (with the same in-degree scaling), speed and background
                as ``large``; ring of 256 steps.
* ``batch``     many independent 2D nets, N log-uniform in [32, 4096]; pairs within
                r = sqrt(40 / (pi N)) kept with p = 0.5 (mean kept in-degree about 20
                away from the border); weight and speed as ``large``; 1-8 random
                nodes get a 2 ms pulse with onset uniform in [5, 50) ms.
  The in-degree scaling keeps a node's total input on the scale of the 20-input
  nets the weight law comes from: unscaled, a hub summing 1000 inputs of mean
  |w| 0.15 drives explicit Euler at dt = 0.05 ms past the cubic's stability
  bound within tens of milliseconds and the run ends in NaN.
* ``fig2``      the five-vertex network of Figs. 1-2 with the printed delays and
                weights (delays are given explicitly, in steps of 0.05 ms).

FHN parameters are given in the paper's notation (Sec. 3.1,
dV = aV - bV^3 - cW + S + U, dW = e(V + f - gW)); the classic choice
(0.7, 0.8, 0.08) is a = 1, b = 1/3, c = 1, e = 0.08, f = 0.7, g = 0.8.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy.spatial import cKDTree

FHN_CLASSIC = dict(a=1.0, b=1.0 / 3.0, c=1.0, e=0.08, f=0.7, g=0.8, i_ext=0.0)
OBS_DEFAULT = dict(tau_ms=5.0, sample_every=20, gain=1.0, offset=0.0, sigma=0.05, seed=2)
# Izhikevich simple model (Sec. 3.1, Eq. izsimple) with regular-spiking cortical
# parameters -- C pF, k nS/mV, mV, a 1/ms, b nS, d pA -- an alpha-function PSC of rate
# psc_a 1/ms (Eq. alphapsc) and a calcium removal time tau_c ms (Eq. casimple).  The
# paper gives the model, not these numbers.
IZH_RS = dict(C=100.0, k=0.7, vr=-60.0, vt=-40.0, vpeak=35.0, vreset=-50.0, a=0.03, b=-2.0, d=100.0,
              i_ext=0.0, psc_a=0.2, tau_c=20.0)
# A fast-spiking interneuron-like parameter set of the same simple model (small
# capacitance, fast recovery, no adaptation jump), for excitatory / inhibitory mixes;
# the PSC and calcium constants are the regular-spiking cell's.
IZH_FS = dict(C=20.0, k=1.0, vr=-55.0, vt=-40.0, vpeak=25.0, vreset=-45.0, a=0.2, b=-2.0, d=0.0,
              i_ext=0.0, psc_a=0.2, tau_c=20.0)
# Hodgkin-Huxley squid-axon constants in the modern convention (uF/cm^2, mS/cm^2,
# mV; rest near -65 mV), V_peak = 0 mV for the spike indicator, and the same PSC
# and calcium time constants as IZH_RS.
HH_CLASSIC = dict(C=1.0, gna=120.0, gk=36.0, gl=0.3, ena=50.0, ek=-77.0, el=-54.387, vpeak=0.0, i_ext=0.0,
                  psc_a=0.2, tau_c=20.0)


@dataclasses.dataclass
class NetSpec:
    """One network and its controls, in the caller's node and edge order."""
    pos: np.ndarray                 # [N, dim] float64, mm
    src: np.ndarray                 # [E] int32, source i of edge i -> j
    dst: np.ndarray                 # [E] int32, target j
    weight: np.ndarray              # [E] float32
    speed: np.ndarray | None        # [E] float64 m/s (= mm/ms), or None
    speed_scalar: float = 0.0       # used when speed is None
    delay: np.ndarray | None = None  # [E] int32 explicit delays in steps (bypasses geometry)
    dt_ms: float = 0.05
    fhn: dict = dataclasses.field(default_factory=lambda: dict(FHN_CLASSIC))
    obs: dict = dataclasses.field(default_factory=lambda: dict(OBS_DEFAULT))
    coupling: str = "rest"
    theta: float = 0.0
    pulses: list = dataclasses.field(default_factory=list)   # (node, t_on_ms, t_off_ms, amp)
    background: dict | None = None  # dict(rate_hz, amp, dur_ms, seed)
    ring_depth: int = 0             # 0 = smallest power of two that holds the delays
    radius: float = 0.0             # radius the edges were drawn within (candidate pairs), 0 = unknown
    name: str = ""
    model: str = "fhn"              # "fhn", "izh" (Izhikevich) or "hh" (Hodgkin-Huxley), + alpha PSC + calcium
    izh: dict = dataclasses.field(default_factory=lambda: dict(IZH_RS))
    hh: dict = dataclasses.field(default_factory=lambda: dict(HH_CLASSIC))
    stdp: dict | None = None        # spike-time-dependent plasticity {alpha, beta} (spiking models)
    cell_types: list | None = None  # heterogeneous cells: parameter sets of the spiking model ...
    cell_type: np.ndarray | None = None  # ... and each node's set (uint8, < 8 sets)

    @property
    def n_nodes(self) -> int:
        return int(self.pos.shape[0])

    @property
    def n_edges(self) -> int:
        return int(self.src.shape[0])

    @property
    def dim(self) -> int:
        return int(self.pos.shape[1])


def izhikevich(spec: "NetSpec", w_scale: float = 2000.0, pulse_amp: float = 2500.0, obs_gain: float = 20.0):
    """The same network and controls with Izhikevich + alpha-PSC nodes: weights
    scaled to PSC units (a spike through an edge of weight w adds dt w to p, so r
    peaks at dt w / (a_s e): 2000 x a weight of 0.3 gives 55 pA at dt = 0.05 ms),
    pulses and background pulses of pulse_amp pA (2 ms at 2500 pA make a resting
    node spike), and the calcium readout scaled by obs_gain (one spike adds dt to c).
    With these defaults the 2.5 %-hub nets fire near their 5 Hz background; the
    tiny net needs a scale near 7000 before its spikes propagate."""
    return dataclasses.replace(
        spec, model="izh", izh=dict(IZH_RS), weight=(np.asarray(spec.weight) * w_scale).astype(np.float32),
        pulses=[(j, t0, t1, pulse_amp) for (j, t0, t1, _) in spec.pulses],
        background=None if spec.background is None else dict(spec.background, amp=pulse_amp),
        obs=dict(spec.obs, gain=obs_gain), name=spec.name + "_izh")


def mixed_cells(spec: "NetSpec", types=None, frac=(0.8, 0.2), inhibitory=(False, True), seed: int = 0):
    """Heterogeneous cells (Sec. 3.1: networks of different cell types as different
    parameter sets of one transition function): each node draws a parameter set of
    the network's spiking model with probabilities `frac`; a source of an inhibitory
    set makes every out-weight negative, of an excitatory set positive (|w| kept).
    Default: Izhikevich regular-spiking 80 % / fast-spiking 20 % (inhibitory)."""
    if spec.model not in ("izh", "hh"):
        raise ValueError("heterogeneous cells need a spiking model")
    if types is None:
        types = [dict(IZH_RS), dict(IZH_FS)] if spec.model == "izh" else [dict(spec.hh), dict(spec.hh)]
    rng = np.random.default_rng(seed + 777)
    cell = rng.choice(len(types), size=spec.n_nodes, p=np.asarray(frac, np.float64) / np.sum(frac)).astype(np.uint8)
    sign = np.where(np.asarray(inhibitory, bool)[cell[np.asarray(spec.src)]], -1.0, 1.0)
    w = (np.abs(np.asarray(spec.weight, np.float64)) * sign).astype(np.float32)
    return dataclasses.replace(spec, cell_types=[dict(t) for t in types], cell_type=cell, weight=w,
                               name=spec.name + "_mixed")


def hodgkin_huxley(spec: "NetSpec", w_scale: float = 3.0, pulse_amp: float = 20.0, obs_gain: float = 1.0,
                   dt_ms: float = 0.03):
    """The same network and controls with Hodgkin-Huxley + alpha-PSC nodes at the
    paper's HH step dt = 0.03 ms: weights in PSC units (uA/cm^2; spd stays 1 for the
    ~1 ms a spike spends above 0 mV, so a spike through weight w adds about w x 1 ms
    to p), pulses and background pulses of pulse_amp uA/cm^2 (2 ms at 20 make a
    resting node spike), calcium readout gain obs_gain; sample interval kept at 1 ms;
    the ring sized afresh for the longer delays in steps.  The default scale keeps
    the signed-weight nets' hyperpolarisation near E_K: at 10 a strongly inhibited
    node of the 300k-node net reaches -120 mV, where forward Euler of the gates at
    dt = 0.03 ms is unstable (beta_m dt > 2) and V becomes NaN -- in the FP64 oracle
    as on the GPU.  The all-excitatory tiny net needs about 10 to propagate."""
    every = max(1, int(round(1.0 / dt_ms)))
    return dataclasses.replace(
        spec, model="hh", hh=dict(HH_CLASSIC), dt_ms=dt_ms, ring_depth=0,
        weight=(np.asarray(spec.weight) * w_scale).astype(np.float32),
        pulses=[(j, t0, t1, pulse_amp) for (j, t0, t1, _) in spec.pulses],
        background=None if spec.background is None else dict(spec.background, amp=pulse_amp),
        obs=dict(spec.obs, gain=obs_gain, sample_every=every), name=spec.name + "_hh")


def _signed_lognormal(rng, n, mu=-2.0, sigma=0.5, neg_frac=0.2):
    w = rng.lognormal(mu, sigma, n)
    w[rng.random(n) < neg_frac] *= -1.0
    return w.astype(np.float32)


def _pairs_within(pos, r):
    """All ordered pairs (i, j), i != j, with |x_i - x_j| < r (both directions)."""
    tree = cKDTree(pos)
    p = tree.query_pairs(r, output_type="ndarray")
    if p.size == 0:
        return np.zeros(0, np.int32), np.zeros(0, np.int32)
    # query_pairs uses <= r; drop exact-distance ties so the rule is strict
    d = np.sqrt(((pos[p[:, 0]] - pos[p[:, 1]]) ** 2).sum(1))
    p = p[d < r]
    src = np.concatenate([p[:, 0], p[:, 1]]).astype(np.int32)
    dst = np.concatenate([p[:, 1], p[:, 0]]).astype(np.int32)
    return src, dst


def _sort_by_dst(src, dst, *extra):
    """Edges in (dst, src) order (ties, i.e. repeated pairs, kept in their order): a
    deterministic caller order."""
    key = np.asarray(dst, np.int64) * (int(max(np.max(src, initial=0), np.max(dst, initial=0))) + 1) + \
        np.asarray(src, np.int64)
    order = np.argsort(key, kind="stable")
    return (src[order], dst[order]) + tuple(x[order] for x in extra)


def tiny(seed: int = 1, n: int = 64, radius: float = 0.2, keep: float = 0.5,
         noise_seed: int = 2) -> NetSpec:
    rng = np.random.default_rng(seed)
    pos = rng.random((n, 2))
    src, dst = _pairs_within(pos, radius)
    keep_mask = rng.random(src.shape[0]) < keep
    src, dst = src[keep_mask], dst[keep_mask]
    src, dst = _sort_by_dst(src, dst)
    w = rng.uniform(0.1, 0.5, src.shape[0]).astype(np.float32)
    obs = dict(OBS_DEFAULT, seed=noise_seed)
    return NetSpec(pos=pos, src=src, dst=dst, weight=w, speed=None, speed_scalar=0.1,
                   obs=obs, pulses=[(0, 10.0, 12.0, 1.0)], name="tiny")


def _radius_for_mean_degree(pos, mean_deg, n_probe=20000, seed=0):
    """Radius at which the mean number of other nodes within r equals mean_deg
    (bisection on a random probe set, so border losses are included)."""
    n, dim = pos.shape
    tree = cKDTree(pos)
    rng = np.random.default_rng(seed)
    probe = pos[rng.choice(n, min(n_probe, n), replace=False)]
    unit = math.pi if dim == 2 else 4.0 * math.pi / 3.0
    r0 = (mean_deg / (n * unit)) ** (1.0 / dim)
    lo, hi = 0.5 * r0, 2.0 * r0
    for _ in range(40):
        mid = 0.5 * (lo + hi)
        cnt = tree.query_ball_point(probe, mid, return_length=True, workers=-1).mean() - 1.0
        if cnt < mean_deg:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def _in_degree_scaled(w: np.ndarray, dst: np.ndarray, n: int, k0: float = 20.0) -> np.ndarray:
    """w_e * min(1, k0 / k_dst(e)): targets with more than k0 inputs get their
    in-weights scaled so their total input stays on the scale of a k0-input node."""
    k = np.bincount(dst, minlength=n).astype(np.float64)
    return (w * np.minimum(1.0, k0 / np.maximum(k[dst], 1.0))).astype(np.float32)


def large(seed: int = 3, n: int = 100_000, mean_deg: float = 100.0, bg_rate_hz: float = 5.0,
          noise_seed: int = 5, dim: int = 3) -> NetSpec:
    rng = np.random.default_rng(seed)
    pos = rng.random((n, dim))
    r = _radius_for_mean_degree(pos, mean_deg, seed=seed)
    src, dst = _pairs_within(pos, r)
    src, dst = _sort_by_dst(src, dst)
    E = src.shape[0]
    w = _in_degree_scaled(_signed_lognormal(rng, E), dst, n)
    speed = rng.uniform(0.05, 0.5, E)
    obs = dict(OBS_DEFAULT, seed=noise_seed)
    bg = dict(rate_hz=bg_rate_hz, amp=1.0, dur_ms=2.0, seed=seed + 1000)
    return NetSpec(pos=pos, src=src, dst=dst, weight=w, speed=speed, obs=obs, background=bg,
                   ring_depth=256, name=f"large_n{n}")


def roofline(seed: int = 4, n: int = 1_000_000, mean_deg: float = 50.0, hub_frac: float = 0.025,
             hub_deg: int = 1000, bg_rate_hz: float = 5.0, noise_seed: int = 6) -> NetSpec:
    rng = np.random.default_rng(seed)
    pos = rng.random((n, 3))
    n_hub = int(round(hub_frac * n))
    hubs = rng.choice(n, n_hub, replace=False).astype(np.int64)
    is_hub = np.zeros(n, bool)
    is_hub[hubs] = True
    # non-hub targets: every node within r (r set for the remaining mean in-degree)
    rest_deg = (mean_deg * n - hub_deg * n_hub) / (n - n_hub)
    r = _radius_for_mean_degree(pos, rest_deg, seed=seed)
    s1, d1 = _pairs_within(pos, r)
    m = ~is_hub[d1]
    s1, d1 = s1[m], d1[m]
    # hub targets: the hub_deg nearest other nodes
    tree = cKDTree(pos)
    _, nn = tree.query(pos[hubs], k=hub_deg + 1, workers=-1)
    nn = nn[:, 1:]
    s2 = nn.reshape(-1).astype(np.int32)
    d2 = np.repeat(hubs, hub_deg).astype(np.int32)
    src = np.concatenate([s1, s2])
    dst = np.concatenate([d1, d2])
    src, dst = _sort_by_dst(src, dst)
    E = src.shape[0]
    w = _in_degree_scaled(_signed_lognormal(rng, E), dst, n)
    speed = rng.uniform(0.05, 0.5, E)
    obs = dict(OBS_DEFAULT, seed=noise_seed)
    bg = dict(rate_hz=bg_rate_hz, amp=1.0, dur_ms=2.0, seed=seed + 1000)
    return NetSpec(pos=pos, src=src, dst=dst, weight=w, speed=speed, obs=obs, background=bg,
                   ring_depth=256, name=f"roofline_n{n}")


def delay_stress(spec: NetSpec, factor: float = 0.1) -> NetSpec:
    """The same network with every conduction speed scaled by `factor` (delays in
    steps grow by 1 / factor: 0.1 takes the 1M-node net's 1-41 steps to about
    10-410), the ring sized afresh for them."""
    if spec.speed is None:
        raise ValueError("the net has one scalar speed; scale speed_scalar instead")
    return dataclasses.replace(spec, speed=np.asarray(spec.speed) * factor, ring_depth=0,
                               name=spec.name + f"_speedx{factor:g}")


def batch_member(seed: int, n: int | None = None, n_lo: int = 32, n_hi: int = 4096,
                 kept_deg: float = 20.0, keep: float = 0.5) -> NetSpec:
    """One network of the batched ensemble (its own seed decides its size)."""
    rng = np.random.default_rng(seed)
    if n is None:
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
    pos = rng.random((n, 2))
    r = math.sqrt(kept_deg / keep / (math.pi * n))
    src, dst = _pairs_within(pos, r)
    m = rng.random(src.shape[0]) < keep
    src, dst = _sort_by_dst(src[m], dst[m])
    E = src.shape[0]
    w = _signed_lognormal(rng, E)
    speed = rng.uniform(0.05, 0.5, E)
    k = int(rng.integers(1, 9))
    nodes = rng.choice(n, min(k, n), replace=False)
    onsets = rng.uniform(5.0, 50.0, nodes.shape[0])
    pulses = [(int(j), float(t), float(t) + 2.0, 1.0) for j, t in zip(nodes, onsets)]
    obs = dict(OBS_DEFAULT, seed=seed + 7)
    return NetSpec(pos=pos, src=src, dst=dst, weight=w, speed=speed, obs=obs, pulses=pulses, radius=r,
                   name=f"batch_s{seed}")


def estimator_control(seed: int, n: int = 512, bg_rate_hz: float = 5.0) -> NetSpec:
    """Positive control of the connectivity estimators: the batch-member laws at a
    kept in-degree of 1 (sparse, so a spike crosses an edge without setting off a
    wave through the whole net), no explicit pulses, and background pulses of 1 ms at
    `bg_rate_hz` that drive every node independently."""
    sp = batch_member(seed, n=n, kept_deg=1.0)
    return dataclasses.replace(sp, pulses=[], background=dict(rate_hz=bg_rate_hz, amp=1.0, dur_ms=1.0, seed=seed + 5),
                               name=f"control_s{seed}")


def batch(n_nets: int = 4096, seed0: int = 1000, **kw) -> list:
    return [batch_member(seed0 + i, **kw) for i in range(n_nets)]


# Fig. 1 / Fig. 2 (Sec. 3): five vertices at the TikZ positions of Fig. 2 and the eight
# edges with their printed delays (ms) and weights.  The delays are used as given.
FIG2_POS = np.array([[0.0, 3.0], [3.0, 3.0], [6.0, 4.0], [2.0, 1.0], [6.0, 1.0]])
FIG2_EDGES = [  # (from, to, delay_ms, weight), vertices numbered from 1 as in the figure
    (1, 2, 3.6, -1.0), (1, 3, 7.4, 1.0), (3, 2, 3.8, 1.0), (2, 4, 2.6, 0.7),
    (4, 5, 4.8, -2.0), (4, 1, 3.4, -2.0), (3, 5, 3.6, 1.0), (5, 2, 4.4, -1.0),
]


def fig2(delay_steps, t_on_ms: float = 10.0, amp: float = 1.0) -> NetSpec:
    """The Fig. 2 network with explicit whole-step delays ``delay_steps`` (edge order
    of ``FIG2_EDGES``) and one pulse on vertex 1."""
    src = np.array([e[0] - 1 for e in FIG2_EDGES], np.int32)
    dst = np.array([e[1] - 1 for e in FIG2_EDGES], np.int32)
    w = np.array([e[3] for e in FIG2_EDGES], np.float32)
    return NetSpec(pos=FIG2_POS.copy(), src=src, dst=dst, weight=w, speed=None, speed_scalar=1.0,
                   delay=np.asarray(delay_steps, np.int32),
                   pulses=[(0, t_on_ms, t_on_ms + 2.0, amp)], name="fig2")


def fig2_hh(w_scale: float = 10.0, dt_ms: float = 0.03, gap_ms: float = 200.0, pulse_amp: float = 20.0) -> NetSpec:
    """The Fig. 2 experiment: the five-vertex network with Hodgkin-Huxley nodes at
    dt_ms, its printed delays quantised to whole steps (half up), its printed weights
    x w_scale (uA/cm^2), and a 2 ms pulse on each vertex in turn, gap_ms apart from
    100 ms on (the figure's sequential stimulation)."""
    delay = [int(math.floor(e[2] / dt_ms + 0.5)) for e in FIG2_EDGES]
    base = fig2(delay)
    pulses = [(j, 100.0 + gap_ms * j, 102.0 + gap_ms * j, pulse_amp) for j in range(5)]
    spec = hodgkin_huxley(base, w_scale=w_scale, dt_ms=dt_ms)
    return dataclasses.replace(spec, pulses=pulses, delay=np.asarray(delay, np.int32), name="fig2_hh")


def chain2(dist_mm: float = 0.5, speed: float = 0.1, t_on_ms: float = 5.0, w: float = 0.5,
           dt_ms: float = 0.05) -> NetSpec:
    """Two nodes on the x axis, one edge 0 -> 1, a pulse on node 0."""
    pos = np.array([[0.0, 0.0], [dist_mm, 0.0]])
    return NetSpec(pos=pos, src=np.array([0], np.int32), dst=np.array([1], np.int32),
                   weight=np.array([w], np.float32), speed=None, speed_scalar=speed, dt_ms=dt_ms,
                   pulses=[(0, t_on_ms, t_on_ms + 2.0, 1.0)], name="chain2")


def random_small(seed: int, n: int = 12, p_edge: float = 0.3, dim: int = 2, speed: float = 0.05,
                 n_pulses: int = 2) -> NetSpec:
    """A tiny random geometric net for brute-force checks (dense random edges)."""
    rng = np.random.default_rng(seed)
    pos = rng.random((n, dim)) * 0.3
    ii, jj = np.nonzero((rng.random((n, n)) < p_edge) & ~np.eye(n, dtype=bool))
    src, dst = _sort_by_dst(ii.astype(np.int32), jj.astype(np.int32))
    w = rng.uniform(-1.0, 1.0, src.shape[0]).astype(np.float32)
    nodes = rng.choice(n, n_pulses, replace=False)
    pulses = [(int(j), float(rng.uniform(0.5, 3.0)), float(rng.uniform(3.5, 6.0)), 1.0) for j in nodes]
    return NetSpec(pos=pos, src=src, dst=dst, weight=w, speed=None, speed_scalar=speed, pulses=pulses,
                   obs=dict(OBS_DEFAULT, seed=seed + 11), name=f"small_s{seed}")


# --------------------------------------------------------------------------- estimator inputs
def candidates(spec: NetSpec):
    """Candidate directed pairs of a net: every ordered pair closer than the radius
    its edges were drawn within, with label 1 where the pair is an edge of the net
    (the ground truth a connectivity estimator is scored against)."""
    assert spec.radius > 0.0, "the net does not record its candidate radius"
    src, dst = _pairs_within(spec.pos, spec.radius)
    src, dst = _sort_by_dst(src, dst)
    N = np.int64(spec.n_nodes)
    # (dst, src) keys: the candidates are in this order; the edges are sorted for the lookup
    edge_key = np.sort(np.asarray(spec.dst, np.int64) * N + np.asarray(spec.src, np.int64))
    key = dst.astype(np.int64) * N + src.astype(np.int64)
    if edge_key.size == 0:
        return src, dst, np.zeros(key.shape[0], np.uint8)
    at = np.minimum(np.searchsorted(edge_key, key), edge_key.size - 1)
    label = (edge_key[at] == key).astype(np.uint8)
    return src, dst, label


def mlp_init(seed: int, in_dim: int = 33, hidden: int = 256):
    """He-uniform initial weights of the in_dim -> hidden -> hidden -> 1 network
    (biases zero), float32: W1 [in_dim, hidden], W2 [hidden, hidden], w3 [hidden]."""
    rng = np.random.default_rng(seed)

    def he(fan_in, shape):
        lim = np.sqrt(6.0 / fan_in)
        return rng.uniform(-lim, lim, shape).astype(np.float32)
    return dict(W1=he(in_dim, (in_dim, hidden)), b1=np.zeros(hidden, np.float32),
                W2=he(hidden, (hidden, hidden)), b2=np.zeros(hidden, np.float32),
                w3=he(hidden, (hidden,)), b3=np.zeros(1, np.float32))


def mlp_toy_batch(seed: int, B: int, in_dim: int = 33):
    """Seeded inputs in [-1, 1] and 0/1 labels for MLP checks."""
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1.0, 1.0, (B, in_dim)).astype(np.float32)
    y = (rng.random(B) < 0.5).astype(np.float32)
    return X, y


def shuffles(seed: int, n: int, epochs: int):
    """The order in which a training run visits n samples, epoch by epoch."""
    rng = np.random.default_rng(seed)
    return [rng.permutation(n).astype(np.int64) for _ in range(epochs)]


# ---------------------------------------------------------------------------
# The paper's standard test set (Sec. 3.5, Table modelspace): N vertices placed at
# random in a square or cube of side L with a minimum distance between any two,
# numbered from the centre outwards, connected by one of four graph classes at a
# low and a high edge density; delays from distance over one speed (Eq. delaydist).
TEST_SET_SIZES = (10, 30, 100, 300, 1000)
TEST_SET_CLASSES = ("lattice", "small_world", "scale_free", "random")
# (low, high) density parameter of each class: nearest neighbours, rewiring
# probability, edges per new vertex, fraction of the N^2 ordered pairs
TEST_SET_DENSITY = {"lattice": (3, 8), "small_world": (0.05, 0.15), "scale_free": (2, 4), "random": (0.10, 0.20)}


def min_distance_placement(rng, n: int, dim: int, side: float, d_min: float, max_tries: int = 1_000_000):
    """Random positions in [0, side)^dim, each candidate kept only if it is at least
    d_min from every vertex kept so far; vertices are then numbered by distance from
    the centre of the region (nearest first)."""
    pos = np.empty((n, dim))
    k = 0
    tries = 0
    while k < n:
        tries += 1
        if tries > max_tries:
            raise ValueError(f"cannot place {n} vertices {d_min} apart in a side of {side}")
        x = rng.random(dim) * side
        if k and np.min(np.sum((pos[:k] - x) ** 2, axis=1)) < d_min * d_min:
            continue
        pos[k] = x
        k += 1
    order = np.argsort(np.sum((pos - side / 2.0) ** 2, axis=1), kind="stable")
    return pos[order]


def _knn_in_edges(pos, k):
    """Directed edges i -> j from each vertex's k nearest neighbours i."""
    tree = cKDTree(pos)
    _, nn = tree.query(pos, k=k + 1)
    src = nn[:, 1:].reshape(-1)
    dst = np.repeat(np.arange(pos.shape[0]), k)
    return src.astype(np.int32), dst.astype(np.int32)


def test_set_net(n: int, dim: int, cls: str, density: str, seed: int = 0, side: float = 1.0,
                 d_min_frac: float = 0.5, speed: float = 0.1, dt_ms: float = 1.0) -> NetSpec:
    """One network of the test set.  Placement: d_min = d_min_frac * side * n^(-1/dim)
    (the cubic-packing distance, reduced to leave room for random placement).
    Classes (each vertex's in-edges; `density` "low" or "high" picks the parameter):
      lattice      its k nearest vertices (k = 3 or 8);
      small_world  the lattice, each edge's source re-drawn uniformly at random with
                   probability p (5 % or 15 %);
      scale_free   growth in the centre-out order: vertex v >= m links to m earlier
                   vertices drawn with probability proportional to their degree + 1
                   (m = 2 or 4), each link's direction drawn at random;
      random       every ordered pair i != j with probability p (10 % or 20 %).
    Weights U(0.1, 0.5), one speed (mm/ms), dt = 1 ms (the paper's Izhikevich
    benchmark step)."""
    if cls not in TEST_SET_CLASSES or density not in ("low", "high"):
        raise ValueError(f"unknown class {cls!r} or density {density!r}")
    rng = np.random.default_rng(seed)
    pos = min_distance_placement(rng, n, dim, side, d_min_frac * side * n ** (-1.0 / dim))
    par = TEST_SET_DENSITY[cls][0 if density == "low" else 1]
    if cls == "lattice":
        src, dst = _knn_in_edges(pos, min(par, n - 1))
    elif cls == "small_world":
        src, dst = _knn_in_edges(pos, min(3, n - 1) if density == "low" else min(8, n - 1))
        rewire = rng.random(src.size) < par
        for e in np.nonzero(rewire)[0]:
            s = int(rng.integers(0, n - 1))
            src[e] = s + (s >= dst[e])          # any vertex but the target
    elif cls == "scale_free":
        m = par
        deg = np.zeros(n)
        edges = []
        for v in range(1, n):
            cand = np.arange(v)
            k = min(m, v)
            p = (deg[:v] + 1.0) / np.sum(deg[:v] + 1.0)
            for u in rng.choice(cand, size=k, replace=False, p=p):
                edges.append((v, int(u)) if rng.random() < 0.5 else (int(u), v))
                deg[u] += 1
                deg[v] += 1
        src = np.array([a for a, _ in edges], np.int32)
        dst = np.array([b for _, b in edges], np.int32)
    else:
        mask = rng.random((n, n)) < par
        np.fill_diagonal(mask, False)
        src, dst = np.nonzero(mask)
        src, dst = src.astype(np.int32), dst.astype(np.int32)
    src, dst = _sort_by_dst(src.astype(np.int32), dst.astype(np.int32))
    w = rng.uniform(0.1, 0.5, src.size).astype(np.float32)
    obs = dict(OBS_DEFAULT, sample_every=max(1, int(round(1.0 / dt_ms))), seed=seed + 17)
    return NetSpec(pos=pos, src=src, dst=dst, weight=w, speed=None, speed_scalar=speed, dt_ms=dt_ms, obs=obs,
                   name=f"testset_{cls}_{density}_{dim}d_n{n}")


def test_set(seed0: int = 500, **kw) -> list:
    """The 80 networks: 2 dimensions x 5 sizes x 4 classes x 2 densities."""
    out = []
    i = 0
    for dim in (2, 3):
        for n in TEST_SET_SIZES:
            for cls in TEST_SET_CLASSES:
                for density in ("low", "high"):
                    out.append(test_set_net(n, dim, cls, density, seed=seed0 + i, **kw))
                    i += 1
    return out


def test_set_hh(spec: NetSpec, bg_rate_hz: float = 20.0, w_scale: float = 2.0, seed: int = 0,
                dt_ms: float = 0.03) -> NetSpec:
    """A test-set network with Hodgkin-Huxley + alpha-PSC nodes at the paper's HH step
    dt = 0.03 ms (delays re-quantised to it), driven by background pulses (2 ms of
    20 uA/cm^2 at bg_rate_hz per node; alone they give about 17 spikes/node/s).  With
    weight scale 2 the 300-vertex dense nets fire at about 20-70 spikes/node/s."""
    bg = dict(rate_hz=bg_rate_hz, amp=1.0, dur_ms=2.0, seed=seed + 4242)
    return hodgkin_huxley(dataclasses.replace(spec, background=bg), w_scale=w_scale, dt_ms=dt_ms)


def test_set_izh(spec: NetSpec, bg_rate_hz: float = 20.0, w_scale: float = 100.0, seed: int = 0) -> NetSpec:
    """A test-set network with Izhikevich + alpha-PSC nodes driven by background pulses
    (2 ms of 2500 pA at bg_rate_hz per node); at dt = 1 ms a weight scale of 100 puts
    the PSC peak near 55 pA for a weight of 0.3."""
    bg = dict(rate_hz=bg_rate_hz, amp=1.0, dur_ms=2.0, seed=seed + 4242)
    return izhikevich(dataclasses.replace(spec, background=bg), w_scale=w_scale)
