"""CUDA path vs the FP64 oracle, through the C ABI (libgeonet.so).

Integers are compared bit for bit; floating point within the tolerance stated in
tests/parity.py (1e-4 relative, 1e-6 absolute, oracle re-synchronised every
1 ms of simulated time)."""
import numpy as np
import pytest

import oracle
from paper_0908_3934_b300 import geonet, netgen

from parity import assert_windows, ratio, windowed

pytestmark = pytest.mark.gpu


def Net(spec, **kw):
    from paper_0908_3934_b300 import geonet
    return geonet.Net(spec, **kw)


# ------------------------------------------------------------------ integers
def test_delays_bit_exact_tiny_and_fig2():
    spec = netgen.tiny()
    net = Net(spec)
    assert np.array_equal(net.gn_get_delays(), oracle.net_delays(spec))
    f = netgen.fig2([72, 148, 76, 52, 96, 68, 72, 88])
    assert Net(f).gn_get_delays().tolist() == [72, 148, 76, 52, 96, 68, 72, 88]


def test_delays_bit_exact_per_edge_speed_3d():
    spec = netgen.large(n=20000, mean_deg=40)
    net = Net(spec)
    D, cl = oracle.delays(spec.pos, spec.src, spec.dst, spec.speed, 0.0, spec.dt_ms)
    assert np.array_equal(net.gn_get_delays(), D)
    assert net.gn_net_get_info()["n_clamped"] == int(cl.sum())


def test_exact_halves_and_clamp():
    pos = np.array([[0.0, 0.0], [0.625, 0.0], [0.375, 0.0], [1e-4, 0.0]])
    spec = netgen.NetSpec(pos=pos, src=np.array([0, 0, 0], np.int32), dst=np.array([1, 2, 3], np.int32),
                          weight=np.ones(3, np.float32), speed=None, speed_scalar=1.0, dt_ms=0.25)
    net = Net(spec)
    assert net.gn_get_delays().tolist() == [3, 2, 1]
    assert net.gn_net_get_info()["n_clamped"] == 1


def test_fig2_arrivals_and_windows():
    spec = netgen.fig2([72, 148, 76, 52, 96, 68, 72, 88])
    net = Net(spec)
    net.gn_step(1000)
    assert net.gn_get_arrivals().tolist() == [201, 274, 350, 327, 423]
    worst, _ = windowed(spec, Net(spec), 4000)
    assert_windows(worst)


def test_two_node_chain_arrival():
    for d, s in [(0.5, 0.1), (0.25, 0.05)]:
        spec = netgen.chain2(dist_mm=d, speed=s)
        net = Net(spec)
        net.gn_step(1000)
        D = int(round(d / (s * 0.05)))
        assert net.gn_get_arrivals().tolist() == [101, 101 + D + 1]


# ------------------------------------------------------------------ config "tiny"
def test_tiny_first_200ms_windows():
    spec = netgen.tiny()
    worst, n_ev = windowed(spec, Net(spec), 4000)
    assert_windows(worst)
    assert n_ev > 20


def test_tiny_arrivals_and_early_events_bit_exact():
    """Uninterrupted run from rest: every first arrival whose value is an FP32
    normal number, and the events of the first 40 ms, match the oracle exactly."""
    spec = netgen.tiny()
    net = Net(spec)
    net.gn_step(4000)
    ref = oracle.simulate(spec, 4000)
    fa = net.gn_get_arrivals()
    ok = ref["first_arrival"] >= 0
    normal = np.abs(ref["first_value"]) >= 2.0 ** -126
    assert np.array_equal(fa[ok & normal], ref["first_arrival"][ok & normal])
    assert np.all(fa[~ok] == -1)
    node, step, _ = net.gn_get_events()
    got = sorted((int(s), int(j)) for j, s in zip(node, step) if s <= 800)
    want = sorted((int(s), int(j)) for j, s in zip(ref["ev_node"], ref["ev_step"]) if s <= 800)
    assert got == want and len(want) > 0


# Unwindowed drift bound: an FP32 evaluation of the same step (the numpy emulation
# of tests/fp32_emulation.py, pinned bit-exact to the oracle in float64) drifts from
# FP64 by the network's conditioning; the GPU is one more FP32 evaluation (its own
# polynomial form and contractions), so its drift is bounded by the worst of the
# emulation's three summation orders times this margin.
DRIFT_MARGIN = 2.0


def _emulated_drift(spec, ref, steps):
    """Worst, over the three summation orders, of the FP32 emulation's per-trace
    max-norm relative error (v~, w~, c~) and of its largest |c~ - c~_oracle| per trace."""
    import fp32_emulation as fe
    rel = dict(v=0.0, w=0.0, c=0.0)
    dc = np.zeros(spec.n_nodes)
    for order in fe.ORDERS:
        e = fe.emulate(spec, steps, np.float32, order)
        for k in rel:
            rel[k] = max(rel[k], fe.trace_maxnorm(e[k], ref[k]))
        dc = np.maximum(dc, np.abs(e["c"].astype(np.float64) - ref["c"]).max(0))
    return rel, dc


@pytest.mark.parametrize("which", ["tiny", "small_s0"])
def test_unwindowed_200ms_drift_is_the_fp32_conditioning(which):
    """200 ms from rest without re-synchronising, every step read back: the GPU's
    per-trace max-norm relative error of v~, w~ and c~ against the FP64 oracle is
    within DRIFT_MARGIN x the FP32 emulation's worst summation order."""
    import fp32_emulation as fe
    spec = netgen.tiny() if which == "tiny" else netgen.random_small(0, n=40, p_edge=0.2)
    steps = 4000
    ref = fe.oracle_trajectory(spec, steps)
    net = Net(spec)
    gpu = {k: np.zeros((steps + 1, spec.n_nodes)) for k in ("v", "w", "c")}
    for n in range(steps):
        net.gn_step(1)
        st = net.gn_get_state()
        for k in gpu:
            gpu[k][n + 1] = st[k]
    emu, _ = _emulated_drift(spec, ref, steps)
    got = {k: fe.trace_maxnorm(gpu[k], ref[k]) for k in gpu}
    print(which, "gpu", got, "emulation worst order", emu)
    for k in gpu:
        assert got[k] <= DRIFT_MARGIN * emu[k], (k, got[k], emu[k])


def test_tiny_full_horizon_runs_and_reports_drift():
    """1000 ms without re-synchronisation: arrivals exact; over the first 200 ms
    the noisy observations differ from the oracle's by the drift of the readout
    (the noise draws are the same), bounded per trace by DRIFT_MARGIN x the FP32
    emulation's worst |c~ - c~_oracle|."""
    import fp32_emulation as fe
    spec = netgen.tiny()
    net = Net(spec)
    net.gn_step(20000)
    ref = oracle.simulate(spec, 20000)
    y, first, _ = net.gn_observe()
    assert first == 0 and y.shape == ref["y"].shape
    fa = net.gn_get_arrivals()
    ok = (ref["first_arrival"] >= 0) & (np.abs(ref["first_value"]) >= 2.0 ** -126)
    assert np.array_equal(fa[ok], ref["first_arrival"][ok])
    _, dc = _emulated_drift(spec, fe.oracle_trajectory(spec, 4000), 4000)
    dy = np.abs(y[:200] - ref["y"][:200]).max(0)
    assert np.all(dy <= DRIFT_MARGIN * spec.obs["gain"] * dc + 1e-6), (dy.max(), dc.max())


def test_unstimulated_network_stays_exactly_at_rest():
    spec = netgen.tiny()
    spec.pulses = []
    net = Net(spec)
    net.gn_step(3000)
    st = net.gn_get_state()
    assert not st["v"].any() and not st["w"].any() and not st["c"].any()
    assert (net.gn_get_arrivals() == -1).all()
    assert net.gn_get_events()[0].size == 0


def test_zero_weights_windows():
    spec = netgen.tiny()
    spec.weight = np.zeros_like(spec.weight)
    net = Net(spec)
    worst, _ = windowed(spec, net, 2000)
    assert_windows(worst)
    st = net.gn_get_state()
    assert not st["v"][1:].any()


def test_raw_coupling_windows():
    spec = netgen.tiny()
    net = Net(spec, coupling="raw")
    worst, _ = windowed(spec, net, 2000, coupling="raw")
    assert_windows(worst)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_small_nets_windows(seed):
    spec = netgen.random_small(seed, n=40, p_edge=0.2)
    net = Net(spec)
    worst, _ = windowed(spec, net, 1500)
    assert_windows(worst)


# ------------------------------------------------------------------ layouts and edge cases
@pytest.mark.parametrize("step_kernel", [1, 2, 3])
def test_wide_edge_format_and_caller_order(step_kernel):
    spec = netgen.tiny()
    for kw in (dict(wide_edges=True), dict(renumber=False), dict(wide_edges=True, renumber=False)):
        net = Net(spec, step_kernel=step_kernel, **kw)
        worst, _ = windowed(spec, net, 600)
        assert_windows(worst)
        info = net.gn_net_get_info()
        assert info["edge_format"] == (1 if kw.get("wide_edges") else 0) and info["step_kernel"] == step_kernel


@pytest.mark.parametrize("step_kernel", [0, 1, 2, 3])
def test_every_step_kernel_on_a_multi_block_net(step_kernel):
    """Thousands of row blocks, so the persistent kernel cycles every pipeline stage
    many times per step."""
    spec = netgen.large(n=30000, mean_deg=40, bg_rate_hz=100.0)
    net = Net(spec, step_kernel=step_kernel)
    worst, n_ev = windowed(spec, net, 200, start=60)
    assert_windows(worst)
    info = net.gn_net_get_info()
    assert info["n_blocks"] > 100
    assert info["step_kernel"] == step_kernel if step_kernel else info["step_kernel"] in (1, 2, 3)


@pytest.mark.parametrize("step_kernel", [1, 2, 3])
def test_long_rows_take_the_whole_block_path(step_kernel):
    """A hub with in-degree 5000 (> one block's edge capacity; for the staged kernel
    157 pieces and a tile of its own) and ragged rows."""
    rng = np.random.default_rng(9)
    n = 6000
    pos = rng.random((n, 2))
    src = np.concatenate([np.arange(1, 5001), rng.integers(0, n, 3000)]).astype(np.int32)
    dst = np.concatenate([np.zeros(5000, np.int64), rng.integers(0, n, 3000)]).astype(np.int32)
    keep = src != dst
    src, dst = src[keep], dst[keep]
    w = rng.uniform(-0.2, 0.4, src.size).astype(np.float32)
    pulses = [(int(j), 2.0, 4.0, 1.0) for j in rng.choice(np.arange(1, 5001), 200, replace=False)]
    spec = netgen.NetSpec(pos=pos, src=src, dst=dst, weight=w, speed=None, speed_scalar=0.05, pulses=pulses)
    net = Net(spec, step_kernel=step_kernel)
    assert net.gn_net_get_info()["n_blocks"] >= 2
    worst, _ = windowed(spec, net, 800)
    assert_windows(worst)


def test_every_kernel_and_shape_gives_the_same_bits(monkeypatch):
    """Every step kernel sums a node's inputs in the same order (short rows in row
    order, rows over 48 edges as 32 lane-strided partials and a butterfly), so
    the row-block kernel in each CTA shape, the pipelined kernel and the staged
    kernel in each shape reach bit-identical states: a 20k-node net with 2.5 %
    hubs of in-degree 1000 and 100 Hz background, 300 steps from rest."""
    spec = netgen.roofline(seed=21, n=20000, bg_rate_hz=100.0)
    ref = None
    cases = [(1, s) for s in range(5)] + [(2, 0)] + [(3, s) for s in range(8)] + [(5, s) for s in range(8)]
    persistent = 0
    for kind, shape in cases:
        monkeypatch.setenv("GN_STEP_SHAPE", str(shape))
        try:
            net = Net(spec, step_kernel=kind)
        except geonet.GeonetError as e:  # kernel 5 in a shape whose tiles the device cannot hold at once
            assert kind == 5 and e.status == geonet.GN_EINVAL, (kind, shape)
            continue
        persistent += kind == 5
        net.gn_step(300)
        st = net.gn_get_state()
        hist = net.gn_get_history(8)
        if ref is None:
            ref = (st, hist)
            assert np.abs(st["v"]).max() > 0.1  # the background drove activity
            continue
        for k in ("v", "w", "c", "bg_count"):
            assert np.array_equal(st[k], ref[0][k]), (kind, shape, k)
        assert np.array_equal(hist, ref[1]), (kind, shape)
    assert persistent >= 2


def test_early_gathers_with_the_fastest_slot_reuse(monkeypatch):
    """The early-gather argument at its tightest: a 4-slot ring and delays of 1 or 2
    steps, so slot n + 1 written in step n is the slot step n - 3 read, on a grid
    with more tiles than the device holds at once (gathers before the grid wait).
    3000 steps bit-identical to the same kernel waiting first, and the first 60
    steps within the tolerance of the oracle, window by window."""
    spec = netgen.large(n=300000, mean_deg=20, bg_rate_hz=100.0)
    rng = np.random.default_rng(17)
    spec.delay = rng.integers(1, 3, spec.n_edges).astype(np.int32)
    spec.ring_depth = 4
    monkeypatch.setenv("GN_STEP_SHAPE", "3")
    monkeypatch.setenv("GN_STAGED_EARLY", "1")
    net = Net(spec, step_kernel=3)
    info = net.gn_net_get_info()
    assert info["ring_depth"] == 4 and info["max_delay"] == 2 and info["n_blocks"] > 148 * 6
    worst, _ = windowed(spec, net, 60)
    assert_windows(worst)
    out = []
    for early in ("1", "0"):
        monkeypatch.setenv("GN_STAGED_EARLY", early)
        n = Net(spec, step_kernel=3)
        n.gn_step(3000)
        out.append((n.gn_get_state(), n.gn_get_history(3), n.gn_get_arrivals()))
    (sa, ha, fa), (sb, hb, fb) = out
    assert np.abs(sa["v"]).max() > 0.1
    for k in ("v", "w", "c", "bg_count"):
        assert np.array_equal(sa[k], sb[k]), k
    assert np.array_equal(ha, hb) and np.array_equal(fa, fb)


@pytest.mark.parametrize("model", ["fhn", "izh", "hh"])
def test_early_gathers_give_the_same_bits(monkeypatch, model):
    """A staged grid with more tiles than the device holds at once gathers before
    its grid wait (history written two or more steps back); the states equal those
    of the same kernel waiting first, bit for bit, and the oracle's over one window:
    300k nodes, mean in-degree 20, 100 Hz background, each node model."""
    from parity import windowed_izh
    base = netgen.large(n=300000, mean_deg=20, bg_rate_hz=100.0)
    spec = {"fhn": base, "izh": netgen.izhikevich(base), "hh": netgen.hodgkin_huxley(base)}[model]
    monkeypatch.setenv("GN_STEP_SHAPE", "3")
    out = []
    for early in ("1", "0"):
        monkeypatch.setenv("GN_STAGED_EARLY", early)
        net = Net(spec, step_kernel=3)
        assert net.gn_net_get_info()["n_blocks"] > 148 * 6
        net.gn_step(400)
        extra = net.gn_get_izh_state() if model != "fhn" else {}
        out.append((net.gn_get_state(), net.gn_get_history(16), net.gn_get_events(), extra))
    (sa, ha, ea, xa), (sb, hb, eb, xb) = out
    for k in ("v", "w", "c", "bg_count"):
        assert np.array_equal(sa[k], sb[k]), k
    for k in xa:
        assert np.array_equal(xa[k], xb[k]), k
    assert np.array_equal(ha, hb)
    assert np.array_equal(ea[0], eb[0]) and np.array_equal(ea[1], eb[1])
    monkeypatch.setenv("GN_STAGED_EARLY", "1")
    net = Net(spec, step_kernel=3)
    if model == "fhn":
        worst, _ = windowed(spec, net, 20, start=200)
    else:
        worst, _, _ = windowed_izh(spec, net, 2 * spec.obs["sample_every"] if model == "izh" else 16, start=200)
    assert_windows(worst)


@pytest.mark.parametrize("model", ["fhn", "izh", "hh"])
def test_small_grid_early_gathers_give_the_same_bits(monkeypatch, model):
    """A staged grid the device holds at once gathers before its grid wait too, the
    next grid starting only after each CTA's own wait (so step n - 2 is complete when
    step n gathers); at the tightest slot reuse -- a 4-slot ring, delays of 1 or 2 steps
    -- 1500 steps in uneven launches equal those of the same kernel waiting first, bit
    for bit, and the first 60 steps equal the oracle's window by window (FHN)."""
    from parity import windowed_izh
    base = netgen.large(n=6000, mean_deg=20.0, bg_rate_hz=100.0, seed=23)
    rng = np.random.default_rng(29)
    base.delay = rng.integers(1, 3, base.n_edges).astype(np.int32)
    base.ring_depth = 4
    spec = {"fhn": base, "izh": netgen.izhikevich(base), "hh": netgen.hodgkin_huxley(base)}[model]
    monkeypatch.setenv("GN_STEP_SHAPE", "0")
    out = []
    for early in ("", "0"):
        if early:
            monkeypatch.setenv("GN_STAGED_EARLY", early)
        else:
            monkeypatch.delenv("GN_STAGED_EARLY", raising=False)
        net = Net(spec, step_kernel=3)
        assert 1 < net.gn_net_get_info()["n_blocks"] < 148
        for c in (1, 499, 1000):
            net.gn_step(c)
        extra = net.gn_get_izh_state() if model != "fhn" else {}
        out.append((net.gn_get_state(), net.gn_get_history(3), net.gn_get_events(), extra, net.gn_get_arrivals()))
    (sa, ha, ea, xa, fa), (sb, hb, eb, xb, fb) = out
    assert np.abs(sa["v"]).max() > 0.1 or len(ea[0]) > 0
    for k in ("v", "w", "c", "bg_count"):
        assert np.array_equal(sa[k], sb[k]), k
    for k in xa:
        assert np.array_equal(xa[k], xb[k]), k
    assert np.array_equal(ha, hb) and np.array_equal(fa, fb)
    assert np.array_equal(ea[0], eb[0]) and np.array_equal(ea[1], eb[1])
    if model == "fhn":
        monkeypatch.delenv("GN_STAGED_EARLY", raising=False)
        worst, _ = windowed(spec, Net(spec, step_kernel=3), 60)
        assert_windows(worst)


def test_staged_kernel_refuses_a_row_beyond_shared_memory():
    """One target with 70,000 distinct (source, delay) reads needs more shared memory
    than a CTA may have: the staged kernel is refused with GN_EINVAL, while the
    autotuner skips it and the row-block kernel runs the net."""
    rng = np.random.default_rng(12)
    n = 70001
    pos = rng.random((n, 2))
    src = np.arange(1, n, dtype=np.int32)
    dst = np.zeros(n - 1, np.int32)
    w = np.full(n - 1, 1e-4, np.float32)
    spec = netgen.NetSpec(pos=pos, src=src, dst=dst, weight=w, speed=None, speed_scalar=0.05)
    with pytest.raises(geonet.GeonetError) as e:
        Net(spec, step_kernel=3)
    assert e.value.status == geonet.GN_EINVAL and "staged" in str(e.value)
    net = Net(spec)
    net.gn_step(3)
    net.gn_synchronize()
    assert net.gn_net_get_info()["step_kernel"] in (1, 2)


def test_a_copy_wait_that_gives_up_reports_a_timeout(monkeypatch):
    """The staged kernel's bounded wait for its bulk copies: with the poll budget set
    to zero the first wait gives up, the CTA records kStatusTimeout, waits the full
    bound for its copies and leaves its rows untouched; the host reports
    GN_ETIMEOUT at the next synchronising call and the context stays usable."""
    spec = netgen.large(n=3000, mean_deg=20)
    monkeypatch.setenv("GN_TEST_WAIT_LIMIT", "0")
    net = Net(spec, step_kernel=3)
    net.gn_step(3)
    with pytest.raises(geonet.GeonetError) as e:
        net.gn_synchronize()
    assert e.value.status == geonet.GN_ETIMEOUT
    st = net.gn_get_state()  # the status word was cleared; no row was updated
    assert not st["v"].any() and not st["w"].any()
    monkeypatch.delenv("GN_TEST_WAIT_LIMIT")
    ok = Net(spec, step_kernel=3)
    ok.gn_step(40)
    ok.gn_synchronize()
    ref = Net(spec, step_kernel=1)
    ref.gn_step(40)
    assert np.array_equal(ok.gn_get_state()["v"], ref.gn_get_state()["v"])


def test_no_edges_and_one_node():
    for n in (1, 37):
        spec = netgen.NetSpec(pos=np.zeros((n, 3)), src=np.zeros(0, np.int32), dst=np.zeros(0, np.int32),
                              weight=np.zeros(0, np.float32), speed=None, speed_scalar=1.0,
                              pulses=[(n - 1, 1.0, 3.0, 1.0)])
        net = Net(spec)
        worst, _ = windowed(spec, net, 400)
        assert_windows(worst)


def test_largest_delay_that_fits_the_ring():
    """D = R - 2 is the largest delay a ring of R slots holds; D = R - 1 is rejected."""
    from paper_0908_3934_b300 import geonet
    spec = netgen.fig2([62, 62, 30, 7, 1, 62, 2, 62])
    net = Net(spec, ring_depth=64)
    worst, _ = windowed(spec, net, 1200)
    assert_windows(worst)
    with pytest.raises(geonet.GeonetError) as e:
        Net(netgen.fig2([63, 1, 1, 1, 1, 1, 1, 1]), ring_depth=64)
    assert e.value.status == geonet.GN_ERANGE


def test_slow_conduction_deep_ring_windows():
    """The delay-stress size (every speed x 0.1): delays of up to ~2400 steps in a
    ring sized afresh (4096 slots, packed keys with 12 delay bits); windows against
    the oracle from step 2100, where gathers of delays beyond 2000 steps read
    written history."""
    spec = netgen.delay_stress(netgen.roofline(seed=23, n=5000, bg_rate_hz=100.0))
    D = oracle.net_delays(spec)
    assert 2048 < D.max() < 4094
    net = Net(spec)
    info = net.gn_net_get_info()
    assert info["max_delay"] == D.max() and info["ring_depth"] == 4096 and info["edge_format"] == 0
    worst, _ = windowed(spec, net, 100, start=2100)
    assert_windows(worst)


def test_background_counters_and_arrivals():
    spec = netgen.large(n=3000, mean_deg=20, bg_rate_hz=200.0)
    worst, _ = windowed(spec, Net(spec), 1000)
    assert_windows(worst)
    net = Net(spec)
    net.gn_step(1000)
    ref = oracle.simulate(spec, 1000)
    ok = (ref["first_arrival"] >= 0) & (np.abs(ref["first_value"]) >= 2.0 ** -126)
    assert np.array_equal(net.gn_get_arrivals()[ok], ref["first_arrival"][ok])
    assert np.array_equal(net.gn_get_state()["bg_count"], ref["bg_count"])


def test_checkpoint_resume_is_bit_exact():
    spec = netgen.large(n=3000, mean_deg=20, bg_rate_hz=200.0)
    a = Net(spec)
    a.gn_step(777)
    blob = a.gn_save_state()
    a.gn_step(777)
    b = Net(spec)
    b.gn_load_state(blob)
    b.gn_step(777)
    sa, sb = a.gn_get_state(), b.gn_get_state()
    for k in ("v", "w", "c", "bg_count"):
        assert np.array_equal(sa[k], sb[k]), k
    assert sa["step"] == sb["step"] == 1554
    assert np.array_equal(a.gn_get_history(16), b.gn_get_history(16))


def test_observation_overflow_keeps_the_latest():
    from paper_0908_3934_b300 import geonet
    spec = netgen.tiny()
    net = Net(spec, obs_capacity=8)
    net.gn_step(20 * 20)
    y, first, st = net.gn_observe()
    assert st == geonet.GN_EOVERFLOW and first == 12 and y.shape[0] == 8
    ref = oracle.simulate(spec, 400)
    assert ratio(y, ref["y"][12:]) <= 1.0


def test_event_overflow_is_reported():
    from paper_0908_3934_b300 import geonet
    spec = netgen.tiny()
    net = Net(spec, event_capacity=5)
    net.gn_step(4000)
    node, step, st = net.gn_get_events()
    assert st == geonet.GN_EOVERFLOW and node.size == 5


# ------------------------------------------------------------------ full sizes, bench launch configuration
@pytest.fixture(scope="module")
def large_spec():
    return netgen.large()


def test_large_full_size_sampled(large_spec):
    """N = 100,000, ~10M edges, 5 Hz background: delays bit-exact; two 20-step
    windows after 200 steps, compared on every node."""
    spec = large_spec
    net = Net(spec)
    assert np.array_equal(net.gn_get_delays(), oracle.net_delays(spec))
    worst, n_ev = windowed(spec, net, 40, start=200)
    assert_windows(worst)


def test_batched_full_size_sampled():
    """The 4096-network ensemble (3.34M nodes, 61M edges) in the configuration the
    bench times -- the kernel and schedule its first step picks by timing (on a B300
    the L2-blocked staged form) -- with 32 sampled members: delays bit-exact, then
    each loaded with the oracle's state after 500 steps (most members active by
    then) and compared over one 20-step window, every node of each."""
    from paper_0908_3934_b300 import geonet
    specs = netgen.batch(4096, seed0=1000)
    b = geonet.Batch(specs, obs_capacity=64)
    b.gn_batch_step(20)  # picks the kernel and schedule, as the bench's warm-up does
    info = b.gn_batch_get_info()
    assert info["n_nets"] == 4096 and info["step_kernel"] in (1, 3)
    sample = [int(i) for i in np.random.default_rng(12).choice(4096, 32, replace=False)]
    K, n0 = 20, 500
    refs, depth, nxt = {}, {}, {}
    for i in sample:
        D = oracle.net_delays(specs[i])
        assert np.array_equal(b.gn_batch_get_delays(i), D), i
        depth[i] = int(D.max()) + 1
        refs[i] = oracle.simulate(specs[i], n0, hist_depth=depth[i], want_y=False)
    b.gn_batch_set_step(n0)
    for i in sample:
        r = refs[i]
        b.gn_batch_set_state(i, r["hist"].astype(np.float32), r["w"].astype(np.float32),
                             r["c"].astype(np.float32), r["bg_count"])
        nxt[i] = oracle.simulate(specs[i], K, hist_depth=depth[i],
                                 init=dict(n0=n0, v=r["v"], w=r["w"], c=r["c"], bg_count=r["bg_count"],
                                           hist=r["hist"]))
    b.gn_batch_step(K)
    worst, active = 0.0, 0
    for i in sample:
        g = b.gn_batch_get_state(i)
        for k in ("v", "w", "c"):
            worst = max(worst, ratio(g[k], nxt[i][k]))
        y, _, _ = b.gn_batch_observe(i)
        worst = max(worst, ratio(y, nxt[i]["y"]))
        active += int(np.abs(nxt[i]["v"]).max() > 1e-3)
    assert worst <= 1.0, worst
    assert active >= 16, active
    b.gn_batch_destroy()


def test_roofline_full_size_sampled():
    """N = 1,000,000, ~50M edges with 2.5 % hubs of in-degree 1000, ring of 256
    steps (the benchmark's network): delays bit-exact; one 20-step window after
    40 steps, compared on every node."""
    spec = netgen.roofline()
    net = Net(spec)
    D = oracle.net_delays(spec)
    assert np.array_equal(net.gn_get_delays(), D)
    info = net.gn_net_get_info()
    assert info["ring_depth"] == 256 and info["edge_format"] == 0
    worst, _ = windowed(spec, net, 20, start=40)
    assert_windows(worst)


@pytest.mark.parametrize("size", ["hubs5", "slow"])
def test_secondary_roofline_sizes_full_size_window(size):
    """The 1M-node net's two secondary sizes in the launch configuration bench.py
    times: the literal 5 % hubs of in-degree 1000 beside non-hubs of mean in-degree 50
    (~97.5M edges), and every conduction speed x 0.1 (delays to ~410 steps, a 512-slot
    ring).  Delays bit-exact; one 20-step window after 40 steps, compared on every node."""
    spec = (netgen.roofline(hub_frac=0.05, mean_deg=97.5) if size == "hubs5"
            else netgen.delay_stress(netgen.roofline()))
    net = Net(spec)
    assert np.array_equal(net.gn_get_delays(), oracle.net_delays(spec))
    info = net.gn_net_get_info()
    if size == "slow":
        assert info["ring_depth"] == 512 and info["max_delay"] > 300
    worst, _ = windowed(spec, net, 20, start=40)
    assert_windows(worst)


@pytest.mark.parametrize("model", ["izh", "hh", "izh_stdp"])
def test_roofline_full_size_spiking_sampled(model):
    """The benchmark's 1M-node network with each spiking node model (Izhikevich at
    dt 0.05 ms, Hodgkin-Huxley at dt 0.03 ms, Izhikevich with plastic weights) in
    the launch configuration bench.py times: one window after 2 ms from rest (the
    background pulses have made about 10^4 spikes), compared on every node (and
    every weight)."""
    from parity import windowed_izh
    base = netgen.roofline()
    if model == "hh":
        spec = netgen.hodgkin_huxley(base)
    else:
        spec = netgen.izhikevich(base)
        if model == "izh_stdp":
            spec = netgen.dataclasses.replace(spec, stdp=dict(alpha=5.0, beta=0.05))
    net = Net(spec)
    every = spec.obs["sample_every"]
    worst, n_spikes, excused = windowed_izh(spec, net, 8 if model == "hh" else every,
                                            start=67 if model == "hh" else 40)
    assert_windows(worst)
    assert excused < 0.001 * spec.n_nodes


def test_asynchronous_observation_copies_match_the_synchronous_ones():
    """gn_observe_async queues the same rows as gn_observe would return, behind the
    steps taken so far, while later steps run; two chunks alternate two buffers."""
    spec = netgen.large(n=20000, mean_deg=20, bg_rate_hz=100.0)
    a, b = Net(spec), Net(spec)
    every = spec.obs["sample_every"]
    rows = 500 // every
    bufs = [np.zeros((rows, spec.n_nodes), np.float32) for _ in range(2)]
    got = []
    for c in range(4):
        a.gn_step(500)
        ya, first_a, _ = a.gn_observe(rows)
        b.gn_step(500)
        b.gn_observe_wait()
        if c:
            got.append(bufs[(c - 1) % 2].copy())
        n, first_b, _ = b.gn_observe_async(bufs[c % 2], rows)
        assert n == rows and first_b == first_a == c * rows
        if c:
            assert np.array_equal(got[-1], prev)
        prev = ya.copy()
    b.gn_observe_wait()
    assert np.array_equal(bufs[3 % 2], prev)
