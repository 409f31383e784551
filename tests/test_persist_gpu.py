"""The persistent staged kernel (kernel 5: one cooperative launch per gn_step, each
CTA keeping its tile's gather keys and edge entries in shared memory, a counting
barrier in global memory between steps) against the staged kernel (kernel 3) on
the same tiles.

Both kernels sum a node's inputs in the same pieces and order and run the same node
update, so states, history, observations, arrivals and events must be the same
bits -- for each node model, with background pulses, over launches of uneven length
(the state passes through global memory between them), and at the tightest slot
reuse (a 4-slot ring, delays of 1 or 2 steps)."""
import numpy as np
import pytest

from paper_0908_3934_b300 import geonet, netgen

from parity import assert_windows, windowed

pytestmark = pytest.mark.gpu


def _snapshot(net, model):
    st = net.gn_get_state()
    out = {k: st[k] for k in ("v", "w", "c", "bg_count")}
    out["step"] = st["step"]
    info = net.gn_net_get_info()
    out["hist"] = net.gn_get_history(min(8, info["ring_depth"] - 1))
    y, first, _ = net.gn_observe()
    out["y"], out["first"] = y, first
    out["arrivals"] = net.gn_get_arrivals()
    node, step, _ = net.gn_get_events(cap=1 << 22)
    out["events"] = sorted(zip(node.tolist(), step.tolist()))
    if model != "fhn":
        out.update({f"izh_{k}": x for k, x in net.gn_get_izh_state().items()})
    if model == "hh":
        out.update({f"hh_{k}": x for k, x in net.gn_get_hh_gates().items()})
    return out


def _same(a, b, what):
    assert a.keys() == b.keys()
    for k in a:
        if isinstance(a[k], np.ndarray):
            assert a[k].shape == b[k].shape and np.array_equal(a[k], b[k]), (what, k)
        else:
            assert a[k] == b[k], (what, k)


def _run(spec, kind, chunks, model, monkeypatch, shape):
    monkeypatch.setenv("GN_STEP_SHAPE", str(shape))
    net = geonet.Net(spec, step_kernel=kind, obs_capacity=4096)
    info = net.gn_net_get_info()
    assert info["step_kernel"] == kind, info
    for c in chunks:
        net.gn_step(c)
    out = _snapshot(net, model)
    out["n_tiles"] = info["n_blocks"]
    out["cluster"] = info["step_cluster"]
    return out


def _cases():
    ts = netgen.test_set_net(1000, 2, "random", "high", seed=5)
    ts300 = netgen.test_set_net(300, 3, "random", "high", seed=6)
    sparse = netgen.test_set_net(1000, 2, "scale_free", "high", seed=8)
    mid = netgen.large(n=20000, mean_deg=20.0, seed=9)
    mid.background = dict(rate_hz=100.0, amp=1.0, dur_ms=2.0, seed=3)
    small = netgen.large(n=1200, mean_deg=20.0, bg_rate_hz=100.0, seed=10)
    # (spec, model, shape, runs as one cluster)
    return {
        "fhn_mid": (mid, "fhn", 0, 0),
        "fhn_mid_wide_tiles": (mid, "fhn", 2, 0),
        "izh_test_set_1000": (netgen.test_set_izh(ts), "izh", 0, 0),
        "hh_test_set_1000": (netgen.test_set_hh(ts), "hh", 0, 0),
        "izh_mid": (netgen.izhikevich(mid), "izh", 1, 0),
        "fhn_small_cluster": (small, "fhn", 0, 1),
        "izh_test_set_300": (netgen.test_set_izh(ts300), "izh", 0, 0),
        "izh_test_set_300_cluster": (netgen.test_set_izh(ts300), "izh", 6, 1),
        "hh_test_set_300_cluster": (netgen.test_set_hh(ts300), "hh", 6, 1),
        "hh_sparse_1000_cluster": (netgen.test_set_hh(sparse), "hh", 1, 1),
    }


@pytest.mark.parametrize("case", list(_cases()))
def test_persistent_equals_the_staged_kernel_bit_for_bit(case, monkeypatch):
    """Kernel 5 as a cooperative grid (more than 16 tiles) or as one thread-block
    cluster (at most 16), bit-identical to kernel 3 on the same tiles."""
    spec, model, shape, cluster = _cases()[case]
    chunks = [1, 7, 64, 100, 428]
    ref = _run(spec, 3, chunks, model, monkeypatch, shape)
    got = _run(spec, 5, chunks, model, monkeypatch, shape)
    assert ref["n_tiles"] == got["n_tiles"] > 1
    assert got.pop("cluster") == cluster and (got["n_tiles"] <= 16) == bool(cluster)
    ref.pop("cluster")
    if model == "fhn":
        assert np.abs(ref["v"]).max() > 0.1
    else:
        assert len(ref["events"]) > 0
    _same(ref, got, case)


def test_persistent_kernel_at_the_fastest_slot_reuse(monkeypatch):
    """A 4-slot ring and delays of 1 or 2 steps: slot n + 1, written in step n, is the
    slot step n - 3 read, so a CTA that updated before the previous step was complete
    everywhere, or gathered before its own wait of the step before, would change the
    bits.  3000 steps against kernel 3, and the first 60 steps against the oracle."""
    spec = netgen.large(n=30000, mean_deg=20.0, bg_rate_hz=100.0, seed=13)
    rng = np.random.default_rng(21)
    spec.delay = rng.integers(1, 3, spec.n_edges).astype(np.int32)
    spec.ring_depth = 4
    ref = _run(spec, 3, [3000], "fhn", monkeypatch, 0)
    got = _run(spec, 5, [3000], "fhn", monkeypatch, 0)
    assert got["n_tiles"] > 100 and got["cluster"] == 0
    assert np.abs(ref["v"]).max() > 0.1
    _same(ref, got, "fastest slot reuse")
    monkeypatch.setenv("GN_STEP_SHAPE", "0")
    worst, _ = windowed(spec, geonet.Net(spec, step_kernel=5), 60)
    assert_windows(worst)


def test_cluster_and_cooperative_grid_give_the_same_bits(monkeypatch):
    """The same small network (at most 16 tiles) with the cluster's barrier and, with
    GN_PERSIST_CLUSTER=0, with the counting barrier of the cooperative grid, at the
    fastest slot reuse (ring 4, delays 1 or 2), 2000 steps in uneven launches."""
    spec = netgen.large(n=1200, mean_deg=20.0, bg_rate_hz=100.0, seed=11)
    rng = np.random.default_rng(5)
    spec.delay = rng.integers(1, 3, spec.n_edges).astype(np.int32)
    spec.ring_depth = 4
    chunks = [3, 997, 1000]
    ref = _run(spec, 3, chunks, "fhn", monkeypatch, 0)
    clu = _run(spec, 5, chunks, "fhn", monkeypatch, 0)
    monkeypatch.setenv("GN_PERSIST_CLUSTER", "0")
    coop = _run(spec, 5, chunks, "fhn", monkeypatch, 0)
    assert clu.pop("cluster") == 1 and coop.pop("cluster") == 0
    ref.pop("cluster")
    assert np.abs(ref["v"]).max() > 0.1
    _same(ref, clu, "cluster")
    _same(ref, coop, "cooperative")


def test_persistent_kernel_refuses_what_it_cannot_hold(monkeypatch):
    monkeypatch.setenv("GN_STEP_SHAPE", "0")
    big = netgen.large(n=400000, mean_deg=40.0, seed=2)  # more tiles than the device holds at once
    with pytest.raises(geonet.GeonetError) as e:
        geonet.Net(big, step_kernel=5)
    assert e.value.status == geonet.GN_EINVAL
    plastic = netgen.izhikevich(netgen.tiny(), w_scale=7000.0)
    plastic.stdp = dict(alpha=1.0, beta=0.05)
    with pytest.raises(geonet.GeonetError) as e:
        geonet.Net(plastic, step_kernel=5)
    assert e.value.status == geonet.GN_EINVAL


@pytest.mark.parametrize("n", [20000, 1200])
def test_a_persistent_wait_that_gives_up_reports_a_timeout(monkeypatch, n):
    """With the poll budget at zero the copy waits (and the cooperative grid's barrier
    polls) give up at once: the CTAs record kStatusTimeout -- in the cluster form
    (1200 nodes) they keep passing the cluster's barriers without work to the end of
    the launch -- the host reports GN_ETIMEOUT at the next synchronising call, and
    the context stays usable."""
    spec = netgen.large(n=n, mean_deg=20.0, seed=9)
    monkeypatch.setenv("GN_STEP_SHAPE", "0")
    monkeypatch.setenv("GN_TEST_WAIT_LIMIT", "0")
    net = geonet.Net(spec, step_kernel=5)
    assert net.gn_net_get_info()["step_cluster"] == (1 if n == 1200 else 0)
    net.gn_step(50)
    with pytest.raises(geonet.GeonetError) as e:
        net.gn_synchronize()
    assert e.value.status == geonet.GN_ETIMEOUT
    monkeypatch.delenv("GN_TEST_WAIT_LIMIT")
    ok = geonet.Net(spec, step_kernel=5)
    ok.gn_step(40)
    ref = geonet.Net(spec, step_kernel=3)
    ref.gn_step(40)
    assert np.array_equal(ok.gn_get_state()["v"], ref.gn_get_state()["v"])
