"""The Izhikevich + alpha-PSC + calcium node model (Eq. izsimple, izpsc, alphapsc,
spd, casimple; Sec. 3.1-3.3) on the GPU against the FP64 oracle, through the C ABI.

Spikes (events) and first spikes are compared exactly; V, W, calcium, r, p and y
within 1e-4 relative (1e-6 absolute) per 1 ms window, the oracle's state loaded at
each window start (tests/parity.py)."""
import numpy as np
import pytest

import oracle
from paper_0908_3934_b300 import geonet, netgen

from parity import assert_windows, windowed_izh

pytestmark = pytest.mark.gpu


def test_tiny_net_windows_and_spikes():
    """64 nodes building up to self-sustained activity (about 400 spikes in 200 ms)."""
    spec = netgen.izhikevich(netgen.tiny(), w_scale=7000.0)
    net = geonet.Net(spec)
    worst, n_spikes, excused = windowed_izh(spec, net, 4000)
    assert_windows(worst)
    assert n_spikes > 200 and excused < 0.01 * 64 * 200


def test_first_spikes_exact_without_resynchronising():
    """One spike travels one hop (node 0 pulsed, one target crosses threshold): a run
    from rest gives the same spikes, step for step, as the oracle."""
    spec = netgen.izhikevich(netgen.tiny(), w_scale=6000.0)
    ref = oracle.simulate(spec, 6000, ev_cap=10000, want_y=False)
    assert ref["ev_count"] == 2 and ref["min_peak_gap"].min() > 1e-2
    net = geonet.Net(spec)
    net.gn_step(6000)
    node, step, _ = net.gn_get_events()
    assert sorted(zip(node.tolist(), step.tolist())) == sorted(zip(ref["ev_node"].tolist(), ref["ev_step"].tolist()))
    assert np.array_equal(net.gn_get_arrivals(), ref["first_arrival"].astype(np.int64))


@pytest.mark.parametrize("step_kernel", [1, 3])
def test_multi_block_net_windows(step_kernel):
    """30k nodes, in-degree 40, 100 Hz background pulses: many row blocks / tiles."""
    spec = netgen.izhikevich(netgen.large(n=30000, mean_deg=40, bg_rate_hz=100.0))
    net = geonet.Net(spec, step_kernel=step_kernel)
    worst, n_spikes, _ = windowed_izh(spec, net, 200, start=100)
    assert_windows(worst)
    assert n_spikes > 0


def test_every_kernel_and_shape_gives_the_same_bits(monkeypatch):
    """The shared summation order holds for spike inputs too: every step kernel and
    CTA shape reaches bit-identical Izhikevich states (hubs of in-degree 1000)."""
    spec = netgen.izhikevich(netgen.roofline(seed=21, n=20000, bg_rate_hz=100.0))
    ref = None
    for kind, shape in [(1, s) for s in range(5)] + [(2, 0)] + [(3, s) for s in range(8)]:
        monkeypatch.setenv("GN_STEP_SHAPE", str(shape))
        net = geonet.Net(spec, step_kernel=kind)
        net.gn_step(600)
        st, iz = net.gn_get_state(), net.gn_get_izh_state()
        cur = [st["w"], st["c"], iz["V"], iz["r"], iz["p"], net.gn_get_history(8)]
        if ref is None:
            ref = cur
            assert len(net.gn_get_events()[0]) > 0
            continue
        for a, b in zip(cur, ref):
            assert np.array_equal(a, b), (kind, shape)


def test_checkpoint_resume_is_bit_exact():
    spec = netgen.izhikevich(netgen.large(n=3000, mean_deg=20, bg_rate_hz=200.0))
    a = geonet.Net(spec)
    a.gn_step(777)
    blob = a.gn_save_state()
    a.gn_step(777)
    b = geonet.Net(spec)
    b.gn_load_state(blob)
    b.gn_step(777)
    for k in ("V", "r", "p"):
        assert np.array_equal(a.gn_get_izh_state()[k], b.gn_get_izh_state()[k]), k
    sa, sb = a.gn_get_state(), b.gn_get_state()
    for k in ("v", "w", "c", "bg_count"):
        assert np.array_equal(sa[k], sb[k]), k


def test_model_specific_calls_are_checked():
    with pytest.raises(geonet.GeonetError) as e:
        geonet.Net(netgen.tiny()).gn_get_izh_state()
    assert e.value.status == geonet.GN_EINVAL
    with pytest.raises(geonet.GeonetError) as e:  # one node model per batch
        geonet.Batch([netgen.izhikevich(netgen.tiny()), netgen.tiny()])
    assert e.value.status == geonet.GN_EINVAL


@pytest.mark.parametrize("cls", ["small_world", "scale_free", "random"])
def test_test_set_networks_at_one_millisecond_steps(cls):
    """Networks of the standard test set (Sec. 3.5) with Izhikevich nodes at the
    paper's benchmark step dt = 1 ms, 20 Hz background pulses: 500 steps, one 1 ms
    observation interval (one step) per window."""
    spec = netgen.test_set_izh(netgen.test_set_net(300, 2, cls, "high", seed=7))
    net = geonet.Net(spec)
    worst, n_spikes, _ = windowed_izh(spec, net, 500)
    assert_windows(worst)
    assert n_spikes > 50
