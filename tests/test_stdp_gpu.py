"""Spike-time-dependent plasticity (Sec. 3.2, the plasticity transition G_ij of Eq.
omegatrans with the spike-time state s_j) on the GPU against the FP64 oracle,
through the C ABI.

Spikes compared exactly; weights, s and the node state within 1e-4 relative (floor
1e-6 of the quantity's largest magnitude) per window, the oracle's state --
weights and the history of s included -- loaded at each window start
(tests/parity.py)."""
import numpy as np
import pytest

import oracle
from paper_0908_3934_b300 import geonet, netgen

from parity import assert_windows, windowed_izh

pytestmark = pytest.mark.gpu

STDP = dict(alpha=0.5, beta=0.05)


def _plastic(spec, **kw):
    return netgen.dataclasses.replace(spec, stdp=dict(STDP, **kw))


def test_zero_rate_is_bit_identical_to_the_static_net():
    """With alpha = 0 the plastic kernel (packed spike-time ring words, weights read
    from its entries) gives the static kernel's states bit for bit."""
    base = netgen.izhikevich(netgen.roofline(seed=21, n=20000, bg_rate_hz=100.0))
    a = geonet.Net(base, step_kernel=3)
    b = geonet.Net(_plastic(base, alpha=0.0))
    a.gn_step(600)
    b.gn_step(600)
    for x, y in ((a.gn_get_state(), b.gn_get_state()), (a.gn_get_izh_state(), b.gn_get_izh_state())):
        for k in x:
            assert np.array_equal(x[k], y[k]), k
    assert np.array_equal(a.gn_get_history(8), b.gn_get_history(8))
    assert np.array_equal(b.gn_get_weights(), np.asarray(base.weight, np.float32))
    ea, eb = a.gn_get_events(), b.gn_get_events()
    assert len(ea[0]) > 0 and np.array_equal(ea[0], eb[0]) and np.array_equal(ea[1], eb[1])


def test_tiny_net_from_rest_spikes_and_weights():
    """64 Izhikevich nodes with plastic weights (up to 3 % weight change), 3500 steps
    from rest without re-synchronising: the same spikes step for step, the weights
    and s within tolerance of the oracle's."""
    spec = _plastic(netgen.izhikevich(netgen.tiny(), w_scale=7000.0), alpha=50.0)
    n = 3500
    ref = oracle.simulate(spec, n, ev_cap=100000, want_y=False)
    assert ref["ev_count"] > 150 and ref["min_peak_gap"].min() > 1e-2
    net = geonet.Net(spec)
    net.gn_step(n)
    node, step, _ = net.gn_get_events()
    assert sorted(zip(node.tolist(), step.tolist())) == sorted(zip(ref["ev_node"].tolist(), ref["ev_step"].tolist()))
    w = net.gn_get_weights().astype(np.float64)
    changed = ref["w_final"] != np.asarray(spec.weight, np.float64)
    assert changed.sum() > 20
    err = np.abs(w - ref["w_final"]) / np.maximum(1e-4 * np.abs(ref["w_final"]), 1e-6 * np.abs(ref["w_final"]).max())
    assert err.max() <= 1.0
    s = net.gn_get_stdp_history(1)[0].astype(np.float64)
    assert np.allclose(s, ref["s"], rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("model", ["izh", "hh"])
def test_tiny_net_windows(model):
    """Weights change by up to 7 % (Izhikevich, 4000 steps) and 3 % (Hodgkin-Huxley,
    1600 steps at dt = 0.03 ms)."""
    base = netgen.tiny()
    if model == "izh":
        spec, n = _plastic(netgen.izhikevich(base, w_scale=7000.0), alpha=50.0), 4000
    else:
        spec, n = _plastic(netgen.hodgkin_huxley(base, w_scale=10.0), alpha=0.05), 1600
    net = geonet.Net(spec)
    worst, n_spikes, excused = windowed_izh(spec, net, n)
    print("worst ratios", worst, "excused", excused)
    assert_windows(worst)
    assert n_spikes > 40


def test_multi_tile_net_windows():
    """30k Izhikevich nodes, in-degree 40, 100 Hz background pulses, plastic weights."""
    spec = _plastic(netgen.izhikevich(netgen.large(n=30000, mean_deg=40, bg_rate_hz=100.0)), alpha=5.0)
    net = geonet.Net(spec)
    worst, n_spikes, excused = windowed_izh(spec, net, 200, start=100)
    print("worst ratios", worst, "excused", excused)
    assert_windows(worst)
    assert n_spikes > 0


def test_checkpoint_resume_is_bit_exact():
    spec = _plastic(netgen.izhikevich(netgen.large(n=3000, mean_deg=20, bg_rate_hz=200.0)))
    a = geonet.Net(spec)
    a.gn_step(777)
    blob = a.gn_save_state()
    a.gn_step(777)
    b = geonet.Net(spec)
    b.gn_load_state(blob)
    b.gn_step(777)
    assert not np.array_equal(a.gn_get_weights(), np.asarray(spec.weight, np.float32))
    assert np.array_equal(a.gn_get_weights(), b.gn_get_weights())
    assert np.array_equal(a.gn_get_stdp_history(4), b.gn_get_stdp_history(4))
    for k in ("V", "r", "p"):
        assert np.array_equal(a.gn_get_izh_state()[k], b.gn_get_izh_state()[k]), k


def test_plasticity_calls_are_checked():
    tiny_izh = netgen.izhikevich(netgen.tiny())
    with pytest.raises(geonet.GeonetError) as e:
        geonet.Net(tiny_izh).gn_get_weights()
    assert e.value.status == geonet.GN_EINVAL
    with pytest.raises(geonet.GeonetError) as e:
        geonet.Net(_plastic(netgen.tiny()))
    assert e.value.status == geonet.GN_EINVAL
    with pytest.raises(geonet.GeonetError) as e:
        geonet.Net(_plastic(tiny_izh), step_kernel=1)
    assert e.value.status == geonet.GN_EINVAL
    net = geonet.Net(_plastic(tiny_izh))
    w = np.linspace(-1.0, 1.0, tiny_izh.n_edges).astype(np.float32)
    net.gn_set_weights(w)
    assert np.array_equal(net.gn_get_weights(), w)
    s = (np.arange(tiny_izh.n_nodes)[None, :] * tiny_izh.dt_ms).astype(np.float32)  # whole steps
    net.gn_set_stdp_history(s)
    assert np.array_equal(net.gn_get_stdp_history(1), s)
