"""The resident step kernel (kernel 4: a small network held in one CTA's shared
memory, many steps per launch) against the row-block kernel (kernel 1) and the
FP64 oracle.

Every step kernel sums a node's inputs in the same order and runs the same node
update, so the resident kernel's states, history, observations, arrivals and
events must equal kernel 1's bit for bit -- for each node model, with pulses,
background pulses, RAW coupling, camera frame averaging and heterogeneous cells,
whether the steps come in one launch or in many of uneven length."""
import numpy as np
import pytest

from paper_0908_3934_b300 import geonet, netgen

from parity import assert_windows, windowed, windowed_izh

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
    node, step, _ = net.gn_get_events(cap=1 << 20)
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


def _run(spec, kind, chunks, model, monkeypatch, shape=None):
    if shape is not None:
        monkeypatch.setenv("GN_STEP_SHAPE", str(shape))
    else:
        monkeypatch.delenv("GN_STEP_SHAPE", raising=False)
    net = geonet.Net(spec, step_kernel=kind, obs_capacity=4096)
    assert net.gn_net_get_info()["step_kernel"] == kind
    for c in chunks:
        net.gn_step(c)
    return _snapshot(net, model)


def _cases():
    tiny = netgen.tiny()
    bg = netgen.tiny()
    bg.background = dict(rate_hz=200.0, amp=1.0, dur_ms=2.0, seed=5)
    frames = netgen.tiny()
    frames.obs = dict(frames.obs, frame_average=1)
    ts = netgen.test_set_net(300, 2, "random", "high", seed=7)
    return {
        "fhn_tiny": (tiny, "fhn"),
        "fhn_background": (bg, "fhn"),
        "fhn_raw": (tiny, "fhn_raw"),
        "fhn_frames": (frames, "fhn"),
        "izh_tiny": (netgen.izhikevich(netgen.tiny(), w_scale=7000.0), "izh"),
        "izh_test_set": (netgen.test_set_izh(ts), "izh"),
        "izh_cells": (netgen.mixed_cells(netgen.izhikevich(netgen.tiny(), w_scale=7000.0), seed=3), "izh"),
        "hh_tiny": (netgen.hodgkin_huxley(netgen.tiny(), w_scale=10.0), "hh"),
        "hh_test_set": (netgen.test_set_hh(ts), "hh"),
        "hh_background": (netgen.hodgkin_huxley(bg), "hh"),
    }


@pytest.mark.parametrize("case", list(_cases()))
def test_resident_equals_the_row_block_kernel_bit_for_bit(case, monkeypatch):
    spec, model = _cases()[case]
    if model == "fhn_raw":
        spec = netgen.tiny()
        spec.coupling = "raw"
        model = "fhn"
    chunks = [1, 7, 64, 100, 428]          # uneven launches: the state moves through global memory between them
    ref = _run(spec, 1, chunks, model, monkeypatch, shape=0)
    if model == "fhn":
        assert np.abs(ref["v"]).max() > 0.1
    else:
        assert len(ref["events"]) > 0
    for shape in range(3):
        got = _run(spec, 4, chunks, model, monkeypatch, shape=shape)
        _same(ref, got, (case, shape))
    # one launch of all the steps, in the default shape
    got = _run(spec, 4, [sum(chunks)], model, monkeypatch)
    _same(ref, got, (case, "one launch"))


def test_autotuner_picks_the_resident_kernel_for_a_small_net():
    net = geonet.Net(netgen.tiny())
    net.gn_step(64)
    assert net.gn_net_get_info()["step_kernel"] == 4


def test_resident_windows_against_the_oracle():
    spec = netgen.tiny()
    worst, n_ev = windowed(spec, geonet.Net(spec, step_kernel=4), 4000)
    assert_windows(worst)
    assert n_ev > 20
    hh = netgen.hodgkin_huxley(netgen.tiny(), w_scale=10.0)
    worst, n_spikes, _ = windowed_izh(hh, geonet.Net(hh, step_kernel=4), 3000)
    assert_windows(worst)
    assert n_spikes > 100


def test_resident_kernel_refuses_a_net_it_cannot_hold():
    big = netgen.large(n=20000, mean_deg=40.0)
    with pytest.raises(geonet.GeonetError) as e:
        geonet.Net(big, step_kernel=4)
    assert e.value.status == geonet.GN_EINVAL
    plastic = netgen.izhikevich(netgen.tiny(), w_scale=7000.0)
    plastic.stdp = dict(alpha=1.0, beta=0.05)
    with pytest.raises(geonet.GeonetError):
        geonet.Net(plastic, step_kernel=4)


def test_switching_kernels_mid_run_keeps_the_bits(monkeypatch):
    """A checkpoint taken under the resident kernel resumes under kernel 1 (and
    the other way round) to the same bits as an uninterrupted kernel-1 run."""
    spec = netgen.hodgkin_huxley(netgen.tiny(), w_scale=10.0)
    ref = _run(spec, 1, [300, 300], "hh", monkeypatch, shape=0)
    for first, second in ((4, 1), (1, 4)):
        a = geonet.Net(spec, step_kernel=first, obs_capacity=4096)
        a.gn_step(300)
        buf = a.gn_save_state()
        b = geonet.Net(spec, step_kernel=second, obs_capacity=4096)
        b.gn_load_state(buf)
        b.gn_step(300)
        got = _snapshot(b, "hh")
        for k in ("v", "w", "c", "bg_count", "hist", "izh_V", "izh_r", "izh_p", "hh_m", "hh_n", "hh_h"):
            assert np.array_equal(got[k], ref[k]), (first, second, k)
