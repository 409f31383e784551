"""Camera frame averaging of the readout (Sec. 3.3) on the GPU against the FP64
oracle: windows aligned to the frames (gn_set_state starts a new frame, as each
oracle window does), the batched form, and checkpoints."""
import numpy as np
import pytest

from paper_0908_3934_b300 import geonet, netgen

from parity import assert_windows, windowed, windowed_izh

pytestmark = pytest.mark.gpu


def _framed(spec):
    return netgen.dataclasses.replace(spec, obs=dict(spec.obs, frame_average=True))


def test_fhn_frames_match_the_oracle():
    spec = _framed(netgen.tiny())
    net = geonet.Net(spec)
    worst, _ = windowed(spec, net, 4000, window=spec.obs["sample_every"])
    assert_windows(worst)


def test_izhikevich_frames_match_the_oracle():
    spec = _framed(netgen.izhikevich(netgen.tiny(), w_scale=7000.0))
    net = geonet.Net(spec)
    worst, n_spikes, _ = windowed_izh(spec, net, 4000)
    assert_windows(worst)
    assert n_spikes > 200


def test_frames_differ_from_last_values_and_batch_equals_single():
    specs = [_framed(netgen.batch_member(i, n=n)) for i, n in enumerate((64, 300, 1000))]
    b = geonet.Batch(specs)
    b.gn_batch_step(600)
    for i, sp in enumerate(specs):
        net = geonet.Net(sp)
        net.gn_step(600)
        y, _, _ = net.gn_observe()
        by = b.gn_batch_observe(i)[0]
        assert np.array_equal(y, by)
        plain = geonet.Net(netgen.dataclasses.replace(sp, obs=dict(sp.obs, frame_average=False)))
        plain.gn_step(600)
        assert not np.array_equal(y, plain.gn_observe()[0])


def test_checkpoint_at_a_frame_boundary_is_bit_exact():
    spec = _framed(netgen.large(n=3000, mean_deg=20, bg_rate_hz=200.0))
    every = spec.obs["sample_every"]
    a = geonet.Net(spec)
    a.gn_step(40 * every)
    blob = a.gn_save_state()
    a.gn_step(30 * every)
    b = geonet.Net(spec)
    b.gn_load_state(blob)
    b.gn_step(30 * every)
    ya, yb = a.gn_observe()[0], b.gn_observe()[0]
    assert np.array_equal(ya[-30:], yb[-30:])
