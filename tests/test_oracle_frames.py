"""Pins of the oracle's camera frame averaging (Sec. 3.3: a camera slower than the
step averages the calcium values of a frame into one reading) against the mean of
the readout state taken from the snapshots of the same run."""
import numpy as np
import pytest

import oracle
from paper_0908_3934_b300 import netgen


def _framed(spec, on=True, every=None):
    obs = dict(spec.obs, frame_average=on)
    if every is not None:
        obs["sample_every"] = every
    return netgen.dataclasses.replace(spec, obs=obs)


@pytest.mark.parametrize("model", ["fhn", "izh"])
def test_a_reading_is_the_mean_over_its_frame(model):
    base = netgen.tiny() if model == "fhn" else netgen.izhikevich(netgen.tiny(), w_scale=7000.0)
    n = 4000
    every = base.obs["sample_every"]
    r = oracle.simulate(_framed(base), n, snap_every=1, ev_cap=100000)
    plain = oracle.simulate(_framed(base, on=False), n, ev_cap=100000)
    C = r["snap_c"]                      # c after steps 1 .. n
    frames = C.reshape(n // every, every, -1).mean(axis=1)
    rest = 0.0 if model == "izh" else r["rest"][0]
    want = base.obs["gain"] * (rest + frames) + base.obs["offset"]
    assert r["y_clean"] == pytest.approx(want, rel=1e-12, abs=1e-12)
    # the readout mode changes neither the dynamics nor the noise draws
    assert np.array_equal(r["c"], plain["c"]) and np.array_equal(r["v"], plain["v"])
    assert np.allclose(r["y"] - r["y_clean"], plain["y"] - plain["y_clean"], rtol=0, atol=1e-12)
    assert not np.allclose(r["y_clean"], plain["y_clean"])


def test_one_step_frames_are_the_plain_readout():
    base = netgen.tiny()
    a = oracle.simulate(_framed(base, on=True, every=1), 600)
    b = oracle.simulate(_framed(base, on=False, every=1), 600)
    assert np.array_equal(a["y"], b["y"]) and np.array_equal(a["y_clean"], b["y_clean"])
