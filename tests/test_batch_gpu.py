"""Batched form (gn_batch_*): many independent networks of uneven size stepped
together -- by the persistent k_batch or by one staged launch per step over every
member's tiles -- checked against the single-network path and the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_0908_3934_b300 import netgen

from parity import ratio

pytestmark = pytest.mark.gpu


@pytest.fixture(params=[1, 3, 4, 5], ids=["persistent", "staged", "staged_l2_groups", "staged_lanes"], autouse=True)
def batch_kernel(request, monkeypatch):
    """Every test runs with each batch kernel (GN_BATCH_KERNEL); the staged form
    also with L2 blocking in two lanes sharing a 512 KB budget, which cuts these
    small members into groups of one to a few networks -- as a chain of launches
    per lane (4) and as one persistent launch of both lanes (5)."""
    monkeypatch.setenv("GN_BATCH_KERNEL", str(request.param))
    monkeypatch.setenv("GN_BATCH_GROUP_KB", "512")
    monkeypatch.setenv("GN_BATCH_LANES", "2")
    return request.param


def _specs(n, seed0=1000, n_hi=1500):
    return [netgen.batch_member(seed0 + i, n_hi=n_hi) for i in range(n)]


def test_batch_equals_single_networks_bit_for_bit(batch_kernel):
    """A member of the batch follows exactly the trajectory of the same network run
    alone (same per-row summation order and node update), over 2000 steps (1500 =
    23 graphs of 64 steps and a ragged tail for the staged kernel)."""
    from paper_0908_3934_b300 import geonet
    specs = _specs(24)
    b = geonet.Batch(specs)
    b.gn_batch_step(1500)
    b.gn_batch_step(500)
    info = b.gn_batch_get_info()
    assert info["n_nets"] == 24 and info["step"] == 2000 and info["cta_threads"] in (128, 256, 512)
    assert info["step_kernel"] == {1: 1, 3: 3, 4: 3, 5: 5}[batch_kernel]
    assert (info["step_groups"] > 1) == (batch_kernel >= 4), info
    assert info["step_lanes"] == (2 if batch_kernel >= 4 else 1 if batch_kernel == 3 else 0), info
    n_blocks = [b.gn_batch_get_net_info(i)["n_blocks"] for i in range(24)]
    assert min(n_blocks) >= 1
    if batch_kernel in (3, 4):  # the staged grid is every member's tiles
        assert sum(n_blocks) == info["grid"], (n_blocks, info)
    for i in range(0, 24, 3):
        net = geonet.Net(specs[i], step_kernel=1)
        net.gn_step(2000)
        sa, sb = net.gn_get_state(), b.gn_batch_get_state(i)
        for k in ("v", "w", "c", "bg_count"):
            assert np.array_equal(sa[k], sb[k]), (i, k)
        assert np.array_equal(net.gn_get_arrivals(), b.gn_batch_get_arrivals(i))
        ya, _, _ = net.gn_observe()
        yb, first, _ = b.gn_batch_observe(i)
        assert first == 0 and np.array_equal(ya, yb)
        na, sa_, _ = net.gn_get_events()
        nb, sb_, _ = b.gn_batch_get_events(i)
        assert np.array_equal(na, nb) and np.array_equal(sa_, sb_)


def test_batch_delays_and_arrivals_match_the_oracle():
    from paper_0908_3934_b300 import geonet
    specs = _specs(16, seed0=5000)
    b = geonet.Batch(specs)
    b.gn_batch_step(1200)
    for i, sp in enumerate(specs):
        assert np.array_equal(b.gn_batch_get_delays(i), oracle.net_delays(sp))
        ref = oracle.simulate(sp, 1200, want_y=False)
        ok = (ref["first_arrival"] >= 0) & (np.abs(ref["first_value"]) >= 2.0 ** -126)
        assert np.array_equal(b.gn_batch_get_arrivals(i)[ok], ref["first_arrival"][ok]), i


def test_batch_windows_against_the_oracle():
    """Sampled members, 1 ms windows over the first 40 ms: the oracle's own FP64
    trajectory is loaded into those members (data flows oracle -> GPU only) and
    the batch's next 20 steps are compared within 1e-4 relative / 1e-6 absolute."""
    from paper_0908_3934_b300 import geonet
    specs = _specs(12, seed0=7000)
    b = geonet.Batch(specs)
    sample = [0, 5, 11]
    K, steps = 20, 800
    refs = {}
    depth = {}
    for i in sample:
        D = oracle.net_delays(specs[i])
        depth[i] = int(D.max()) + 1
        refs[i] = oracle.simulate(specs[i], 0, hist_depth=depth[i], want_y=False)
    worst = 0.0
    for n0 in range(0, steps, K):
        b.gn_batch_set_step(n0)
        nxt = {}
        for i in sample:
            r = refs[i]
            b.gn_batch_set_state(i, r["hist"].astype(np.float32), r["w"].astype(np.float32),
                                 r["c"].astype(np.float32), r["bg_count"])
            nxt[i] = oracle.simulate(specs[i], K, hist_depth=depth[i],
                                     init=dict(n0=n0, v=r["v"], w=r["w"], c=r["c"], bg_count=r["bg_count"],
                                               hist=r["hist"]))
        b.gn_batch_step(K)
        for i in sample:
            g = b.gn_batch_get_state(i)
            for k in ("v", "w", "c"):
                worst = max(worst, ratio(g[k], nxt[i][k]))
            y, _, _ = b.gn_batch_observe(i)
            worst = max(worst, ratio(y, nxt[i]["y"]))
            refs[i] = nxt[i]
    assert worst <= 1.0, worst


def test_batch_of_one_and_empty_networks():
    from paper_0908_3934_b300 import geonet
    lone = netgen.NetSpec(pos=np.zeros((3, 2)), src=np.zeros(0, np.int32), dst=np.zeros(0, np.int32),
                          weight=np.zeros(0, np.float32), speed=None, speed_scalar=1.0,
                          pulses=[(1, 1.0, 3.0, 1.0)])
    b = geonet.Batch([lone, netgen.tiny(), lone])
    b.gn_batch_step(400)
    ref = oracle.simulate(lone, 400)
    for i in (0, 2):
        g = b.gn_batch_get_state(i)
        assert ratio(g["v"], ref["v"]) <= 1.0 and not g["v"][[0, 2]].any()
    ref_t = oracle.simulate(netgen.tiny(), 400)
    ok = ref_t["first_arrival"] >= 0
    assert np.array_equal(b.gn_batch_get_arrivals(1)[ok], ref_t["first_arrival"][ok])
