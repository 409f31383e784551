"""The persistent lanes schedule of the batched form (GN_BATCH_KERNEL=5): one
cooperative launch per 64-step chunk in which lanes of CTAs step L2-sized member
groups, meeting at counting barriers in global memory, against the chain of
per-step launches (kernel 3) over the same members.

Every member's states, history, arrivals, observations and events must be the
same bits: the kernels share the tile step, and the lanes' barriers must order
each step's node updates after the previous step and its gathers after the one
before (the tightest case: a 4-slot ring and delays of 1 or 2 steps, where slot
n + 1, written in step n, is the one step n - 3 read)."""
import numpy as np
import pytest
import torch

from paper_0908_3934_b300 import geonet, netgen

pytestmark = pytest.mark.gpu


def _fast_members(n, seed0=3000, n_hi=2000):
    """Batch members with delays of 1 or 2 steps in a 4-slot ring and 200 Hz
    background pulses (the nets keep firing)."""
    out = []
    rng = np.random.default_rng(seed0)
    for i in range(n):
        sp = netgen.batch_member(seed0 + i, n_hi=n_hi)
        sp.delay = rng.integers(1, 3, sp.n_edges).astype(np.int32)
        sp.ring_depth = 4
        sp.background = dict(rate_hz=200.0, amp=1.0, dur_ms=2.0, seed=seed0 + 7 * i)
        out.append(sp)
    return out


def _run(specs, monkeypatch, kernel, group_kb, lanes, chunks):
    monkeypatch.setenv("GN_BATCH_KERNEL", kernel)
    monkeypatch.setenv("GN_BATCH_GROUP_KB", group_kb)
    monkeypatch.setenv("GN_BATCH_LANES", lanes)
    b = geonet.Batch(specs)
    for c in chunks:
        b.gn_batch_step(c)
    info = b.gn_batch_get_info()
    out = []
    for i in range(len(specs)):
        y, first, _ = b.gn_batch_observe(i)
        ev = b.gn_batch_get_events(i)
        out.append(dict(state=b.gn_batch_get_state(i), hist=b.gn_batch_get_history(i, 3),
                        arr=b.gn_batch_get_arrivals(i), y=y, first=first, ev=(ev[0], ev[1])))
    b.gn_batch_destroy()
    return info, out


def _same(ref, got, what):
    for i, (a, b) in enumerate(zip(ref, got)):
        for k in ("v", "w", "c", "bg_count"):
            assert np.array_equal(a["state"][k], b["state"][k]), (what, i, k)
        assert np.array_equal(a["hist"], b["hist"]), (what, i)
        assert np.array_equal(a["arr"], b["arr"]), (what, i)
        assert a["first"] == b["first"] and np.array_equal(a["y"], b["y"]), (what, i)
        assert np.array_equal(a["ev"][0], b["ev"][0]) and np.array_equal(a["ev"][1], b["ev"][1]), (what, i)


def test_lanes_equal_the_launch_chain_at_the_fastest_slot_reuse(monkeypatch):
    """40 members, 3000 steps (46 chunks and a ragged tail of 56): the lanes schedule
    in 1, 2, 3 and 8 lanes with groups of one to a few members (an 8-lane launch
    with fewer groups than lanes in some chunks' lanes), bit-identical to every
    member every step in a chain of launches."""
    specs = _fast_members(40)
    chunks = [1000, 1944, 56]
    info, ref = _run(specs, monkeypatch, "3", "0", "1", chunks)
    assert info["step_kernel"] == 3 and info["step_groups"] == 1
    assert max(np.abs(r["state"]["v"]).max() for r in ref) > 0.1
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for group_kb, lanes in (("0", "1"), ("256", "1"), ("256", "2"), ("128", "3"), ("64", "8")):
        info, got = _run(specs, monkeypatch, "5", group_kb, lanes, chunks)
        assert info["step_kernel"] == 5 and info["grid"] % sms == 0, info
        assert (info["step_groups"] > 1) == (group_kb != "0"), info
        _same(ref, got, (group_kb, lanes))


def test_lanes_with_several_tiles_per_cta(monkeypatch):
    """700 members in one group: more tiles than the cooperative grid, so each CTA
    steps several tiles of different members per step (its step arguments change
    between them, and its mbarrier phase runs on); 300 steps bit-identical to the
    chain of launches."""
    specs = [netgen.batch_member(1000 + i) for i in range(700)]
    info, ref = _run(specs, monkeypatch, "3", "0", "1", [300])
    sel = list(range(0, 700, 23))
    for group_kb, lanes in (("0", "1"), ("24576", "4")):
        info5, got = _run(specs, monkeypatch, "5", group_kb, lanes, [300])
        assert info5["step_kernel"] == 5
        if group_kb == "0":
            assert info["grid"] > info5["grid"], (info, info5)  # tiles against the cooperative CTAs
        _same([ref[i] for i in sel], [got[i] for i in sel], (group_kb, lanes))


def test_a_lane_wait_that_gives_up_reports_a_timeout(monkeypatch):
    """With the poll budget set to zero every bounded wait of the lanes kernel gives
    up at once (the copy waits, and the barrier waits of CTAs that reach one): the
    CTAs record kStatusTimeout and return, the host reports GN_ETIMEOUT at the next
    synchronising call, and the context stays usable."""
    specs = _fast_members(12)
    monkeypatch.setenv("GN_BATCH_KERNEL", "5")
    monkeypatch.setenv("GN_BATCH_GROUP_KB", "256")
    monkeypatch.setenv("GN_BATCH_LANES", "2")
    monkeypatch.setenv("GN_TEST_WAIT_LIMIT", "0")
    b = geonet.Batch(specs)
    b.gn_batch_step(64)
    with pytest.raises(geonet.GeonetError) as e:
        b.gn_batch_synchronize()
    assert e.value.status == geonet.GN_ETIMEOUT
    b.gn_batch_destroy()
    monkeypatch.delenv("GN_TEST_WAIT_LIMIT")
    info, got = _run(specs, monkeypatch, "5", "256", "2", [200])
    info, ref = _run(specs, monkeypatch, "3", "0", "1", [200])
    _same(ref, got, "after a timeout")
