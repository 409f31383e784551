"""The batched form with spiking nodes (Izhikevich, Hodgkin-Huxley): networks of
the standard test set (Sec. 3.5) advanced together by the staged batch kernel give,
member by member, the bit-identical states of the same networks run alone."""
import numpy as np
import pytest

from paper_0908_3934_b300 import geonet, netgen

pytestmark = pytest.mark.gpu


def _members(model):
    nets = [netgen.test_set_net(n, dim, cls, dens, seed=11 + i)
            for i, (n, dim, cls, dens) in enumerate([(10, 2, "lattice", "low"), (30, 3, "small_world", "high"),
                                                    (100, 2, "scale_free", "high"), (300, 3, "random", "low"),
                                                    (1000, 2, "random", "high"), (300, 2, "lattice", "high")])]
    return [netgen.test_set_hh(sp) if model == "hh" else netgen.test_set_izh(sp) for sp in nets]


@pytest.mark.parametrize("schedule", ["timed", "l2_groups", "lanes"])
@pytest.mark.parametrize("model", ["izh", "hh"])
def test_members_equal_their_networks_run_alone(model, schedule, monkeypatch):
    """Each schedule of the staged form: the one the first step times (these
    members fit one group), or L2 blocking in three lanes sharing a 48 KB budget
    (groups of one or two members, each running 64-step chunks) as chains of
    launches or as one persistent launch."""
    if schedule != "timed":
        monkeypatch.setenv("GN_BATCH_KERNEL", "4" if schedule == "l2_groups" else "5")
        monkeypatch.setenv("GN_BATCH_GROUP_KB", "48")
        monkeypatch.setenv("GN_BATCH_LANES", "3")
    specs = _members(model)
    steps = 700 if model == "izh" else 1500
    b = geonet.Batch(specs)
    b.gn_batch_step(steps)
    info = b.gn_batch_get_info()
    assert info["step_kernel"] in ((5,) if schedule == "lanes" else (3,) if schedule == "l2_groups" else (3, 5)), info
    assert (info["step_groups"] > 1) == (schedule != "timed"), info
    n_spikes = 0
    for i, sp in enumerate(specs):
        net = geonet.Net(sp)
        net.gn_step(steps)
        st, bst = net.gn_get_state(), b.gn_batch_get_state(i)
        for k in ("v", "w", "c", "bg_count"):
            assert np.array_equal(st[k], bst[k]), (i, k)
        iz, biz = net.gn_get_izh_state(), b.gn_batch_get_izh_state(i)
        for k in ("V", "r", "p"):
            assert np.array_equal(iz[k], biz[k]), (i, k)
        if model == "hh":
            g, bg = net.gn_get_hh_gates(), b.gn_batch_get_hh_gates(i)
            for k in ("m", "n", "h"):
                assert np.array_equal(g[k], bg[k]), (i, k)
        assert np.array_equal(net.gn_get_history(4), b.gn_batch_get_history(i, 4))
        ev, bev = net.gn_get_events(), b.gn_batch_get_events(i)
        if bev[2] != geonet.GN_EOVERFLOW:  # a member's event buffer holds max(1024, 8 N) events
            assert np.array_equal(ev[0], bev[0]) and np.array_equal(ev[1], bev[1])
            n_spikes += len(ev[0])
        assert np.array_equal(net.gn_get_arrivals(), b.gn_batch_get_arrivals(i))
    assert n_spikes > 100


def test_spiking_batches_are_checked(monkeypatch):
    izh = _members("izh")[:2]
    hh = _members("hh")[:1]
    with pytest.raises(geonet.GeonetError) as e:
        geonet.Batch(izh + hh)
    assert e.value.status == geonet.GN_EINVAL
    plastic = netgen.dataclasses.replace(izh[0], stdp=dict(alpha=1.0, beta=0.1))
    with pytest.raises(geonet.GeonetError) as e:
        geonet.Batch([plastic])
    assert e.value.status == geonet.GN_EINVAL
    b = geonet.Batch(izh)
    with pytest.raises(geonet.GeonetError) as e:
        b.gn_batch_step_static(10)
    assert e.value.status == geonet.GN_EINVAL
    with pytest.raises(geonet.GeonetError) as e:
        b.gn_batch_get_hh_gates(0)
    assert e.value.status == geonet.GN_EINVAL
    monkeypatch.setenv("GN_BATCH_KERNEL", "1")
    with pytest.raises(geonet.GeonetError) as e:
        geonet.Batch(izh).gn_batch_step(10)
    assert e.value.status == geonet.GN_EINVAL


@pytest.mark.parametrize("model", ["fhn", "izh"])
def test_a_batch_larger_than_the_device_launches_first_bit_identically(monkeypatch, model):
    """A staged batch grid with more tiles than the device holds at once lets the
    next step's grid start at once (its gathers read history two or more steps
    old); its members equal those of the same batch waiting first, bit for bit,
    and those of the same batch stepped in L2-blocked groups."""
    specs = [netgen.batch_member(1000 + i) for i in range(700)]
    if model == "izh":
        specs = [netgen.izhikevich(sp) for sp in specs]
    out = []
    # every member every step, launching first or waiting first; then L2 blocking
    # in one lane with groups of about half the tiles (more than the device holds:
    # each group launches first), and in four lanes with groups of a few hundred
    # tiles (fewer: each waits first)
    for kernel, early, group_kb, lanes in (("3", "1", "0", "1"), ("3", "0", "0", "1"), ("4", "1", "131072", "1"),
                                           ("4", "1", "24576", "4"), ("5", "1", "24576", "4")):
        monkeypatch.setenv("GN_BATCH_KERNEL", kernel)
        monkeypatch.setenv("GN_STAGED_EARLY", early)
        monkeypatch.setenv("GN_BATCH_GROUP_KB", group_kb)
        monkeypatch.setenv("GN_BATCH_LANES", lanes)
        b = geonet.Batch(specs)
        b.gn_batch_step(300)
        info = b.gn_batch_get_info()
        assert info["step_kernel"] == (5 if kernel == "5" else 3) and (info["step_groups"] > 1) == (kernel != "3"), info
        out.append([(b.gn_batch_get_state(i), b.gn_batch_get_history(i, 4)) for i in range(0, 700, 37)])
        b.gn_batch_destroy()
    for other in out[1:]:
        for (sa, ha), (sb, hb) in zip(out[0], other):
            for k in ("v", "w", "c", "bg_count"):
                assert np.array_equal(sa[k], sb[k]), k
            assert np.array_equal(ha, hb)
