"""Heterogeneous cells (Sec. 3.1: cell types as parameter sets of one transition
function) on the GPU against the FP64 oracle: each node reads its set's parameters;
windows as for the homogeneous spiking models (tests/parity.py)."""
import numpy as np
import pytest

from paper_0908_3934_b300 import geonet, netgen

from parity import assert_windows, windowed_izh

pytestmark = pytest.mark.gpu


def test_one_set_is_bit_identical_to_the_homogeneous_net():
    base = netgen.izhikevich(netgen.roofline(seed=21, n=20000, bg_rate_hz=100.0))
    one = netgen.dataclasses.replace(base, cell_types=[dict(base.izh)], cell_type=np.zeros(base.n_nodes, np.uint8))
    a, b = geonet.Net(base), geonet.Net(one)
    a.gn_step(500)
    b.gn_step(500)
    for x, y in ((a.gn_get_state(), b.gn_get_state()), (a.gn_get_izh_state(), b.gn_get_izh_state())):
        for k in x:
            assert np.array_equal(x[k], y[k]), k


@pytest.mark.parametrize("model", ["izh", "hh"])
def test_mixed_tiny_net_windows(model):
    if model == "izh":
        spec = netgen.mixed_cells(netgen.izhikevich(netgen.tiny(), w_scale=7000.0), seed=3)
        n = 4000
    else:
        base = netgen.hodgkin_huxley(netgen.tiny(), w_scale=10.0)
        spec = netgen.mixed_cells(base, types=[dict(netgen.HH_CLASSIC), dict(netgen.HH_CLASSIC, gk=24.0, i_ext=2.0)],
                                  frac=(0.5, 0.5), inhibitory=(False, False), seed=3)
        n = 2000
    net = geonet.Net(spec)
    worst, n_spikes, excused = windowed_izh(spec, net, n)
    print("worst ratios", worst, "excused", excused)
    assert_windows(worst)
    assert n_spikes > 50


@pytest.mark.parametrize("step_kernel", [1, 3])
def test_mixed_multi_block_net_windows(step_kernel):
    spec = netgen.mixed_cells(netgen.izhikevich(netgen.large(n=30000, mean_deg=40, bg_rate_hz=100.0)), seed=5)
    net = geonet.Net(spec, step_kernel=step_kernel)
    worst, n_spikes, _ = windowed_izh(spec, net, 200, start=100)
    assert_windows(worst)
    assert n_spikes > 0


def test_every_kernel_and_shape_gives_the_same_bits(monkeypatch):
    spec = netgen.mixed_cells(netgen.izhikevich(netgen.roofline(seed=21, n=20000, bg_rate_hz=100.0)), seed=7)
    ref = None
    for kind, shape in [(1, s) for s in range(5)] + [(2, 0)] + [(3, s) for s in range(8)]:
        monkeypatch.setenv("GN_STEP_SHAPE", str(shape))
        net = geonet.Net(spec, step_kernel=kind)
        net.gn_step(600)
        st, iz = net.gn_get_state(), net.gn_get_izh_state()
        cur = [st["w"], st["c"], iz["V"], iz["r"], iz["p"], net.gn_get_history(8)]
        if ref is None:
            ref = cur
            continue
        for a, b in zip(cur, ref):
            assert np.array_equal(a, b), (kind, shape)


def test_mixed_batch_members_equal_single_nets():
    specs = [netgen.mixed_cells(netgen.test_set_izh(netgen.test_set_net(n, 2, "random", "high", seed=i)), seed=i)
             for i, n in enumerate((30, 100, 300))]
    specs.append(netgen.test_set_izh(netgen.test_set_net(100, 2, "lattice", "high", seed=9)))  # homogeneous member
    b = geonet.Batch(specs)
    b.gn_batch_step(500)
    for i, sp in enumerate(specs):
        net = geonet.Net(sp)
        net.gn_step(500)
        iz, biz = net.gn_get_izh_state(), b.gn_batch_get_izh_state(i)
        for k in ("V", "r", "p"):
            assert np.array_equal(iz[k], biz[k]), (i, k)
        assert np.array_equal(net.gn_get_state()["w"], b.gn_batch_get_state(i)["w"])


def test_cell_types_are_checked():
    spec = netgen.izhikevich(netgen.tiny())
    bad = netgen.dataclasses.replace(spec, cell_types=[dict(spec.izh)], cell_type=np.ones(64, np.uint8))
    with pytest.raises(geonet.GeonetError) as e:
        geonet.Net(bad)
    assert e.value.status == geonet.GN_EINVAL
    fhn = netgen.dataclasses.replace(netgen.tiny(), cell_types=[dict(spec.izh)], cell_type=np.zeros(64, np.uint8))
    with pytest.raises(geonet.GeonetError) as e:
        geonet.Net(fhn)
    assert e.value.status == geonet.GN_EINVAL
