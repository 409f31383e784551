"""Pins of the oracle's heterogeneous cells (Sec. 3.1: networks of different cell
types as different parameter sets of one transition function): a single set equals
the homogeneous network, every node of an edgeless network equals a lone node of its
own set, and the ring equals the dense history."""
import numpy as np
import pytest

import oracle
from paper_0908_3934_b300 import netgen

RS, FS = netgen.IZH_RS, netgen.IZH_FS


def _lone(izh, n=1, pulses=(), dt=0.05, **kw):
    return netgen.NetSpec(pos=np.zeros((n, 2)), src=np.array([], np.int32), dst=np.array([], np.int32),
                          weight=np.array([], np.float32), speed=None, speed_scalar=1.0, delay=None, dt_ms=dt,
                          pulses=list(pulses), model="izh", izh=dict(izh), obs=dict(netgen.OBS_DEFAULT), **kw)


def test_one_set_is_the_homogeneous_network():
    base = netgen.izhikevich(netgen.tiny(), w_scale=7000.0)
    one = netgen.dataclasses.replace(base, cell_types=[dict(base.izh)],
                                     cell_type=np.zeros(base.n_nodes, np.uint8))
    a = oracle.simulate(base, 3000, ev_cap=100000)
    b = oracle.simulate(one, 3000, ev_cap=100000)
    assert a["ev_count"] > 50
    for k in ("v", "w", "c", "r", "p", "y", "ev_node", "ev_step", "first_arrival"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("model", ["izh", "hh"])
def test_each_node_follows_its_own_set(model):
    """Four unconnected nodes of two sets, each pulsed: node j's trajectory is bit
    for bit that of a lone homogeneous node of its set under the same pulse."""
    if model == "izh":
        sets = [dict(RS), dict(FS)]
        amps = (2500.0, 400.0)
        dt = 0.05
    else:
        sets = [dict(netgen.HH_CLASSIC), dict(netgen.HH_CLASSIC, gk=24.0, i_ext=2.0)]
        amps = (20.0, 20.0)
        dt = 0.03
    cell = np.array([0, 1, 1, 0], np.uint8)
    pulses = [(j, 1.0 + 2 * j, 3.0 + 2 * j, amps[cell[j]]) for j in range(4)]
    spec = _lone(RS, n=4, pulses=pulses, dt=dt, cell_types=sets, cell_type=cell)
    if model == "hh":
        spec = netgen.dataclasses.replace(spec, model="hh", hh=dict(netgen.HH_CLASSIC))
    n = 2000
    r = oracle.simulate(spec, n, snap_every=1, want_y=False, ev_cap=10000)
    assert r["ev_count"] >= 4
    for j in range(4):
        lone = _lone(RS, pulses=[(0, *pulses[j][1:])], dt=dt)
        if model == "hh":
            lone = netgen.dataclasses.replace(lone, model="hh", hh=dict(sets[cell[j]]))
        else:
            lone = netgen.dataclasses.replace(lone, izh=dict(sets[cell[j]]))
        q = oracle.simulate(lone, n, snap_every=1, want_y=False, ev_cap=10000)
        assert np.array_equal(r["snap_v"][:, j], q["snap_v"][:, 0]), j
        assert np.array_equal(r["ev_step"][r["ev_node"] == j], q["ev_step"]), j


def test_mixed_ring_equals_dense_history():
    spec = netgen.mixed_cells(netgen.izhikevich(netgen.tiny(), w_scale=7000.0), seed=3)
    assert 0 < spec.cell_type.sum() < spec.n_nodes
    a = oracle.simulate(spec, 3000, ev_cap=100000)
    b = oracle.simulate(spec, 3000, dense=True, ev_cap=100000)
    for k in ("v", "w", "c", "r", "p", "y", "ev_node", "ev_step"):
        assert np.array_equal(a[k], b[k]), k


def test_cell_types_are_checked():
    base = netgen.izhikevich(netgen.tiny())
    bad = netgen.dataclasses.replace(base, cell_types=[dict(RS)], cell_type=np.ones(base.n_nodes, np.uint8))
    with pytest.raises(ValueError):
        oracle.simulate(bad, 10)
    fhn = netgen.dataclasses.replace(netgen.tiny(), cell_types=[dict(RS)],
                                     cell_type=np.zeros(64, np.uint8))
    with pytest.raises(ValueError):
        oracle.simulate(fhn, 10)
