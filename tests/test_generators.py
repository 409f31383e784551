"""Host logic of the seeded input generators that convert a network to the
spiking models and mix cell types (no GPU)."""
import numpy as np
import pytest

import oracle
from paper_0908_3934_b300 import netgen


def test_hodgkin_huxley_conversion_requantises_the_delays():
    base = netgen.large(n=5000, mean_deg=20, bg_rate_hz=5.0)
    hh = netgen.hodgkin_huxley(base)
    assert hh.model == "hh" and hh.dt_ms == 0.03 and hh.ring_depth == 0
    assert hh.obs["sample_every"] == 33
    assert np.allclose(hh.weight, np.asarray(base.weight) * 3.0)
    d_base, d_hh = oracle.net_delays(base), oracle.net_delays(hh)
    # the same geometric delays in shorter steps: D_hh = round(D_ms / 0.03) within rounding
    assert np.all(np.abs(d_hh * 0.03 - d_base * base.dt_ms) <= 0.5 * 0.03 + 0.5 * base.dt_ms + 1e-12)
    assert d_hh.max() > d_base.max()
    assert all(amp == 20.0 for (_, _, _, amp) in hh.pulses) and hh.background["amp"] == 20.0


def test_mixed_cells_draws_sets_and_signs_out_weights_by_source():
    base = netgen.izhikevich(netgen.large(n=20000, mean_deg=20, bg_rate_hz=5.0))
    mixed = netgen.mixed_cells(base, seed=4)
    cell = mixed.cell_type
    assert cell.dtype == np.uint8 and set(np.unique(cell)) == {0, 1}
    assert abs(cell.mean() - 0.2) < 0.02
    src = np.asarray(mixed.src)
    w = np.asarray(mixed.weight)
    assert np.all(w[cell[src] == 1] <= 0) and np.all(w[cell[src] == 0] >= 0)
    assert np.array_equal(np.abs(w), np.abs(np.asarray(base.weight, np.float32)))
    assert mixed.cell_types[1]["C"] == netgen.IZH_FS["C"]
    again = netgen.mixed_cells(base, seed=4)
    assert np.array_equal(again.cell_type, cell)
    with pytest.raises(ValueError):
        netgen.mixed_cells(netgen.tiny())


def test_test_set_hh_adds_background_at_the_hh_step():
    net = netgen.test_set_net(100, 2, "lattice", "low", seed=1)
    hh = netgen.test_set_hh(net)
    assert hh.model == "hh" and hh.background["rate_hz"] == 20.0 and hh.dt_ms == 0.03
    assert np.allclose(hh.weight, np.asarray(net.weight) * 2.0)
