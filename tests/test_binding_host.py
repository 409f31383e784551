"""Marshalling checks of the Python binding that run before any library call (no
GPU): a caller's output buffer must be a writable C-contiguous float32 array with
room for the rows the library may write."""
import numpy as np
import pytest

from paper_0908_3934_b300 import geonet


def test_output_buffer_checks():
    ok = np.zeros((4, 10), np.float32)
    assert geonet._out_rows(ok, 4, 10) is ok
    assert geonet._out_rows(np.zeros(40, np.float32), 4, 10) is not None  # flat buffers of the right size
    assert geonet._out_rows(ok, 0, 10) is ok
    with pytest.raises(ValueError):
        geonet._out_rows(ok, 5, 10)  # one row short
    with pytest.raises(ValueError):
        geonet._out_rows(np.zeros((4, 10), np.float64), 4, 10)
    with pytest.raises(ValueError):
        geonet._out_rows(np.zeros((10, 4), np.float32).T, 4, 10)  # not C-contiguous
    ro = np.zeros((4, 10), np.float32)
    ro.flags.writeable = False
    with pytest.raises(ValueError):
        geonet._out_rows(ro, 4, 10)
    with pytest.raises(ValueError):
        geonet._out_rows([[0.0] * 10] * 4, 4, 10)


def test_input_length_checks():
    """Inputs the library reads n values from (state vectors, weights) or rows of n
    values from (history) are converted and their lengths checked first."""
    v = geonet._vec([1, 2, 3], np.float32, 3, "w")
    assert v.dtype == np.float32 and v.flags.c_contiguous and v.tolist() == [1.0, 2.0, 3.0]
    assert geonet._vec(None, np.float32, 3, "w") is None
    assert geonet._vec(np.arange(6, dtype=np.int64)[::2], np.int32, 3, "bg_count").tolist() == [0, 2, 4]
    with pytest.raises(ValueError):
        geonet._vec(np.zeros(2), np.float32, 3, "w")
    with pytest.raises(ValueError):
        geonet._vec(np.zeros(4), np.float32, 3, "w")
    h = geonet._rows_in(np.zeros((2, 5)), 5, "hist")
    assert h.dtype == np.float32 and h.shape == (2, 5)
    for bad in (np.zeros(5), np.zeros((2, 4)), np.zeros((0, 5)), np.zeros((1, 2, 5))):
        with pytest.raises(ValueError):
            geonet._rows_in(bad, 5, "hist")


def test_device_tensor_checks_reject_host_tensors_and_arrays():
    """The estimator calls take device tensors only: host tensors and numpy arrays
    are refused before their address could reach the library."""
    import torch
    for bad in (torch.zeros((4, 33), dtype=torch.float32), np.zeros((4, 33), np.float32)):
        with pytest.raises(ValueError):
            geonet._dev(bad, "float32", "X", shape=(None, 33))
