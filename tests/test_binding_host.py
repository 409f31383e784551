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
