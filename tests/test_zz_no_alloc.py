"""gn_batch_step_static: stepping a batch without allocating any memory.

Some callers cannot allocate device memory while they step the simulation (a
real-time loop that must not take the allocator's latency or locks, a program
whose device memory comes from a fixed arena owned by someone else).  For them
the library steps a batch with its per-launch work queue in a fixed device array
inside the library.  Both entry points run the same persistent kernel with the
same summation order, so their results are compared bit for bit.  This file is
collected last so that a run stopping at the first failure has already run every
other test."""
import ctypes as C

import numpy as np
import pytest

from paper_0908_3934_b300 import geonet, netgen

pytestmark = pytest.mark.gpu


def _same_members(a, b, n):
    for i in range(n):
        sa, sb = a.gn_batch_get_state(i), b.gn_batch_get_state(i)
        for k in ("v", "w", "c", "bg_count"):
            assert np.array_equal(sa[k], sb[k]), (i, k)
        ya, fa, _ = a.gn_batch_observe(i)
        yb, fb, _ = b.gn_batch_observe(i)
        assert fa == fb and np.array_equal(ya, yb), i
        assert np.array_equal(a.gn_batch_get_arrivals(i), b.gn_batch_get_arrivals(i)), i


def test_static_step_matches_gn_batch_step_on_two_calls(monkeypatch):
    # the persistent kernel for gn_batch_step too, so both calls run the same code
    monkeypatch.setenv("GN_BATCH_KERNEL", "1")
    specs = [netgen.batch_member(9000 + i, n_hi=1200) for i in range(10)]
    a = geonet.Batch(specs)
    b = geonet.Batch(specs)
    L = geonet.lib()
    for call in range(2):
        geonet.check(L.gn_batch_step_static(a.h, C.c_int64(300)))
        b.gn_batch_step(300)
        assert a.gn_batch_get_info()["step"] == b.gn_batch_get_info()["step"] == 300 * (call + 1)
        _same_members(a, b, len(specs))


def test_static_step_allocates_nothing():
    """After a first call (which may load the kernel's module), further calls leave
    the device's free memory unchanged."""
    import torch
    specs = [netgen.batch_member(9200 + i, n_hi=1200) for i in range(8)]
    a = geonet.Batch(specs)
    L = geonet.lib()
    geonet.check(L.gn_batch_step_static(a.h, C.c_int64(50)))
    a.gn_batch_synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        geonet.check(L.gn_batch_step_static(a.h, C.c_int64(100)))
    a.gn_batch_synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert a.gn_batch_get_info()["step"] == 550


def test_static_step_after_the_staged_form_and_a_new_background(monkeypatch):
    """gn_batch_step_static runs the persistent kernel on the block descriptors of
    its first CTA size even when gn_batch_step chose the staged form and a member's
    background changed afterwards (the argument upload keeps valid descriptors);
    the staged form sums in the same order, so the two agree bit for bit."""
    monkeypatch.setenv("GN_BATCH_KERNEL", "3")
    specs = [netgen.batch_member(9100 + i, n_hi=1200) for i in range(6)]
    a = geonet.Batch(specs)
    b = geonet.Batch(specs)
    L = geonet.lib()
    for x in (a, b):
        x.gn_batch_step(100)
        assert x.gn_batch_get_info()["step_kernel"] == 3
        geonet.check(L.gn_batch_set_background(x.h, 2, C.c_double(40.0), C.c_float(0.5), C.c_double(1.0),
                                               C.c_uint64(77)))
    geonet.check(L.gn_batch_step_static(a.h, C.c_int64(200)))
    b.gn_batch_step(200)
    _same_members(a, b, len(specs))
