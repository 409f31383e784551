"""The C ABI library loads without a GPU, exports every entry point that
include/*.h declares, and rejects invalid descriptors before touching the device."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

from paper_0908_3934_b300 import build, geonet, netgen


@pytest.fixture(scope="module")
def L():
    build.build()
    return geonet.lib()


def test_every_declared_symbol_is_exported(L):
    names = geonet.exported_symbols()
    assert len(names) >= 34
    out = subprocess.run(["nm", "-D", "--defined-only", geonet.LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(L, n)


def test_only_the_abi_is_exported(L):
    out = subprocess.run(["nm", "-D", "--defined-only", geonet.LIB_PATH], capture_output=True, text=True).stdout
    ours = [line.split()[-1] for line in out.splitlines() if " T " in line]
    assert ours and all(n.startswith("gn_") for n in ours), ours


def test_struct_layouts_match_the_header(L, tmp_path):
    """sizeof and offsetof of every ABI struct, from gcc on the header, equal the binding's."""
    structs = {"gn_fhn_params": geonet.gn_fhn_params, "gn_obs_params": geonet.gn_obs_params,
               "gn_izh_params": geonet.gn_izh_params, "gn_hh_params": geonet.gn_hh_params,
               "gn_stdp_params": geonet.gn_stdp_params,
               "gn_net_desc": geonet.gn_net_desc, "gn_pulse": geonet.gn_pulse, "gn_net_info": geonet.gn_net_info,
               "gn_batch_info": geonet.gn_batch_info}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "geonet.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.check_call(["gcc", "-I", inc, str(src), "-o", str(exe)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == C.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(cls, f).offset, f"{name}.{f}"


def _desc(spec, **over):
    keep = dict(pos=np.ascontiguousarray(spec.pos, np.float64), src=np.ascontiguousarray(spec.src, np.int32),
                dst=np.ascontiguousarray(spec.dst, np.int32), w=np.ascontiguousarray(spec.weight, np.float32))
    f = spec.fhn
    d = geonet.gn_net_desc(
        n_nodes=spec.n_nodes, dim=spec.dim, pos=keep["pos"].ctypes.data, n_edges=spec.n_edges,
        src=keep["src"].ctypes.data, dst=keep["dst"].ctypes.data, weight=keep["w"].ctypes.data, speed=None,
        speed_scalar=spec.speed_scalar, dt_ms=0.05,
        fhn=geonet.gn_fhn_params(**{k: f[k] for k in ("a", "b", "c", "e", "f", "g", "i_ext")}),
        obs=geonet.gn_obs_params(tau_ms=5.0, sample_every=20, gain=1.0, offset=0.0, sigma=0.05, seed=1))
    for k, v in over.items():
        setattr(d, k, v)
    return d, keep


def _create(L, d):
    h = C.c_void_p()
    st = L.gn_net_create(C.byref(d), C.byref(h))
    return st, h


@pytest.mark.parametrize("bad", ["selfloop", "range", "nan", "speed", "dt", "rest", "ring", "dim", "format"])
def test_invalid_descriptors_are_rejected(L, bad):
    spec = netgen.tiny()
    if bad == "selfloop":
        spec.dst = spec.dst.copy()
        spec.dst[3] = spec.src[3]
    if bad == "range":
        spec.src = spec.src.copy()
        spec.src[0] = spec.n_nodes
    if bad == "nan":
        spec.pos = spec.pos.copy()
        spec.pos[5, 1] = np.nan
    over = {}
    if bad == "speed":
        over["speed_scalar"] = 0.0
    if bad == "dt":
        over["dt_ms"] = -1.0
    if bad == "ring":
        over["ring_depth"] = 48
    if bad == "dim":
        over["dim"] = 4
    if bad == "format":
        over["edge_format"] = 7
    d, keep = _desc(spec, **over)
    if bad == "rest":
        d.fhn.a = 2.0  # a > c/g: no unique rest point
    st, h = _create(L, d)
    assert st == geonet.GN_EINVAL
    assert not h.value
    assert L.gn_last_error().decode()


def test_null_handles(L):
    assert L.gn_net_destroy(None) == geonet.GN_OK
    assert L.gn_step(None, 1) == geonet.GN_EINVAL
    assert L.gn_net_create(None, None) == geonet.GN_EINVAL
