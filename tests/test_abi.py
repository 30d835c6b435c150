"""The C ABI without a GPU: the library loads, exports every entry point that
include/fcs.h declares, its structs have the documented layout, and host-side
argument validation rejects bad input before any device work."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2103_14737_gb300 import fcs, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fcs.h")


def header_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fcs_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    return fcs.load_library()


def test_exports_every_declared_symbol(lib):
    names = header_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(fcs.EXPORTED) == names


def test_struct_layouts():
    assert synth.REGION_DTYPE.itemsize == 48 and synth.LAYER_DTYPE.itemsize == 16
    assert C.sizeof(fcs.fcs_particles) == 40
    assert C.sizeof(fcs.fcs_config) == 40
    assert C.sizeof(fcs.fcs_stats) == 40
    assert C.sizeof(fcs.fcs_debug) == 72


def test_version_and_error_text(lib):
    assert "libfcs" in fcs.fcs_version()
    rc = lib.fcs_load_geometry(None, None, 0, None, 0, None, None)
    assert rc == fcs.FCS_E_ARG
    buf = C.create_string_buffer(256)
    assert lib.fcs_last_error(buf, 256) == fcs.FCS_E_ARG and buf.value


def _geo_call(lib, regions, lrb, layers):
    out = C.c_void_p()
    reg = np.ascontiguousarray(regions)
    l = np.ascontiguousarray(lrb, dtype=np.int32)
    lay = np.ascontiguousarray(layers)
    return lib.fcs_load_geometry(C.byref(out), reg.ctypes.data_as(C.c_void_p), len(reg),
                                 l.ctypes.data_as(C.c_void_p), len(l) - 1, lay.ctypes.data_as(C.c_void_p), None)


def test_geometry_validation_rejects_bad_tables(lib, geo):
    bad = geo.regions.copy()
    bad[5]["deta"] = -0.1
    assert _geo_call(lib, bad, geo.layer_region_begin, geo.layers) == fcs.FCS_E_ARG
    bad = geo.regions.copy()
    bad[3]["cell_offset"] += 1
    assert _geo_call(lib, bad, geo.layer_region_begin, geo.layers) == fcs.FCS_E_ARG
    bad = geo.regions.copy()
    bad[1]["eta_lo"] = bad[0]["eta_lo"]  # overlaps its predecessor
    assert _geo_call(lib, bad, geo.layer_region_begin, geo.layers) == fcs.FCS_E_ARG
    lrb = geo.layer_region_begin.copy()
    lrb[-1] -= 1
    assert _geo_call(lib, geo.regions, lrb, geo.layers) == fcs.FCS_E_ARG
    lay = geo.layers.copy()
    lay[2]["rz"] = 0.0
    assert _geo_call(lib, geo.regions, geo.layer_region_begin, lay) == fcs.FCS_E_ARG


def test_params_and_simulate_validation(lib):
    out = C.c_void_p()
    z = np.zeros(4, np.float32)
    # NULL geometry -> FCS_E_ARG before any device work
    assert lib.fcs_load_params(C.byref(out), None, z.ctypes.data, z.ctypes.data, z.ctypes.data, z.ctypes.data,
                               z.ctypes.data, 1, 1, 1, 16, 8, 20.0, 6, None) == fcs.FCS_E_ARG
    cfg = fcs.make_config()
    st = fcs.fcs_stats()
    parts = fcs.fcs_particles()
    assert lib.fcs_simulate_events(None, None, None, C.byref(parts), 0, 1, 1, 0, C.byref(cfg), None, None, None,
                                   None, 0, C.byref(st), None, None) == fcs.FCS_E_ARG
    assert lib.fcs_simulate_backward(None, None, None, None, 0, 0, 0, 0, None, None, None, None,
                                     None, None) == fcs.FCS_E_ARG
    assert lib.fcs_update_params(None, None, None, None, None) == fcs.FCS_E_ARG
    assert lib.fcs_selftest_wait_timeout(None, None) == fcs.FCS_E_ARG
    assert lib.fcs_workspace_reserve(None, None, 0, 1, 0, 0) == fcs.FCS_E_ARG
