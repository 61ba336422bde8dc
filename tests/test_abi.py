"""The C ABI library loads and exports what include/ssvp.h declares; host-side argument checks.

No test here launches GPU work: these run on machines without a GPU.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ssvp.h")


@pytest.fixture(scope="module")
def ss():
    import __graft_entry__ as g
    g._load_builder().build()
    import paper_2102_03011_gb300 as ss
    return ss


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ssvp_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("ssvp_create", "ssvp_destroy", "ssvp_load_clip", "ssvp_set_cameras", "ssvp_gather_filter",
              "ssvp_read_output", "ssvp_read_stats", "ssvp_sync", "ssvp_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(ss):
    lib = ctypes.CDLL(ss.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_params_struct_matches_header(ss):
    # the binding's structure and the C structure must agree in size: ssvp_params_default writes
    # exactly sizeof(ssvp_params) bytes
    buf = (ctypes.c_char * (ctypes.sizeof(ss.ssvp_params) + 64))()
    ctypes.memset(buf, 0x5A, len(buf))
    ss.lib.ssvp_params_default(ctypes.cast(buf, ctypes.POINTER(ss.ssvp_params)))
    assert bytes(buf[ctypes.sizeof(ss.ssvp_params):]) == b"\x5a" * 64
    p = ss.ssvp_params_default()
    assert p.mode == ss.SSVP_MODE_DENOISE and p.k == 7 and p.half_window == 15
    assert p.radius == pytest.approx(-0.005)
    assert p.sigma_rgb == pytest.approx(40 / 255) and p.sigma_f == 6.0 and p.sigma_xyz == 0.0
    assert p.frame_end == -1 and p.crop_w == 0 and p.membership_out is None


def test_null_context_is_rejected(ss):
    lib = ss.lib
    assert lib.ssvp_load_clip(None, 0, 4, 4, 1, None, None, 0, 0) == ss.SSVP_EINVAL
    assert lib.ssvp_set_cameras(None, 0, None, 0, None) == ss.SSVP_EINVAL
    p = ss.ssvp_params_default()
    ids = (ctypes.c_int * 1)(0)
    assert lib.ssvp_gather_filter(None, ctypes.byref(p), ids, 1) == ss.SSVP_EINVAL
    assert lib.ssvp_read_output(None, 0, 0, 1, None, 0) == ss.SSVP_EINVAL
    assert lib.ssvp_sync(None) == ss.SSVP_EINVAL
    assert lib.ssvp_read_stats(None, None, None, None) == ss.SSVP_EINVAL
    assert lib.ssvp_trace_enable(None, 1) == ss.SSVP_EINVAL
    assert lib.ssvp_trace_read(None, 4, None, None, None, None) == ss.SSVP_EINVAL
    assert "NULL" in ss.ssvp_last_error(None)
    lib.ssvp_destroy(None)  # no-op


def test_create_without_device_reports_edevice(ss):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(ss.SsvpError) as e:
        ss.ssvp_create(0, None)
    assert e.value.code == ss.SSVP_EDEVICE


def test_noalloc_median_refuses_host_arrays_before_any_launch(ss):
    """The allocation-free median takes device memory only: host arrays and CPU tensors are
    refused by the binding before the library is called (no GPU needed)."""
    import numpy as np
    import torch
    with pytest.raises(TypeError):
        ss.ssvp_median_depth_noalloc(np.ones(8, np.float32), 8, np.zeros(1, np.float32))
    with pytest.raises(TypeError):
        ss.ssvp_median_depth_noalloc(torch.ones(8), 8, torch.zeros(1))


def test_trace_kinds_have_names(ss):
    """Every trace kind of the header has a distinct short name; unknown kinds give ""."""
    names = [ss.ssvp_trace_kind_name(k) for k in range(ss.SSVP_TRACE_KINDS)]
    assert names == ["gather", "aperture", "frustum", "superres", "extract", "infer", "train", "adam", "batch", "load",
                     "mask"]
    assert ss.ssvp_trace_kind_name(-1) == "" and ss.ssvp_trace_kind_name(ss.SSVP_TRACE_KINDS) == ""
    text = open(HEADER).read()
    assert f"SSVP_TRACE_KINDS = {ss.SSVP_TRACE_KINDS}" in text
