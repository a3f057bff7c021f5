"""The C-ABI library loads and exports every entry point that include/terra_wedge.h declares (CPU only)."""
import ctypes
import os

import pytest

import paper_2609_21633_gb300 as tn
from paper_2609_21633_gb300 import build as tnbuild


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(tn._lib.LIB_PATH):
        tnbuild.build()
    return tn.lib()


def test_exports_every_declared_entry_point(lib):
    names = tn._lib.header_entry_points()
    assert len(names) >= 17
    for name in names:
        assert hasattr(lib, name), name
        assert name in tn._lib._SIGS, name


def test_invalid_arguments_fail_before_any_device_work(lib):
    out = ctypes.c_void_p()
    assert lib.tn_mesh_create(0, 5, 0.55, 1.0, None, ctypes.byref(out)) == tn.TN_EINVAL
    assert b"lateral_level" in lib.tn_last_error()
    assert lib.tn_mesh_create(3, 4, 0.55, 1.0, None, ctypes.byref(out)) == tn.TN_EINVAL
    assert lib.tn_mesh_create(3, 5, 1.0, 0.55, None, ctypes.byref(out)) == tn.TN_EINVAL
    for quad, kappa in ((3, 0.0), (-1, 0.0), (2, 0.3)):  # radial points 1 or 2, not with hourglass control
        o = tn._lib.tn_mesh_opts(0, 0, 1, 0, 0, kappa, quad)
        assert lib.tn_mesh_create(3, 5, 0.55, 1.0, ctypes.byref(o), ctypes.byref(out)) == tn.TN_EINVAL
        assert b"radial" in lib.tn_last_error()
    assert lib.tn_operator_steps_host(None, 0, 1, None, None, None, None) == tn.TN_EINVAL
    so = tn._lib.tn_server_opts(4, 0.8, 1, 1e-8, 0, 0, 0.3, 2)  # the server checks the same pair
    srv = ctypes.c_void_p()
    assert lib.tn_server_create(ctypes.byref(so), ctypes.byref(srv)) == tn.TN_EINVAL
    assert lib.tn_mesh_info(None, 0, None) == tn.TN_EINVAL
    assert lib.tn_mesh_destroy(None) == tn.TN_OK
