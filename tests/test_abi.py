"""The C-ABI library builds, loads and exports every entry point the public
header declares; argument checks run without a GPU."""
import ctypes
import os
import re

import pytest

import paper_2101_05888_gb300 as sas
from paper_2101_05888_gb300 import build as sas_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sas.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sas_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libsas():
    sas_build.build()
    return sas.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("sas_geometry_create", "sas_echo_upload", "sas_backproject_2d", "sas_backproject_3d",
              "sas_backproject_adjoint"):
        assert n in names


def test_every_declared_symbol_is_exported(libsas):
    for name in declared_functions():
        assert hasattr(libsas, name), name
        assert isinstance(getattr(libsas, name), ctypes._CFuncPtr)


def test_python_binding_covers_the_header():
    assert sorted(sas.ENTRY_POINTS) == declared_functions()
    for name in declared_functions():
        assert callable(getattr(sas, name))


def test_version_and_error_string(libsas):
    assert sas.sas_version() == 10000
    assert isinstance(sas.sas_last_error(), str)


def test_argument_errors_without_gpu(libsas):
    h = ctypes.c_void_p()
    assert libsas.sas_geometry_create(None, None, None, ctypes.byref(h)) == sas.SAS_ERR_ARG
    assert "null" in sas.sas_last_error()
    nav = sas.sas_nav(0, 1, 1, 1, 1, 1)
    sig = sas.make_signal(1e5, 4e4, 1500.0, 0.0, 1024)
    assert libsas.sas_geometry_create(ctypes.byref(nav), ctypes.byref(sig), None, ctypes.byref(h)) == sas.SAS_ERR_ARG
    assert libsas.sas_backproject_2d(None, None, None, None, 0, None) == sas.SAS_ERR_ARG
    assert libsas.sas_sharpness(None, 0, None, None, None) == sas.SAS_ERR_ARG
    assert libsas.sas_debug_starve_copies(None, 1, 10) == sas.SAS_ERR_ARG
    for rows in (7, 24, 1024, -8):
        assert libsas.sas_debug_dpc_solve_chunk(rows) == sas.SAS_ERR_ARG
    assert libsas.sas_debug_dpc_solve_chunk(16) == sas.SAS_OK
    assert libsas.sas_debug_dpc_solve_chunk(0) == sas.SAS_OK


def test_conditioning_and_dpc_argument_errors_without_gpu(libsas):
    """The host-side checks of the conditioning and micronavigation calls
    refuse bad sizes before any CUDA call (the placeholder pointers are never
    used)."""
    fake = ctypes.c_void_p(0x1000)
    assert libsas.sas_matched_filter(fake, 4, 100, fake, 0, fake, None) == sas.SAS_ERR_ARG       # L < 1
    assert libsas.sas_matched_filter(fake, 4, 100, fake, 4097, fake, None) == sas.SAS_ERR_ARG    # L > 4096
    assert libsas.sas_matched_filter(fake, 0, 100, fake, 8, fake, None) == sas.SAS_OK            # no rows
    assert libsas.sas_whiten(fake, fake, 4, 300, 0.1, None, None) == sas.SAS_ERR_ARG             # n not 2^k
    assert libsas.sas_whiten(fake, fake, 4, 32768, 0.1, None, None) == sas.SAS_ERR_ARG           # n > 16384
    assert libsas.sas_whiten(fake, fake, 4, 256, -1.0, None, None) == sas.SAS_ERR_ARG            # gamma < 0
    assert libsas.sas_tvg(fake, fake, 0, 16, 0.1, None, None, None) == sas.SAS_ERR_ARG           # no rows
    assert libsas.sas_tvg(fake, fake, 4, 16, -0.5, None, None, None) == sas.SAS_ERR_ARG          # alpha < 0
    assert libsas.sas_drc(fake, 100, 1.0, fake, None, None) == sas.SAS_ERR_ARG                  # b = 1
    assert libsas.sas_drc(fake, 0, 0.3, fake, None, None) == sas.SAS_ERR_ARG                    # no pixels
    assert libsas.sas_dpc_delays(None, 2, fake, 10, 128, 8, None, None, None, None) == sas.SAS_ERR_ARG
    assert libsas.sas_dpc_footprints(None, fake, fake, fake, None) == sas.SAS_ERR_ARG
    pr = sas.sas_dpc_problem(P=1, C=8, shift=2, K=4, side=1, c=1500.0)                          # P < 2
    assert libsas.sas_dpc_solve(ctypes.byref(pr), fake, fake, 10, None, None, None) == sas.SAS_ERR_ARG


def test_build_flags_and_interp_form_degree_without_gpu(libsas):
    """The plain library reports no checked build (the checked one, built with
    -DSAS_CHECKED, reports bit 0); the Farrow-form evaluation refuses a degree
    other than the cubic (3) and the quadratic (2) before touching a device."""
    expect = 1 if os.environ.get("SAS_CHECKED") == "1" else 0
    assert libsas.sas_build_flags() == expect
    it = sas.kaiser(4.0)
    for degree in (0, 1, 4):
        rc = libsas.sas_interp_eval_form(ctypes.byref(it), degree, None, 0, None, None, None)
        assert rc == sas.SAS_ERR_ARG
