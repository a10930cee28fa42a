"""The C interface loads, exports every entry point include/tkf.h declares, and rejects bad
arguments without touching a GPU (runs on a machine without one)."""

import ctypes
import os
import re

import pytest

import paper_2505_22822_gb300 as tkf

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "tkf.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:tkf_status|void|const char\s*\*)\s*(tkf_\w+)\s*\(", src, flags=re.M)))


def test_library_exports_every_declared_function():
    L = tkf.lib()
    decl = declared_functions()
    assert len(decl) >= 11
    for name in decl:
        assert hasattr(L, name), name
    # the binding knows every declared entry point
    assert set(decl) <= set(tkf.exported_symbols())


def test_option_defaults():
    o = tkf.FitOptions()
    tkf.lib().tkf_fit_options_default(ctypes.byref(o))
    assert (o.precision, o.step_mode, o.tol, o.h_max, o.h_min, o.surf_tol, o.max_steps) == \
        (0, 0, 1e-4, 1000.0, 1e-4, 1e-2, 10000)
    assert abs(o.mass - 0.1056583755) < 1e-12
    assert o.seed_cov_scale == 1.0 and o.kernel_events is None
    assert (o.lanes_per_track, o.smoother, o.backward_inflation) == (0, tkf.SMOOTHER_RTS, 1e3)
    c = tkf.CkfOptions()
    tkf.lib().tkf_ckf_options_default(ctypes.byref(c))
    assert (c.chi2_max, c.beam, c.max_holes, c.max_entries) == (15.0, 3, 2, 24)
    # the C structs and their ctypes mirrors agree in size
    assert ctypes.sizeof(tkf.CkfInputs) == 8 * 13 and ctypes.sizeof(tkf.FitOptions) % 8 == 0


def test_null_and_handle_errors_need_no_device():
    L = tkf.lib()
    assert L.tkf_context_create(0, None) == 1  # TKF_ERR_INVALID_ARG
    assert b"NULL" in L.tkf_last_error(None)
    assert L.tkf_geometry_create(None, None, 0, None, None) == 2  # TKF_ERR_BAD_HANDLE
    assert L.tkf_field_create(None, None, None) == 2
    o = tkf.FitOptions()
    L.tkf_fit_options_default(ctypes.byref(o))
    assert L.tkf_fit(None, None, None, ctypes.byref(o), None, None, None) == 2
    assert L.tkf_fit_host(None, None, None, ctypes.byref(o), None, None, None) == 2
    assert L.tkf_estimate_seeds(None, None, None, 0, None, None, None) == 2
    assert L.tkf_find_tracks(None, None, None, ctypes.byref(o), None, None, None, None) == 2
    L.tkf_context_destroy(None)
    L.tkf_geometry_destroy(None)
    L.tkf_field_destroy(None)


def test_context_create_reports_missing_or_wrong_device():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present; covered by the GPU tests")
    h = ctypes.c_void_p()
    code = tkf.lib().tkf_context_create(0, ctypes.byref(h))
    assert code == 3  # TKF_ERR_DEVICE
    assert tkf.lib().tkf_last_error(None)
    with pytest.raises(tkf.TkfError):
        tkf.Context(0)


def test_silicon_material():
    m = tkf.Material()
    tkf.lib().tkf_material_silicon(ctypes.byref(m))
    assert (m.z_over_a, m.i_ev, m.rho_g_cm3, m.hbar_omega_p_ev) == (0.49848, 173.0, 2.329, 31.05)
