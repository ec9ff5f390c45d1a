"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/sph.h declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sph.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(sph_[a-z_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libsph():
    from paper_2305_13380_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for f in ("sph_create", "sph_destroy", "sph_build_cells", "sph_density", "sph_force",
              "sph_step", "sph_error_string", "sph_status"):
        assert f in names


def test_every_declared_symbol_is_exported(libsph):
    for name in _declared():
        assert hasattr(libsph, name), name


def test_error_strings_and_defaults(libsph):
    from paper_2305_13380_gb300 import sph
    assert sph.error_string(sph.SPH_E_REBUILD).startswith("kernel support")
    assert sph.error_string(12345) == "unknown error"
    p = sph.sph_default_params()
    assert p.eta == pytest.approx(1.2348) and p.gamma == pytest.approx(5.0 / 3.0)
    assert p.alpha_v == pytest.approx(0.8) and p.beta_v == 3.0 and p.eps_balsara == 1e-4


def test_create_rejects_bad_params_without_gpu(libsph):
    from paper_2305_13380_gb300 import sph
    p = sph.sph_default_params(box_size=-1.0)
    h = ctypes.c_void_p()
    assert sph.lib().sph_create(ctypes.byref(h), ctypes.byref(p), None) == sph.SPH_E_INVAL
    assert sph.lib().sph_create(None, ctypes.byref(p), None) == sph.SPH_E_INVAL



def test_sphenix_defaults_and_argument_checks_without_gpu(libsph):
    from paper_2305_13380_gb300 import sph
    x = sph.sph_sphenix_default_params()
    assert (x.alpha_v_max, x.ell, x.beta_c, x.alpha_c_min, x.alpha_c_max) == (2.0, 0.05, 1.0, 0.0, 1.0)
    # NULL context and parameters are rejected before any device work
    L = sph.lib()
    assert L.sph_sphenix_gradient(None, None, None, None, ctypes.byref(x), 0.0, None) == sph.SPH_E_INVAL
    assert L.sph_force_sphenix(None, None, None, None, None, None, None) == sph.SPH_E_INVAL
    bad = sph.sph_sphenix_default_params(alpha_c_max=-1.0)
    assert L.sph_step_sphenix(None, None, ctypes.byref(bad), None, None) == sph.SPH_E_INVAL


def test_kernel_parameter_checked_without_gpu(libsph):
    from paper_2305_13380_gb300 import sph
    h = ctypes.c_void_p()
    for kw in (dict(kernel=3), dict(kernel=-1)):
        p = sph.sph_default_params(**kw)
        assert sph.lib().sph_create(ctypes.byref(h), ctypes.byref(p), None) == sph.SPH_E_INVAL, kw
    assert sph.sph_default_params().kernel == sph.SPH_KERNEL_CUBIC


def test_new_entry_points_reject_null_arguments_without_gpu(libsph):
    from paper_2305_13380_gb300 import sph
    L = sph.lib()
    t = ctypes.c_int64(0)
    assert L.sph_density_active(None, None, None, None, None, None) == sph.SPH_E_INVAL
    assert L.sph_force_active(None, None, None, None, None, None) == sph.SPH_E_INVAL
    assert L.sph_time_bins(None, None, None, None, None, 0.1, 1.0, 10, None) == sph.SPH_E_INVAL
    assert L.sph_hier_substep(None, None, None, None, 1.0, 4, 0, 1, None, ctypes.byref(t)) == sph.SPH_E_INVAL
    assert L.sph_hier_substep_dev(None, None, None, None, 1.0, 4, None, 1, None) == sph.SPH_E_INVAL


def test_lanes_per_target_checked_without_gpu(libsph):
    import ctypes
    from paper_2305_13380_gb300 import sph
    assert sph.sph_default_params().lanes_per_target == 0
    for bad in (1, 3, 8, -2):
        p = sph.sph_default_params(lanes_per_target=bad)
        h = ctypes.c_void_p()
        assert sph.lib().sph_create(ctypes.byref(h), ctypes.byref(p), None) == sph.SPH_E_INVAL, bad
