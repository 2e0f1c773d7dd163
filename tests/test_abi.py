"""C-ABI checks that need no GPU: the library builds, loads and exports every
entry point declared in include/gridspt.h; host-only logic (argument
validation, spectrum normalisation) behaves as documented."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gridspt.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1807_04215_gb300 import _lib, build
    build.build()
    return _lib.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gridspt_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_four_named_calls():
    names = declared_functions()
    for n in ("gridspt_make_linear_field", "gridspt_run_orders", "gridspt_power", "gridspt_bispectrum"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1807_04215_gb300 import _lib
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"binding lacks {name}"


def test_plan_create_rejects_bad_sizes_before_touching_cuda(lib):
    from paper_1807_04215_gb300 import _lib
    for n, n_max, box in [(10, 3, 100.0), (2048, 3, 100.0), (7, 3, 100.0), (64, 0, 100.0), (64, 9, 100.0),
                          (64, 3, -1.0)]:
        d = _lib.GridsptDesc(n, n_max, 1, 0, box, 0.0, 0.0, 0)
        h = ctypes.c_void_p()
        st = lib.gridspt_plan_create(ctypes.byref(d), ctypes.byref(h))
        assert st == 1, (n, n_max, box)
        assert h.value is None
        assert lib.gridspt_last_error()


def test_plan_create_rejects_unknown_source_form(lib):
    from paper_1807_04215_gb300 import _lib
    for form in (-1, 2, 7):
        d = _lib.GridsptDesc(64, 3, 1, form, 100.0, 0.0, 0.0, 0)
        h = ctypes.c_void_p()
        assert lib.gridspt_plan_create(ctypes.byref(d), ctypes.byref(h)) == 1, form
        assert h.value is None
        assert b"form" in lib.gridspt_last_error()


def test_plan_create_rejects_bad_truncation(lib):
    from paper_1807_04215_gb300 import _lib
    for form, trunc in ((0, 2), (0, -1), (1, 1)):      # bad value; divergence form with truncation
        d = _lib.GridsptDesc(64, 3, 1, form, 100.0, 0.0, 0.0, trunc)
        h = ctypes.c_void_p()
        assert lib.gridspt_plan_create(ctypes.byref(d), ctypes.byref(h)) == 1, (form, trunc)
        assert h.value is None
        assert b"truncate" in lib.gridspt_last_error()


def test_null_plan_is_rejected(lib):
    b = ctypes.c_size_t()
    assert lib.gridspt_workspace_size(None, ctypes.byref(b)) == 1
    assert lib.gridspt_plan_destroy(None) == 0


def test_linear_amplitude_matches_oracle(lib):
    """The library's FP64 sigma_8 normalisation (its own Simpson rule in C)
    against the oracle's, for two cosmologies."""
    from oracle import cosmology
    from paper_1807_04215_gb300 import _lib
    for c in [cosmology.DEFAULT_COSMO, dict(omega_m=0.25, h=0.7, n_s=1.0, sigma8=0.9, gamma=0.18)]:
        A = ctypes.c_double()
        cc = _lib.GridsptCosmo(**c)
        assert lib.gridspt_linear_amplitude(ctypes.byref(cc), ctypes.byref(A)) == 0
        ref = cosmology.amplitude(dict(c))
        assert abs(A.value / ref - 1) < 1e-10


def test_growth_factor_matches_oracle(lib):
    """The library's FP64 growth factor (its own Simpson rule in C) against the
    oracle's, and the invalid arguments it rejects."""
    from oracle import cosmology
    from paper_1807_04215_gb300 import _lib
    for om in (0.3, 0.25, 1.0):
        c = dict(cosmology.DEFAULT_COSMO, omega_m=om)
        cc = _lib.GridsptCosmo(**c)
        for z in (0.0, 0.5, 1.0, 3.0):
            D = ctypes.c_double()
            assert lib.gridspt_growth_factor(ctypes.byref(cc), z, ctypes.byref(D)) == 0
            assert abs(D.value - cosmology.growth_factor(z, c)) < 1e-12
    D = ctypes.c_double()
    bad = _lib.GridsptCosmo(**dict(cosmology.DEFAULT_COSMO, omega_m=0.0))
    assert lib.gridspt_growth_factor(ctypes.byref(bad), 0.5, ctypes.byref(D)) == 1
    good = _lib.GridsptCosmo(**cosmology.DEFAULT_COSMO)
    assert lib.gridspt_growth_factor(ctypes.byref(good), -1.0, ctypes.byref(D)) == 1
