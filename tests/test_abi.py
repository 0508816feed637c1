"""The C ABI without a GPU: the library loads, exports every function that
include/se.h declares, and validates arguments and derives parameters on the
host (no device call is made by these entry points)."""
import ctypes
import math
import os
import re

import pytest

import oracle
from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "se.h")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1712_04718_gb300 import _native
    return _native.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(se_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    from paper_1712_04718_gb300 import _native
    names = declared_functions()
    assert "se_energy_force" in names and "se_plan_create" in names
    for n in names:
        assert hasattr(lib, n), n
        assert n in _native.SIGNATURES, "binding lacks " + n


def _create(lib, N, L, xi, M, P):
    h = ctypes.c_void_p()
    rc = lib.se_plan_create(ctypes.byref(h), N, L, xi, M, P)
    return rc, h


def test_argument_validation(lib):
    from paper_1712_04718_gb300 import _native as nat
    bad = [(-1, 1.0, 1.0, 16, 4), (10, 0.0, 1.0, 16, 4), (10, 1.0, -2.0, 16, 4),
           (10, float("nan"), 1.0, 16, 4), (10, 1.0, 1.0, 4, 8), (10, 1.0, 1.0, 16, 0)]
    for args in bad:
        rc, h = _create(lib, *args)
        assert rc == nat.SE_ERR_ARG and not h.value, args
    for P in (5, 34):
        rc, h = _create(lib, 10, 1.0, 1.0, 64, P)
        assert rc == nat.SE_ERR_UNSUPPORTED, P
    rc, h = _create(lib, 0, 1.0, 3.0, 16, 4)   # an empty system is valid
    assert rc == nat.SE_OK and h.value
    assert lib.se_plan_set_precision(h, 7) == nat.SE_ERR_ARG
    assert lib.se_plan_set_shape(h, 1.5, 1) == nat.SE_ERR_ARG        # eta >= 1
    assert lib.se_plan_set_tuning(h, 6, 0) == nat.SE_ERR_ARG
    assert lib.se_plan_set_tuning(h, 5, 0) == nat.SE_ERR_UNSUPPORTED  # single precision only
    assert lib.se_plan_set_tuning(h, 3, 0) == nat.SE_ERR_UNSUPPORTED  # the FP32 pipeline, FP64 plan
    assert lib.se_plan_set_tuning(h, 4, 0) == nat.SE_ERR_UNSUPPORTED
    assert lib.se_plan_set_precision(h, nat.SE_FP32) == nat.SE_OK
    assert lib.se_plan_set_tuning(h, 2, 0) == nat.SE_ERR_UNSUPPORTED  # direct spread is FP64 only
    # force mode: ik differentiation moves the FP32 plan to the cuFFT pipeline
    assert lib.se_plan_set_force_mode(h, 2) == nat.SE_ERR_ARG
    assert lib.se_plan_set_force_mode(None, nat.SE_FORCE_IK) == nat.SE_ERR_ARG
    prm = (ctypes.c_double * 10)()
    assert lib.se_plan_get_params(h, prm) == nat.SE_OK and prm[7] == 3
    assert lib.se_plan_set_force_mode(h, nat.SE_FORCE_IK) == nat.SE_OK
    assert lib.se_plan_get_params(h, prm) == nat.SE_OK and prm[7] == 1
    assert lib.se_plan_set_force_mode(h, nat.SE_FORCE_ANALYTIC) == nat.SE_OK
    assert lib.se_plan_get_params(h, prm) == nat.SE_OK and prm[7] == 3
    # compute calls before any spread are rejected without touching the device
    assert lib.se_scale(h, None) == nat.SE_ERR_ARG
    assert lib.se_gather(h, None, None, None, None, None) == nat.SE_ERR_ARG
    assert lib.se_plan_destroy(h) == nat.SE_OK
    assert lib.se_plan_destroy(None) == nat.SE_OK
    assert lib.se_strerror(nat.SE_ERR_NONFINITE).decode().startswith("non-finite")
    out = ctypes.c_double()
    assert lib.se_probe_peak(9, ctypes.byref(out)) == nat.SE_ERR_ARG
    assert lib.se_probe_peak(0, None) == nat.SE_ERR_ARG


def test_spread_noalloc_rejects_on_the_host(lib):
    """se_spread_noalloc decides every rejection before any CUDA call, so
    dummy non-null pointers are safe here: sizes beyond its static scratch
    (N > 32768, M > 128), a NULL grid, P outside [2, M], odd P."""
    from paper_1712_04718_gb300 import _native as nat
    dummy = ctypes.c_void_p(16)
    f = lib.se_spread_noalloc
    assert f(dummy, dummy, 32769, 3.0, 3.5, 32, 8, dummy, None) == nat.SE_ERR_ARG
    assert f(dummy, dummy, 4, 30.0, 0.5, 129, 8, dummy, None) == nat.SE_ERR_ARG
    assert f(dummy, dummy, 4, 3.0, 3.5, 32, 8, None, None) == nat.SE_ERR_ARG
    assert f(dummy, dummy, -1, 3.0, 3.5, 32, 8, dummy, None) == nat.SE_ERR_ARG
    assert f(None, None, 4, 3.0, 3.5, 32, 8, dummy, None) == nat.SE_ERR_ARG
    assert f(dummy, dummy, 4, 3.0, 3.5, 32, 0, dummy, None) == nat.SE_ERR_ARG
    assert f(dummy, dummy, 4, 3.0, 3.5, 16, 18, dummy, None) == nat.SE_ERR_ARG
    assert f(dummy, dummy, 4, 3.0, 3.5, 32, 7, dummy, None) == nat.SE_ERR_UNSUPPORTED


def test_real_space_arguments(lib):
    """se_real_create validates its arguments on the host; the cell grid is
    floor(K L / rc) per dimension (K = 2, or 3 when K = 2 gives under 512
    cells), at most 40; rc > L/3 is not supported."""
    from paper_1712_04718_gb300 import _native as nat
    h = ctypes.c_void_p()
    for args in ((-1, 3.0, 3.0, 1.0), (10, 0.0, 3.0, 1.0), (10, 3.0, -1.0, 1.0),
                 (10, 3.0, 3.0, 0.0), (10, float("inf"), 3.0, 1.0)):
        assert lib.se_real_create(ctypes.byref(h), *args) == nat.SE_ERR_ARG, args
    assert lib.se_real_create(ctypes.byref(h), 10, 3.0, 3.0, 1.01) == nat.SE_ERR_UNSUPPORTED
    n = ctypes.c_int()
    for L, rc, cells in ((3.0, 1.0, 9), (6.0, 1.0, 12), (10.0, 0.9, 22), (100.0, 1.0, 40)):
        assert lib.se_real_create(ctypes.byref(h), 10, L, 3.0, rc) == nat.SE_OK
        assert lib.se_real_get_cells(h, ctypes.byref(n)) == nat.SE_OK and n.value == cells
        assert lib.se_real_set_reach(h, 4) == nat.SE_ERR_ARG
        assert lib.se_real_set_reach(h, 1) == nat.SE_OK
        assert lib.se_real_get_cells(h, ctypes.byref(n)) == nat.SE_OK
        assert n.value == min(40, int(L / rc))
        assert lib.se_real_set_reach(h, 0) == nat.SE_OK
        assert lib.se_real_set_precision(h, 5) == nat.SE_ERR_ARG
        assert lib.se_real_set_prefactor(h, -1.0) == nat.SE_ERR_ARG
        assert lib.se_real_destroy(h) == nat.SE_OK
    assert lib.se_real_destroy(None) == nat.SE_OK
    # missing inputs are rejected before any device call
    assert lib.se_real_create(ctypes.byref(h), 10, 3.0, 3.0, 1.0) == nat.SE_OK
    assert lib.se_real_evaluate(h, None, None, None, None, None, 0) == nat.SE_ERR_ARG
    assert lib.se_real_evaluate(None, None, None, None, None, None, 0) == nat.SE_ERR_ARG
    assert lib.se_real_destroy(h) == nat.SE_OK


@pytest.mark.parametrize("L,xi,M,P", [(3.0, 3.5, 32, 16), (6.0, 3.12, 52, 6), (10.0, 3.12, 84, 8)])
def test_derived_parameters_match_oracle(lib, L, xi, M, P):
    """h, w, eta (Eq. 4.2), alpha and c_g of the library equal the oracle's."""
    rc, h = _create(lib, 100, L, xi, M, P)
    assert rc == 0
    out = (ctypes.c_double * 10)()
    assert lib.se_plan_get_params(h, out) == 0
    ref = oracle.se_params(L, xi, M, P)
    for i, k in enumerate(["h", "w", "eta", "alpha", "cg", "m"]):
        assert math.isclose(out[i], ref[k], rel_tol=1e-14), k
    lib.se_plan_destroy(h)


def test_self_energy(lib):
    """Self term of Eq. 1.6: -xi/sqrt(pi) sum q^2."""
    rc, h = _create(lib, 4, 2.0, 3.0, 16, 4)
    q = (ctypes.c_double * 4)(1.0, -1.0, 0.5, -0.5)
    E = ctypes.c_double()
    assert lib.se_self_energy(h, q, 4, ctypes.byref(E)) == 0
    assert math.isclose(E.value, -3.0 / math.sqrt(math.pi) * 2.5, rel_tol=1e-15)
    lib.se_plan_destroy(h)


def test_library_links_no_oracle():
    """The product library shares nothing with the oracle: no oracle symbol is
    exported by libse, and no file of the package refers to the oracle."""
    from paper_1712_04718_gb300 import _native
    _native.load()
    pkg = os.path.join(ROOT, "paper_1712_04718_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in src.lower(), f
