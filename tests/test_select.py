"""Parameter selection (se_select_params, host code of libse): the Lambert
function against its closed forms, the support rule against the paper's
remark after the error bounds (Sec. 4), and the selected (xi, M, P) against
the errors the oracles actually measure: the real-space sum at the cut-off
plus the SE k-space sum at the selected parameters, against the converged
Ewald total (each of the three error sources is sized to the tolerance, so
the total stays within 2 tol)."""
import ctypes
import math

import numpy as np
import pytest

import oracle
from paper_1712_04718_gb300 import _native as nat
from paper_1712_04718_gb300 import se, systems


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()


def test_lambert_w0_closed_forms():
    """W0(n e^n) = n; W0(0) = 0; w e^w = z over 300 decades; NaN below 0."""
    for n in (1e-9, 0.01, 0.5, 1.0, 2.0, 3.0, 10.0, 50.0, 300.0):
        assert abs(se.lambert_w0(n * math.exp(n)) - n) <= 1e-14 * max(1.0, n)
    assert se.lambert_w0(0.0) == 0.0
    assert se.lambert_w0(math.e) == pytest.approx(1.0, abs=1e-15)
    for lz in np.linspace(-25.0, 690.0, 143):
        w = se.lambert_w0(math.exp(lz))
        assert abs(w + math.log(w) - lz) <= 1e-13 * max(1.0, abs(lz))
    assert math.isnan(se.lambert_w0(-0.1))


def test_support_rule_paper_remark():
    """The remark after the force bound: relative approximation errors of
    1e-6 and 1e-12 need P of about 10 and 20 (e^{-pi P c^2/2}, c = 0.95,
    rounded up to even); smaller tolerances never need smaller P."""
    assert se.select_support(1e-6) == 10
    assert se.select_support(1e-12) == 20
    prev = 2
    for t in np.logspace(0, -15, 46):
        P = se.select_support(t)
        assert P % 2 == 0 and P >= prev
        assert math.exp(-math.pi * P * 0.95 ** 2 / 2) <= t * (1 + 1e-12)
        prev = P
    assert se.select_support(5.0) == 2
    lib = nat.load()
    assert lib.se_select_support(0.0, 0.95) == nat.SE_ERR_ARG
    assert lib.se_select_support(1e-6, -1.0) == nat.SE_ERR_ARG


CASES = [("potential", 1e-4, 0.6), ("potential", 1e-7, 0.8), ("potential", 1e-10, 1.0),
         ("energy", 1e-4, 0.6), ("energy", 1e-7, 0.8),
         ("force", 1e-3, 0.6), ("force", 1e-5, 0.7), ("force", 1e-8, 0.9)]


@pytest.mark.parametrize("quantity,tol,rc", CASES)
def test_selected_parameters_meet_tolerance(quantity, tol, rc):
    L = 2.0
    x, q = systems.uniform_charges(300, L, seed=3)
    Q = float((q ** 2).sum())
    s = se.select_params(quantity, tol, rc, L, Q)
    assert s["supported"]
    xi, M, P = s["xi"], s["M"], s["P"]
    assert M % 2 == 0 and P % 2 == 0 and 2 <= P <= M and M >= 2 * math.ceil(s["k_inf"])
    eta = P * L * L * xi * xi / (0.95 ** 2 * math.pi * M * M)
    assert eta <= 0.5 + 1e-12
    E_t, phi_t, F_t = oracle.ewald_total(x, q, L, xi)
    r = oracle.ewald_real(x, q, L, xi, rc)
    k = oracle.se_kspace(x, q, L, xi, M, P)
    if quantity == "potential":
        err = math.sqrt(((r["phi_real"] + r["phi_self"] + k["phi"] - phi_t) ** 2).mean())
    elif quantity == "energy":
        err = abs(r["E_real"] + r["E_self"] + k["E"] - E_t)
    else:
        err = math.sqrt(((r["F_real"] + k["F"] - F_t) ** 2).sum(1).mean())
    assert err <= 2.0 * tol, (s, err / tol)
    if quantity != "energy":   # one signed number can fall far below its rms estimate
        assert err >= tol / 50.0, (s, err / tol)


def test_truncation_terms_match_their_estimates():
    """The real-space and Fourier-space truncation errors at the selected
    xi and k_inf are of the size the estimates (Eq. 2.2) put at tol."""
    L, tol, rc = 2.0, 1e-7, 0.8
    x, q = systems.uniform_charges(300, L, seed=3)
    Q = float((q ** 2).sum())
    s = se.select_params("potential", tol, rc, L, Q)
    xi, M = s["xi"], s["M"]
    _, phi_t, _ = oracle.ewald_total(x, q, L, xi)
    r = oracle.ewald_real(x, q, L, xi, rc)
    Mbig = max(M, 2 * math.ceil(6.2 * xi * L / math.pi))
    exact_k = oracle.se_kspace(x, q, L, xi, Mbig, 24)
    e_real = math.sqrt(((r["phi_real"] + r["phi_self"] + exact_k["phi"] - phi_t) ** 2).mean())
    assert tol / 3 < e_real < 3 * tol
    # the Fourier sum cut at |n| <= M/2 (the grid's modes) against the full one
    nmax = M // 2
    _, phi_cut, _ = oracle.ewald_kspace(x, q, L, xi, nmax=nmax)
    e_four = math.sqrt(((phi_cut - exact_k["phi"]) ** 2).mean())
    assert e_four < 3 * tol


def test_selection_argument_errors():
    lib = nat.load()
    xi, kinf = ctypes.c_double(), ctypes.c_double()
    M, P = ctypes.c_int(), ctypes.c_int()
    args = (ctypes.byref(xi), ctypes.byref(M), ctypes.byref(P), ctypes.byref(kinf))
    good = (nat.SE_QUANTITY_FORCE, 1e-5, 0.8, 3.0, 100.0, 0.95)
    assert lib.se_select_params(*good, *args) == nat.SE_OK
    for i, bad in ((0, 3), (1, 0.0), (1, float("nan")), (2, -1.0), (3, 0.0), (4, 0.0),
                   (5, -0.5)):
        a = list(good)
        a[i] = bad
        assert lib.se_select_params(*a, *args) == nat.SE_ERR_ARG, (i, bad)
    assert lib.se_select_params(*good, None, ctypes.byref(M), ctypes.byref(P),
                                None) == nat.SE_ERR_ARG
    # a tolerance that needs P > 32: outputs written, status unsupported
    s = se.select_params("force", 1e-19, 0.8, 3.0, 100.0)
    assert not s["supported"] and s["P"] > 32
    # a tolerance met by the real-space sum alone (the force estimate's log <= 0)
    s = se.select_params("force", 1e6, 0.8, 3.0, 100.0)
    assert not s["supported"]
