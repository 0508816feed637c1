"""Pins of oracle O1 (classic Ewald sum, Sec. 1 Eq. 1.5-1.7) against facts
that do not come from the oracle itself: a lattice constant, invariances of
the exact sum, brute-force image sums and derivative identities."""
import math

import numpy as np
import pytest

import oracle
from paper_1712_04718_gb300 import systems
from conftest import read_golden


def test_nacl_madelung():
    """Rock salt: E = -4 M / r0 for the 8-ion cell (tests/golden/nacl_madelung.txt),
    for several xi and two cell sizes; forces vanish by symmetry."""
    M_ref = float(read_golden("nacl_madelung.txt")["madelung"])
    for a in (1.0, 2.5):
        x, q = systems.nacl_cell(a)
        for xiL in (4.0, 7.0, 10.0):
            E, phi, F = oracle.ewald_total(x, q, a, xiL / a)
            mad = -E * (a / 2) / 4
            assert abs(mad - M_ref) < 2e-13 * M_ref, (a, xiL, mad)
            # every ion sits on a centre of symmetry
            assert np.abs(F).max() < 1e-12
            # phi_m = -M / r0 * q_m (each ion sees the same lattice)
            assert np.allclose(phi * q, -M_ref / (a / 2), rtol=1e-12)


def test_xi_independence():
    """Sec. 1: the Ewald energy and force do not depend on xi."""
    rng = np.random.default_rng(5)
    L = 2.0
    x = rng.uniform(0, L, size=(8, 3))
    q = np.array([1, -1, 2, -2, 0.5, -0.5, 1.5, -1.5])
    ref = None
    for xiL in (5.0, 8.0, 11.0, 15.0):
        E, phi, F = oracle.ewald_total(x, q, L, xiL / L)
        if ref is None:
            ref = (E, phi, F)
            continue
        assert abs(E - ref[0]) < 1e-12 * abs(ref[0])
        assert np.abs(phi - ref[1]).max() < 1e-11 * np.abs(ref[1]).max()
        assert np.abs(F - ref[2]).max() < 1e-11 * np.abs(ref[2]).max()


def _shell_sum(x, q, L, R):
    """Energy of the periodic system summed over image cells |p| <= R in
    spherical order (plain Coulomb, no splitting)."""
    r = np.arange(-R, R + 1)
    P = np.array(np.meshgrid(r, r, r, indexing="ij")).reshape(3, -1).T
    P = P[(P ** 2).sum(1) <= R * R]
    E = 0.0
    for m in range(len(q)):
        for n in range(len(q)):
            d = x[m] - x[n] + P * L
            rr = np.sqrt((d ** 2).sum(1))
            if m == n:
                rr = rr[rr > 0]
            E += 0.5 * q[m] * q[n] * (1.0 / rr).sum()
    return E


@pytest.mark.parametrize("case", ["dipole_pair", "zero_dipole_quad"])
def test_brute_force_spherical_image_sum(case):
    """Summed shell by shell, the Coulomb sum tends to the Ewald (tin-foil)
    energy plus 2 pi |D|^2 / (3 L^3), D = sum q x (the Ewald result corresponds
    to a conducting boundary; Sec. 1 says spherical order, which in vacuum
    carries this dipole term)."""
    L = 1.0
    if case == "dipole_pair":
        x = np.array([[0.1, 0.2, 0.3], [0.45, 0.25, 0.35]])
        q = np.array([1.0, -1.0])
    else:
        x = np.array([[0.1, 0.2, 0.3], [0.45, 0.25, 0.35],
                      [0.3, 0.6, 0.5], [0.65, 0.65, 0.55]])
        q = np.array([1.0, -1.0, -1.0, 1.0])
    D = (q[:, None] * x).sum(0)
    E_ew, _, _ = oracle.ewald_total(x, q, L, 6.0)
    E_bf = _shell_sum(x, q, L, 48)
    expect = E_ew + 2 * math.pi * (D @ D) / (3 * L ** 3)
    assert abs(E_bf - expect) < 1e-6 * abs(expect), (E_bf, expect)


def _random_neutral(N, L, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, L, size=(N, 3))
    q = rng.uniform(-1, 1, size=N)
    q -= q.mean()
    return x, q


def test_kspace_force_is_minus_energy_gradient():
    """F^L = -dE^L/dx (Eq. 1.3), by central differences."""
    L, xi = 1.5, 4.0
    x, q = _random_neutral(12, L, 7)
    E, phi, F = oracle.ewald_kspace(x, q, L, xi)
    hstep = 1e-5
    for m in (0, 5, 11):
        for d in range(3):
            xp, xm = x.copy(), x.copy()
            xp[m, d] += hstep
            xm[m, d] -= hstep
            Ep = oracle.ewald_kspace(xp, q, L, xi)[0]
            Em = oracle.ewald_kspace(xm, q, L, xi)[0]
            fd = -(Ep - Em) / (2 * hstep)
            assert abs(fd - F[m, d]) < 1e-6 * np.abs(F).max(), (m, d, fd, F[m, d])


def test_kspace_potential_is_energy_charge_gradient():
    """E^L is quadratic in q with E = 1/2 sum q phi, so dE/dq_m = phi_m."""
    L, xi = 1.5, 4.0
    x, q = _random_neutral(10, L, 8)
    E, phi, F = oracle.ewald_kspace(x, q, L, xi)
    assert abs(E - 0.5 * (q * phi).sum()) < 1e-12 * abs(E)
    dq = 1e-3
    for m in (0, 4, 9):
        qp, qm = q.copy(), q.copy()
        qp[m] += dq
        qm[m] -= dq
        fd = (oracle.ewald_kspace(x, qp, L, xi)[0] - oracle.ewald_kspace(x, qm, L, xi)[0]) / (2 * dq)
        assert abs(fd - phi[m]) < 1e-9 * np.abs(phi).max()


def test_kspace_momentum_and_translation():
    """The Ewald k-space force sums to zero and E^L is translation invariant."""
    L, xi = 2.0, 3.0
    x, q = _random_neutral(20, L, 9)
    E, phi, F = oracle.ewald_kspace(x, q, L, xi)
    assert np.abs(F.sum(0)).max() < 1e-12 * np.abs(F).max() * len(q)
    E2, phi2, F2 = oracle.ewald_kspace(x + np.array([0.3, -0.7, 1.1]), q, L, xi)
    assert abs(E2 - E) < 1e-12 * abs(E)
    assert np.abs(F2 - F).max() < 1e-11 * np.abs(F).max()


def test_kspace_targets_match_all():
    """Structure-factor evaluation at a subset equals the full evaluation."""
    L, xi = 2.0, 3.0
    x, q = _random_neutral(30, L, 10)
    E, phi, F = oracle.ewald_kspace(x, q, L, xi)
    nmax = oracle.nmax_for(xi, L)
    S = oracle.ewald_structure(x, q, L, nmax)
    idx = np.array([0, 7, 29])
    p2, F2 = oracle.ewald_eval(x[idx], q[idx], S, L, xi, nmax)
    assert np.allclose(p2, phi[idx], rtol=1e-12, atol=1e-14)
    assert np.allclose(F2, F[idx], rtol=1e-12, atol=1e-14)


def test_kolafa_perram_fourier_estimate():
    """Truncating the k sum at |n| <= k_inf leaves a force error of the size
    the Kolafa-Perram estimate (Eq. 2.2c) predicts.  With Q = sum q^2 the
    estimate is read as the root of the summed squared error over all
    particles, i.e. sqrt(N) times the per-particle rms; measured and estimated
    agree within a factor of 2."""
    L, xi = 1.0, 8.0
    N = 400
    x, q = systems.uniform_charges(N, L, seed=3)
    Q = (q ** 2).sum()
    _, _, Fref = oracle.ewald_kspace(x, q, L, xi)
    for kinf in (6, 8, 10):
        _, _, F = oracle.ewald_kspace(x, q, L, xi, nmax=kinf)
        err = np.sqrt(((F - Fref) ** 2).sum(1).mean())
        est = xi / (L * math.pi) * math.sqrt(8.0 / kinf) * Q * math.exp(-(math.pi * kinf / (xi * L)) ** 2)
        est_rms = est / math.sqrt(N)
        assert 0.5 < err / est_rms < 2.0, (kinf, err, est_rms)


def test_real_space_at_targets_equals_full_sum():
    """ewald_real_at at a sample of particles equals the full real-space sum
    there (same images, cut-off and terms), bit for bit."""
    x, q = systems.uniform_charges(300, 2.0, seed=1)
    r = oracle.ewald_real(x, q, 2.0, 4.0, 0.6)
    idx = [0, 7, 150, 299]
    ph, F = oracle.ewald_real_at(x, q, 2.0, 4.0, 0.6, idx)
    assert np.array_equal(ph, r["phi_real"][idx])
    assert np.array_equal(F, r["F_real"][idx])
