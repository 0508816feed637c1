"""Pins of the oracle's forces by ik differentiation (Sec. 2.3: the force from
multiplication by i k in Fourier space, with extra inverse transforms) against
closed forms, the direct Ewald sum O1 and exact identities."""
import math

import numpy as np

import oracle
from paper_1712_04718_gb300 import systems


def _rel_rms(a, b):
    return math.sqrt(((a - b) ** 2).sum() / (b ** 2).sum())


def _plane_wave(M, n, theta):
    j = np.arange(M)
    X, Y, Z = np.meshgrid(j, j, j, indexing="ij")
    return 2.0 * math.pi * (n[0] * X + n[1] * Y + n[2] * Z) / M + theta


def test_spectral_derivative_of_plane_wave():
    """d/dx_d cos(k.x + theta) = -k_d sin(k.x + theta), k = 2 pi n / L, for a
    wave with a different wave number on each axis (sign, scale and axis)."""
    M, L = 12, 1.7
    n = (1, -2, 3)
    ph = _plane_wave(M, n, 0.4)
    fr, fi = oracle.dft3(np.cos(ph), np.zeros_like(ph), -1)
    for d in range(3):
        dr, di = oracle.spectral_derivative(fr, fi, L, d)
        br, bi = oracle.dft3(dr, di, +1)
        expect = -(2.0 * math.pi * n[d] / L) * np.sin(ph)
        assert np.abs(br / M ** 3 - expect).max() < 1e-12
        assert np.abs(bi / M ** 3).max() < 1e-12


def test_spectral_derivative_nyquist_reading():
    """The Nyquist mode of an even grid (cos(pi j) along x) has no defined
    derivative on the grid; the reading gives 0, and leaves other axes at 0."""
    M, L = 10, 2.0
    ph = _plane_wave(M, (M // 2, 0, 0), 0.0)
    fr, fi = oracle.dft3(np.cos(ph), np.zeros_like(ph), -1)
    for d in range(3):
        dr, di = oracle.spectral_derivative(fr, fi, L, d)
        br, bi = oracle.dft3(dr, di, +1)
        assert np.abs(br / M ** 3).max() < 1e-12 and np.abs(bi / M ** 3).max() < 1e-12
    # without the reading (k = +pi M / L at the Nyquist index) the x
    # derivative would be imaginary, -i (pi M / L) cos(pi j)
    dr, di = oracle.spectral_derivative(fr, fi, L, 0)
    assert np.abs(fr).max() > 100.0 and np.abs(dr).max() < 1e-9 * np.abs(fr).max()
    # an odd grid has no Nyquist index: the highest mode is differentiated
    M = 9
    ph = _plane_wave(M, (4, 0, 0), 0.3)
    fr, fi = oracle.dft3(np.cos(ph), np.zeros_like(ph), -1)
    dr, di = oracle.spectral_derivative(fr, fi, L, 0)
    br, _ = oracle.dft3(dr, di, +1)
    assert np.abs(br / M ** 3 + (2.0 * math.pi * 4 / L) * np.sin(ph)).max() < 1e-12


def test_ik_forces_match_ewald_at_large_P_and_M():
    """With P = 24 and M = 4 xi L + margin the ik forces equal the direct
    Ewald k-space forces to FP64 rounding; the potential is the analytic
    mode's, bit for bit (the same spread, transforms and gather)."""
    L, xi = 3.0, 3.5
    x, q = systems.uniform_charges(200, L, seed=12)
    E1, _, F1 = oracle.ewald_kspace(x, q, L, xi)
    M = 2 * math.ceil(6.2 * xi * L / math.pi)
    r = oracle.se_kspace_ik(x, q, L, xi, M, 24)
    ra = oracle.se_kspace(x, q, L, xi, M, 24)
    assert _rel_rms(r["F"], F1) < 1e-12
    assert abs(r["E"] - E1) < 1e-12 * abs(E1)
    assert np.array_equal(r["phi"], ra["phi"])
    assert r["E"] == ra["E"]


def test_ik_forces_conserve_momentum():
    """With one window for spread and gather, sum_m F_m = -(h^3/M^3) sum_k
    i k G |Hhat_k|^2 is a sum of terms odd in k: zero to rounding for ik
    forces, while the analytic forces carry a net force of the order of their
    error (Sec. 4.5)."""
    L, xi, M = 3.0, 3.5, 32
    x, q = systems.uniform_charges(200, L, seed=12)
    for P in (6, 8):
        r = oracle.se_kspace_ik(x, q, L, xi, M, P)
        ra = oracle.se_kspace(x, q, L, xi, M, P)
        scale = np.abs(r["F"]).sum()
        assert np.linalg.norm(r["F"].sum(0)) < 1e-14 * scale
        assert np.linalg.norm(ra["F"].sum(0)) > 1e-6 * scale


def test_ik_forces_more_accurate_than_analytic_at_moderate_P():
    """At moderate P both force modes converge to O1; differentiation in
    Fourier space is the more accurate one (Sec. 2.3): its rms force error
    is below the analytic force's at every P here."""
    L, xi = 3.0, 3.5
    x, q = systems.uniform_charges(200, L, seed=12)
    _, _, F1 = oracle.ewald_kspace(x, q, L, xi)
    prev = None
    for P, M in ((6, 32), (8, 32), (10, 40)):
        e_ik = _rel_rms(oracle.se_kspace_ik(x, q, L, xi, M, P)["F"], F1)
        e_an = _rel_rms(oracle.se_kspace(x, q, L, xi, M, P)["F"], F1)
        assert e_ik < e_an
        if prev is not None:
            assert e_ik < prev
        prev = e_ik


def test_ik_water_box_force_error():
    """A small SPC/E-like water box at the water workload's spacing (h = 6/52):
    at P = 6 and 8 the ik forces are closer to O1 than the analytic ones, and
    both are within a factor 3 of each other (for the charged water layout the
    window's truncation, common to both modes, dominates)."""
    L, xi = 2.0, 3.12
    x, q = systems.water_box(L, seed=2)
    M = int(round(L / (6.0 / 52)))
    M += M % 2
    _, _, F1 = oracle.ewald_kspace(x, q, L, xi)
    for P in (6, 8):
        e_ik = _rel_rms(oracle.se_kspace_ik(x, q, L, xi, M, P)["F"], F1)
        e_an = _rel_rms(oracle.se_kspace(x, q, L, xi, M, P)["F"], F1)
        assert e_an / 3.0 < e_ik < e_an, (P, e_ik, e_an)
