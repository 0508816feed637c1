"""The elementwise comparison of the GPU tests (tests/parity.py), on host
arrays only: a single particle perturbed on the host is caught although the
normwise error stays below the tolerance, small forces are held to an
absolute bound of the typical force, and grids compare point by point.
The arrays are the oracle's own results (O2), so the test also runs on the
shapes and magnitudes the GPU tests compare."""
import numpy as np
import pytest

import oracle
from paper_1712_04718_gb300 import systems
from parity import assert_close, measure


@pytest.fixture(scope="module")
def o2():
    x, q = systems.water_box(2.2, seed=5)
    return x, q, oracle.se_kspace(x, q, 2.2, 3.12, 20, 6, grids=True)


def test_identical_arrays_pass(o2):
    x, q, r = o2
    assert assert_close(r["F"], r["F"], 1e-15, q=q) == (0.0, 0.0)
    assert_close(r["phi"], r["phi"], 1e-15)
    assert_close(r["H"], r["H"], 1e-15)


def test_one_perturbed_particle_is_caught(o2):
    """One particle's force off by tol sqrt(N)/2 of a typical force (0.16 %
    here): the normwise error is tol/2, the elementwise check fails."""
    x, q, r = o2
    N = len(q)
    tol = 1e-4
    F = r["F"].copy()
    typical = np.sqrt((F ** 2).sum(axis=1).mean())
    i = int(np.argmin(np.sqrt((F ** 2).sum(axis=1))))       # the weakest force
    F[i, 0] += 0.5 * tol * np.sqrt(N) * typical
    normwise, elem, j = measure(F, r["F"], q)
    assert normwise < tol                                     # normwise alone would pass
    assert j == i and elem > tol
    with pytest.raises(AssertionError):
        assert_close(F, r["F"], tol, q=q)


def test_perturbed_potential_and_grid_point_are_caught(o2):
    x, q, r = o2
    phi = r["phi"].copy()
    phi[7] += 5e-3 * np.sqrt((phi ** 2).mean())
    with pytest.raises(AssertionError):
        assert_close(phi, r["phi"], 1e-3)
    H = r["H"].copy()
    H[3, 4, 5] += 5e-3 * np.sqrt((H ** 2).mean())
    with pytest.raises(AssertionError):
        assert_close(H, r["H"], 1e-3)
    assert measure(H, r["H"])[0] < 1e-3


def test_scale_is_relative_for_large_and_absolute_for_small(o2):
    """A relative error tol/2 on every particle passes; the same absolute
    error (tol/2 of the typical field times the charge) on a particle whose
    force is tiny passes too; twice the bound fails."""
    x, q, r = o2
    tol = 1e-4
    F = r["F"] * (1.0 + 0.5 * tol)
    assert_close(F, r["F"], tol, q=q)
    Fa = r["F"].copy()
    rn = np.sqrt((Fa ** 2).sum(axis=1))
    e_rms = np.sqrt(((rn / np.abs(q)) ** 2).mean())
    i = int(np.argmin(rn))
    Fa[i, 1] += 0.5 * tol * abs(q[i]) * e_rms
    assert_close(Fa, r["F"], tol, q=q)
    Fa[i, 1] += 4.0 * tol * abs(q[i]) * e_rms
    with pytest.raises(AssertionError):
        assert_close(Fa, r["F"], tol, q=q)


def test_shape_mismatch_and_empty():
    with pytest.raises(AssertionError):
        assert_close(np.zeros((3, 3)), np.zeros((4, 3)), 1e-3)
    assert assert_close(np.zeros((0, 3)), np.zeros((0, 3)), 1e-3) == (0.0, 0.0)
