"""ctypes wrapper of ``se_oracle.c`` (test infrastructure; see package docstring).

The C file is compiled with gcc on first use (``build()``), into
``oracle/_build/``.  Arrays are passed as contiguous float64 numpy arrays.
"""
import ctypes
import math
import os
import platform
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "se_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libseoracle_%s.so" % platform.machine())
_lib = None

__all__ = [
    "build", "num_threads", "set_num_threads", "se_params", "nmax_for",
    "ewald_kspace", "ewald_structure", "ewald_eval", "ewald_real", "ewald_total",
    "se_kspace", "se_spread", "dft3", "se_scale", "se_gather",
    "spectral_derivative", "se_kspace_ik", "ewald_real_at",
]


def build(force=False):
    """Compile se_oracle.c with gcc (-O2, OpenMP, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        d, i64, i = ctypes.c_double, ctypes.c_int64, ctypes.c_int
        p = ctypes.c_void_p
        lib.oracle_num_threads.restype = i
        lib.oracle_set_num_threads.argtypes = [i]
        lib.oracle_ewald_structure.argtypes = [i64, p, p, d, i, p, p]
        lib.oracle_ewald_structure.restype = i
        lib.oracle_ewald_energy.argtypes = [p, p, d, d, i]
        lib.oracle_ewald_energy.restype = d
        lib.oracle_ewald_eval.argtypes = [i64, p, p, p, p, d, d, i, p, p]
        lib.oracle_ewald_kspace.argtypes = [i64, p, p, d, d, i, p, p, p]
        lib.oracle_ewald_kspace.restype = i
        lib.oracle_ewald_real.argtypes = [i64, p, p, d, d, d, p, p, p, p, p]
        lib.oracle_ewald_real_at.argtypes = [i64, p, p, d, d, d, i64, p, p, p]
        lib.oracle_se_params.argtypes = [d, d, i, i, d, d, p]
        lib.oracle_dft3.argtypes = [p, p, i, i]
        lib.oracle_spectral_derivative.argtypes = [p, p, i, d, i]
        lib.oracle_se_kspace_ik.argtypes = [i64, p, p, d, d, i, i, d, d, i, p, p, p]
        lib.oracle_se_kspace_ik.restype = i
        lib.oracle_se_spread.argtypes = [i64, p, p, d, i, i, d, d, i, p]
        lib.oracle_se_scale.argtypes = [p, p, i, d, d, d, p]
        lib.oracle_se_gather.argtypes = [i64, p, p, d, i, i, d, d, i, p, p, p]
        lib.oracle_se_kspace.argtypes = [i64, p, p, d, d, i, i, d, d, i,
                                         p, p, p, p, p, p]
        lib.oracle_se_kspace.restype = i
        _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads():
    return _L().oracle_num_threads()


def set_num_threads(n):
    _L().oracle_set_num_threads(int(n))


def se_params(L, xi, M, P, c=0.95, eta=None):
    """h, w, eta, alpha, c_g, m of Sec. 3 / Eq. 4.2 (eta given overrides c)."""
    out = np.zeros(6)
    _L().oracle_se_params(float(L), float(xi), int(M), int(P), float(c),
                          float(eta) if eta else 0.0, _ptr(out))
    return dict(h=out[0], w=out[1], eta=out[2], alpha=out[3], cg=out[4], m=out[5])


def nmax_for(xi, L, tol=1e-16):
    """Largest |n| so that e^{-k^2/(4 xi^2)} >= tol is kept (k = 2 pi n / L)."""
    kmax = 2.0 * xi * math.sqrt(math.log(1.0 / tol))
    return int(math.ceil(kmax * L / (2.0 * math.pi)))


def ewald_structure(x, q, L, nmax):
    x, q = _f64(x), _f64(q)
    W = 2 * nmax + 1
    Sr = np.zeros((nmax + 1) * W * W)
    Si = np.zeros_like(Sr)
    rc = _L().oracle_ewald_structure(len(q), _ptr(x), _ptr(q), float(L), int(nmax),
                                     _ptr(Sr), _ptr(Si))
    if rc:
        raise MemoryError("oracle_ewald_structure")
    return Sr, Si


def ewald_eval(xt, qt, S, L, xi, nmax):
    """phi^L, F^L at target positions xt with charges qt from S = (Sr, Si)."""
    xt, qt = _f64(xt), _f64(qt)
    phi = np.zeros(len(qt))
    F = np.zeros((len(qt), 3))
    _L().oracle_ewald_eval(len(qt), _ptr(xt), _ptr(qt), _ptr(S[0]), _ptr(S[1]),
                           float(L), float(xi), int(nmax), _ptr(phi), _ptr(F))
    return phi, F


def ewald_kspace(x, q, L, xi, nmax=None, tol=1e-16):
    """O1 k-space part: (E^L, phi^L [N], F^L [N,3]) by the direct k sum."""
    x, q = _f64(x), _f64(q)
    if nmax is None:
        nmax = nmax_for(xi, L, tol)
    phi = np.zeros(len(q))
    F = np.zeros((len(q), 3))
    E = ctypes.c_double()
    rc = _L().oracle_ewald_kspace(len(q), _ptr(x), _ptr(q), float(L), float(xi),
                                  int(nmax), ctypes.byref(E), _ptr(phi), _ptr(F))
    if rc:
        raise MemoryError("oracle_ewald_kspace")
    return E.value, phi, F


def ewald_real(x, q, L, xi, rc):
    """O1 real-space image sum and self term.

    Returns dict(E_real, E_self, phi_real, phi_self, F_real)."""
    x, q = _f64(x), _f64(q)
    N = len(q)
    phi = np.zeros(N)
    phis = np.zeros(N)
    F = np.zeros((N, 3))
    Er, Es = ctypes.c_double(), ctypes.c_double()
    _L().oracle_ewald_real(N, _ptr(x), _ptr(q), float(L), float(xi), float(rc),
                           ctypes.byref(Er), ctypes.byref(Es), _ptr(phi), _ptr(phis),
                           _ptr(F))
    return dict(E_real=Er.value, E_self=Es.value, phi_real=phi, phi_self=phis,
                F_real=F)


def ewald_real_at(x, q, L, xi, rc, idx):
    """O1 real-space phi (self term excluded) and F at the particles idx."""
    x, q = _f64(x), _f64(q)
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
    phi = np.zeros(len(idx))
    F = np.zeros((len(idx), 3))
    _L().oracle_ewald_real_at(len(q), _ptr(x), _ptr(q), float(L), float(xi), float(rc),
                              len(idx), idx.ctypes.data_as(ctypes.c_void_p), _ptr(phi), _ptr(F))
    return phi, F


def ewald_total(x, q, L, xi, tol=1e-16):
    """Full Ewald E, phi, F (real + k-space + self), converged to about tol."""
    # erfc(xi rc) <= tol  (erfc(t) < e^{-t^2}); take t with e^{-t^2} = tol/10
    rc = math.sqrt(math.log(10.0 / tol)) / xi
    r = ewald_real(x, q, L, xi, rc)
    Ek, phik, Fk = ewald_kspace(x, q, L, xi, tol=tol)
    E = r["E_real"] + Ek + r["E_self"]
    phi = r["phi_real"] + phik + r["phi_self"]
    F = r["F_real"] + Fk
    return E, phi, F


def dft3(re, im, sign):
    """Direct separable 3-D DFT (in place on copies); returns (re, im)."""
    re, im = _f64(re).copy(), _f64(im).copy()
    M = re.shape[0]
    _L().oracle_dft3(_ptr(re), _ptr(im), int(M), int(sign))
    return re, im


def se_spread(x, q, L, M, P, alpha, cg, cell_mode=64):
    x, q = _f64(x), _f64(q)
    H = np.zeros((M, M, M))
    _L().oracle_se_spread(len(q), _ptr(x), _ptr(q), float(L), int(M), int(P),
                          float(alpha), float(cg), int(cell_mode), _ptr(H))
    return H


def se_scale(re, im, L, xi, eta):
    re, im = _f64(re).copy(), _f64(im).copy()
    M = re.shape[0]
    eg = ctypes.c_double()
    _L().oracle_se_scale(_ptr(re), _ptr(im), int(M), float(L), float(xi), float(eta),
                         ctypes.byref(eg))
    return re, im, eg.value


def se_gather(x, q, L, M, P, alpha, cg, Ht, cell_mode=64):
    x, q, Ht = _f64(x), _f64(q), _f64(Ht)
    phi = np.zeros(len(q))
    F = np.zeros((len(q), 3))
    _L().oracle_se_gather(len(q), _ptr(x), _ptr(q), float(L), int(M), int(P),
                          float(alpha), float(cg), int(cell_mode), _ptr(Ht),
                          _ptr(phi), _ptr(F))
    return phi, F


def se_kspace(x, q, L, xi, M, P, c=0.95, eta=None, cell_mode=64, grids=False):
    """O2: the SE k-space evaluation.

    Returns dict(E, phi, F, E_grid[, H, Ht]).  cell_mode=32 takes the wrap and
    cell-index decisions in single precision (to match a float32 GPU path)."""
    x, q = _f64(x), _f64(q)
    N = len(q)
    phi = np.zeros(N)
    F = np.zeros((N, 3))
    E = ctypes.c_double()
    Eg = ctypes.c_double()
    H = np.zeros((M, M, M)) if grids else None
    Ht = np.zeros((M, M, M)) if grids else None
    rc = _L().oracle_se_kspace(N, _ptr(x), _ptr(q), float(L), float(xi), int(M),
                               int(P), float(c), float(eta) if eta else 0.0,
                               int(cell_mode), ctypes.byref(E), _ptr(phi), _ptr(F),
                               _ptr(H) if grids else None, _ptr(Ht) if grids else None,
                               ctypes.byref(Eg))
    if rc:
        raise MemoryError("oracle_se_kspace")
    out = dict(E=E.value, phi=phi, F=F, E_grid=Eg.value)
    if grids:
        out["H"] = H
        out["Ht"] = Ht
    return out


def spectral_derivative(re, im, L, axis):
    """Full spectrum times i k_axis (0 at the Nyquist index); returns (re, im)."""
    re, im = _f64(re).copy(), _f64(im).copy()
    M = re.shape[0]
    _L().oracle_spectral_derivative(_ptr(re), _ptr(im), int(M), float(L), int(axis))
    return re, im


def se_kspace_ik(x, q, L, xi, M, P, c=0.95, eta=None, cell_mode=64):
    """O2 with forces by ik differentiation (Sec. 2.3).  Returns dict(E, phi, F)."""
    x, q = _f64(x), _f64(q)
    N = len(q)
    phi = np.zeros(N)
    F = np.zeros((N, 3))
    E = ctypes.c_double()
    rc = _L().oracle_se_kspace_ik(N, _ptr(x), _ptr(q), float(L), float(xi), int(M), int(P),
                                  float(c), float(eta) if eta else 0.0, int(cell_mode),
                                  ctypes.byref(E), _ptr(phi), _ptr(F))
    if rc:
        raise MemoryError("oracle_se_kspace_ik")
    return dict(E=E.value, phi=phi, F=F)
