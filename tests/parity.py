"""Comparison of GPU results with the oracle, element by element.

Every parity assertion of the GPU tests goes through `assert_close`, which
checks two things:

* normwise: ||got - ref|| / ||ref|| <= tol over the whole array;
* elementwise: for every element i, |got_i - ref_i| <= tol * s_i, with a
  per-element scale s_i = |ref_i| + floor_i.

For rows of vectors (forces [N, 3]) |.| is the row's Euclidean norm.  The
floor is the array's rms magnitude, except for forces with charges given:
there floor_i = |q_i| * E_rms, E_rms the rms field magnitude |F*_j| / |q_j|
over the charged particles.  The reasoning: the errors of the pipeline are
rounding errors of the grids (fixed-point spread, transforms, scaling),
spread evenly over the box at a relative level of the grid's rms, so a
particle's force error is about |q_i| times a field error that does not
depend on the particle, and its potential error is about a potential error
that does not depend on the particle.  A particle with a small force or
potential is therefore held to an absolute bound of the size of the
typical one, a particle with a large one to a relative bound, and a single
particle that is wrong by a fraction f of a typical force fails as soon as
f > 2 tol, whatever N is (normwise alone lets one wrong particle through
when f < tol sqrt(N)).

With SE_PARITY_LOG=<file> every comparison appends its two measured ratios
(normwise, worst element / tol scale) as one JSON line: the record from
which the tolerances of the tests were calibrated.
"""
import json
import math
import os

import numpy as np


def _rows(a):
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 2 and a.shape[1] == 3:
        return np.sqrt((a ** 2).sum(axis=1)), a
    return np.abs(a).ravel(), a.ravel()


def measure(got, ref, q=None):
    """(normwise relative error, max over elements of |got_i - ref_i| / s_i,
    index of that element)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if got.shape != ref.shape:
        raise AssertionError("shape %s against %s" % (got.shape, ref.shape))
    if ref.size == 0:
        return 0.0, 0.0, -1
    dn, _ = _rows(got - ref)
    rn, _ = _rows(ref)
    norm = math.sqrt(float((dn ** 2).sum()))
    rnorm = math.sqrt(float((rn ** 2).sum()))
    nw = norm / rnorm if rnorm > 0 else norm
    if q is not None and ref.ndim == 2:
        qa = np.abs(np.asarray(q, dtype=np.float64).ravel())
        if qa.shape[0] != rn.shape[0]:
            raise AssertionError("q has %d entries for %d rows" % (qa.shape[0], rn.shape[0]))
        charged = qa > 0
        e_rms = math.sqrt(float(((rn[charged] / qa[charged]) ** 2).mean())) if charged.any() else 0.0
        floor = qa * e_rms
        if not (floor > 0).all():   # uncharged particles: the rms force
            floor = np.where(floor > 0, floor, math.sqrt(float((rn ** 2).mean())))
    else:
        floor = math.sqrt(float((rn ** 2).mean()))
    scale = rn + floor
    with np.errstate(divide="ignore", invalid="ignore"):
        ratio = np.where(scale > 0, dn / scale, np.where(dn > 0, np.inf, 0.0))
    i = int(np.argmax(ratio))
    return nw, float(ratio[i]), i


def normwise(got, ref):
    """||got - ref|| / ||ref|| over the whole array: the form of an rms error
    statement (a workload's relative rms force error against the direct
    Ewald sum), not a parity check."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    n = math.sqrt(float((ref ** 2).sum()))
    d = math.sqrt(float(((got - ref) ** 2).sum()))
    return d / n if n > 0 else d


def assert_close(got, ref, tol, q=None, label=""):
    """Assert normwise and elementwise agreement within tol (see module doc);
    returns (normwise, elementwise) for further checks."""
    nw, elem, i = measure(got, ref, q)
    path = os.environ.get("SE_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"test": os.environ.get("PYTEST_CURRENT_TEST", ""), "label": label,
                                "tol": tol, "normwise": nw, "elementwise": elem}) + "\n")
    assert nw <= tol, "%s: normwise %.3g > %.3g" % (label, nw, tol)
    assert elem <= tol, "%s: element %d off by %.3g of its scale > %.3g" % (label, i, elem, tol)
    return nw, elem
