"""Host-side pins of the real-space kernel's single-precision erfc: the
coefficient table embedded in se_real.cu, evaluated as the kernel does (in
float32), against the scaled complementary error function erfcx(x) =
erfc(x) e^{x^2} of scipy."""
import os
import re

import numpy as np
import pytest

scipy_special = pytest.importorskip("scipy.special")

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_1712_04718_gb300", "csrc", "se_real.cu")


def _table():
    s = open(SRC).read()
    p = float(re.search(r"kErfcxP = ([-0-9.e+]+)f;", s).group(1))
    body = re.search(r"kErfcx\[9\] = \{(.*?)\};", s, re.S).group(1)
    c = [float(v.strip().rstrip("f")) for v in body.split(",")]
    return np.float32(p), np.asarray(c, dtype=np.float32)


def _eval_f32(x, p, c):
    x = np.asarray(x, dtype=np.float32)
    t = (np.float32(1) / (p * x + np.float32(1))).astype(np.float32)
    a = np.full_like(t, c[-1])
    for k in range(len(c) - 2, -1, -1):
        a = (a * t + c[k]).astype(np.float32)
    return (a * t).astype(np.float64)


def test_erfcx_table_relative_accuracy():
    p, c = _table()
    assert len(c) == 9
    x = np.linspace(0.0, 6.0, 120001)
    ref = scipy_special.erfcx(x)
    assert np.max(np.abs(_eval_f32(x, p, c) / ref - 1.0)) < 1e-6
    # beyond x = 6 erfc(x) < 2e-17: a looser relative bound suffices
    x = np.linspace(6.0, 12.0, 6001)
    assert np.max(np.abs(_eval_f32(x, p, c) / scipy_special.erfcx(x) - 1.0)) < 1e-4
    # erfc itself, as the kernel forms it, against scipy's erfc (relative)
    x = np.linspace(0.0, 4.5, 4501)
    erfc = _eval_f32(x, p, c) * np.exp(-x * x)
    assert np.max(np.abs(erfc / scipy_special.erfc(x) - 1.0)) < 2e-6
