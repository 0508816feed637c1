"""Writes the coefficients of the single-precision erfcx fit used by the
real-space kernel (se_real.cu): erfcx(x) = erfc(x) e^{x^2} ~ t P(t) with
t = 1 / (1 + p x), P a polynomial of degree 8 -- the form of Hastings'
approximations (Abramowitz and Stegun 7.1.26), with coefficients fitted here
for relative accuracy on 0 <= x <= 6 by Lawson's iteratively reweighted
least squares (which tends to the minimax fit) against scipy's erfcx.

Run: python gen_erfcx_fit.py   (prints the C table to paste into se_real.cu)
"""
import numpy as np
from scipy.special import erfcx

P_PARAM = 0.45
TERMS = 9
X_MAX = 6.0


def fit(p=P_PARAM, n=TERMS, xmax=X_MAX, iters=60, m=4000):
    tmin = 1.0 / (1.0 + p * xmax)
    t = np.cos(np.pi * (np.arange(m) + 0.5) / m) * (1.0 - tmin) / 2 + (1.0 + tmin) / 2
    x = (1.0 / t - 1.0) / p
    g = erfcx(x) / t
    V = np.vander(t, n, increasing=True)
    w = np.ones(m)
    for _ in range(iters):
        W = np.sqrt(w) / g
        c, *_ = np.linalg.lstsq(V * W[:, None], g * W, rcond=None)
        e = np.abs(V @ c / g - 1.0)
        w = w * e
        w /= w.sum()
    return c


def evaluate_f32(c, x, p=P_PARAM):
    """The kernel's evaluation, in float32: t by one rounded division, Horner."""
    x = np.asarray(x, dtype=np.float32)
    c32 = np.asarray(c, dtype=np.float32)
    t = (np.float32(1) / (np.float32(1) + np.float32(p) * x)).astype(np.float32)
    acc = np.full_like(t, c32[-1])
    for k in range(len(c32) - 2, -1, -1):
        acc = (acc * t + c32[k]).astype(np.float32)
    return (acc * t).astype(np.float32)


if __name__ == "__main__":
    c = fit()
    xs = np.linspace(0.0, X_MAX, 200001)
    err = np.max(np.abs(evaluate_f32(c, xs).astype(np.float64) / erfcx(xs) - 1.0))
    print("// max relative error on [0, %g] in float32: %.2e" % (X_MAX, err))
    print("constexpr float kErfcxP = %.8ef;" % P_PARAM)
    print("constexpr float kErfcx[%d] = {" % TERMS)
    print(",\n".join("    %.9ef" % float(np.float32(v)) for v in c) + "};")
