// se_select.cu -- choice of the Ewald and SE parameters for an error
// tolerance (host code only).
//
// arXiv:1712.04718, Sec. 2 and Sec. 4:
//  * xi from the real-space truncation estimates of Kolafa and Perram for a
//    cut-off r_c (Eq. 2.3): the potential and energy forms through the
//    principal branch W0 of the Lambert function, the force form through a
//    logarithm;
//  * k_inf from the Fourier-space truncation estimates (Eq. 2.4), again
//    through W0, and M = 2 k_inf (Sec. 3, the grid resolving modes up to
//    k_inf);
//  * P from the approximation-error bounds A e^{-pi P c^2 / 2} (Sec. 4:
//    A_phi = sqrt(Q xi L) / L, A_E = Q sqrt(xi L) / L, A_F = 4 pi Q
//    sqrt(xi^3 / L)), rounded up to the next even integer as the force
//    bound's discussion prescribes; eta then follows from Eq. 4.2 inside the
//    plan.  The bounds were established on grids of about 4 xi L points
//    (eta = P / (16 pi c^2)); M is raised where needed so that eta <= 1/2.
// The paper defines W as the inverse of x e^{-x}; the estimates it inverts
// give w e^{w} = z, so W here is the standard W0 (the inverse of x e^{x}).
#include <math.h>

#include "../../include/se.h"

namespace {

constexpr double kPi = 3.14159265358979323846;

// W0(z) for z >= 0: the w >= 0 with w e^w = z.  Halley's iteration on
// f(w) = w e^w - z (Corless, Gonnet, Hare, Jeffrey, Knuth, "On the Lambert W
// function", Adv. Comput. Math. 5, 1996, Sec. 5), started from the first
// terms of the series at 0 (z < 1) or of the asymptotic expansion ln z -
// ln ln z (z >= 1); at most 64 steps.
double lambert_w0(double z) {
    if (!(z >= 0.0) || !isfinite(z)) return NAN;
    if (z == 0.0) return 0.0;
    double w;
    if (z < 1.0) {
        w = z * (1.0 - z + 1.5 * z * z);
        if (w <= 0.0) w = 0.5 * z;
    } else {
        w = log(z);
        if (w > 1.0) w -= log(w);
    }
    for (int it = 0; it < 64; ++it) {
        const double ew = exp(w);
        const double f = w * ew - z;
        const double d1 = ew * (w + 1.0);
        const double step = f / (d1 - (w + 2.0) * f / (2.0 * w + 2.0));
        w -= step;
        if (fabs(step) <= 1e-15 * (1.0 + fabs(w))) break;
    }
    return w;
}

// W0(e^lz) for any real lz, so that arguments beyond the double range can
// be given by their logarithm: below lz = 700 as lambert_w0(e^lz), above it
// Newton's iteration on g(w) = w + ln w - lz (the logarithm of w e^w = e^lz)
// from w = lz - ln lz; at most 64 steps.
double lambert_w0_of_log(double lz) {
    if (!(lz == lz)) return NAN;
    if (lz < 700.0) return lambert_w0(exp(lz));
    double w = lz - log(lz);
    for (int it = 0; it < 64; ++it) {
        const double step = (w + log(w) - lz) / (1.0 + 1.0 / w);
        w -= step;
        if (fabs(step) <= 1e-15 * w) break;
    }
    return w;
}

bool pos(double v) { return v > 0.0 && isfinite(v); }

}  // namespace

extern "C" double se_lambert_w0(double z) { return lambert_w0(z); }

extern "C" int se_select_support(double scaled_tol, double c) {
    if (!pos(scaled_tol) || !(c >= 0.0) || !isfinite(c)) return SE_ERR_ARG;
    if (c == 0.0) c = 0.95;
    if (scaled_tol >= 1.0) return 2;
    const double Preal = 2.0 * log(1.0 / scaled_tol) / (kPi * c * c);
    if (Preal > 1e6) return SE_ERR_UNSUPPORTED;
    const int P = 2 * (int)ceil(Preal / 2.0);
    return P < 2 ? 2 : P;
}

extern "C" int se_select_params(int quantity, double tol, double rc, double L, double Q,
                                double c, double* xi_out, int* M_out, int* P_out,
                                double* kinf_out) {
    if (quantity < SE_QUANTITY_POTENTIAL || quantity > SE_QUANTITY_FORCE || !pos(tol) ||
        !pos(rc) || !pos(L) || !pos(Q) || !(c >= 0.0) || !xi_out || !M_out || !P_out)
        return SE_ERR_ARG;
    if (c == 0.0) c = 0.95;
    const double L3 = L * L * L;
    // Eq. 2.3: xi r_c = sqrt(W0(...)) (potential, energy) or sqrt(log(...)) (force)
    double u;
    if (quantity == SE_QUANTITY_POTENTIAL)
        u = lambert_w0(sqrt(Q * rc / (2.0 * L3)) / tol);
    else if (quantity == SE_QUANTITY_ENERGY)
        u = lambert_w0(Q * sqrt(rc / (2.0 * L3)) / tol);
    else
        u = log(2.0 * Q / tol * sqrt(1.0 / (rc * L3)));
    if (!(u > 0.0)) return SE_ERR_UNSUPPORTED;   // tolerance met without a Fourier part
    const double xi = sqrt(u) / rc;
    // Eq. 2.4: k_inf, the W0 arguments given by their logarithms
    double kinf;
    if (quantity == SE_QUANTITY_POTENTIAL)
        kinf = sqrt(3.0) * L * xi / (2.0 * kPi) *
               sqrt(lambert_w0_of_log(log(4.0 / (3.0 * L * L)) +
                                      2.0 / 3.0 * (log(Q / (kPi * xi)) - 2.0 * log(tol))));
    else if (quantity == SE_QUANTITY_ENERGY)
        kinf = sqrt(3.0) * L * xi / (2.0 * kPi) *
               sqrt(lambert_w0_of_log(log(4.0 / (3.0 * L * L)) +
                                      2.0 / 3.0 * (2.0 * log(Q) - log(kPi * xi) - 2.0 * log(tol))));
    else
        kinf = L * xi / (2.0 * kPi) *
               sqrt(lambert_w0_of_log(log(256.0 * xi * xi / (kPi * kPi)) + 4.0 * log(Q / tol) -
                                      6.0 * log(L)));
    if (!pos(kinf) || kinf > 1e6) return SE_ERR_UNSUPPORTED;
    int M = 2 * (int)ceil(kinf);
    // Sec. 4: A e^{-pi P c^2 / 2} <= tol, P rounded up to even
    double A;
    if (quantity == SE_QUANTITY_POTENTIAL)
        A = sqrt(Q * xi * L) / L;
    else if (quantity == SE_QUANTITY_ENERGY)
        A = Q * sqrt(xi * L) / L;
    else
        A = 4.0 * kPi * Q * sqrt(xi * xi * xi / L);
    const int P = se_select_support(tol / A, c);
    if (P < 0) return P;
    // the bounds hold for a moderate Gaussian width: eta = P L^2 xi^2 /
    // (c^2 pi M^2) (Eq. 4.2) at most 1/2, so M is raised to L xi sqrt(2 P /
    // (pi c^2)) where the truncation rule gives less (near eta = 1 the
    // approximation error grows far beyond the bound)
    const double Meta = L * xi * sqrt(2.0 * P / (kPi * c * c));
    if (Meta > 2e6) return SE_ERR_UNSUPPORTED;
    if (M < Meta) M = (int)ceil(Meta);
    if (M < P) M = P;
    M += M & 1;
    *xi_out = xi;
    *M_out = M;
    *P_out = P;
    if (kinf_out) *kinf_out = kinf;
    return P > 32 ? SE_ERR_UNSUPPORTED : SE_OK;
}
