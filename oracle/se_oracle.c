/*
 * se_oracle.c -- FP64 CPU oracle for the Spectral Ewald (SE) k-space path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library, its
 * Python binding, the autograd layer) may include, link or call this file.
 * It is loaded by the tests, by __graft_entry__.smoke() and by the
 * cpu_baseline leg of bench.py, and by nothing else.  It shares no code,
 * headers, tables or constants with the CUDA path.
 *
 * Paper: D. Saffar Shamshirgar, B. Hess, A.-K. Tornberg, "A comparison of
 * the Spectral Ewald and Smooth Particle Mesh Ewald methods in GROMACS"
 * (arXiv:1712.04718).
 *
 * Two oracles live here, both plain and slow on purpose:
 *
 *   O1  the classic Ewald sum (Sec. 1, Eq. 1.5-1.7): the k-space part by a
 *       direct sum over wave vectors, the real-space part by an explicit
 *       image sum, and the self term.  This is the exact quantity that SE
 *       approximates.
 *
 *   O2  the SE k-space method itself (Sec. 3, Eq. 3.5-3.13), step by step in
 *       the paper's order: spread with the truncated Gaussian (direct exp at
 *       every support point, no fast Gaussian gridding), forward DFT (direct,
 *       separable, FP64 twiddles), scaling by the modified Green's function
 *       (Eq. 3.6), inverse DFT, and gather of potential and force with the
 *       same Gaussian (Eq. 3.9, 3.13).
 *       With forces by ik differentiation (Sec. 2.3) instead, the scaled
 *       spectrum is also multiplied by i k_d and transformed back per axis,
 *       and the gather applies the plain window to those derivative grids.
 *
 * Readings of the paper taken here (each also listed in the design notes):
 *  - Force = -dE/dx exactly (Eq. 1.3 first equality).  Eq. 1.7 and 3.13 carry
 *    an extra factor 1/2 and Eq. 3.13 the opposite sign; the derivative of
 *    the energy is what both oracles return.
 *  - Discrete SE normalisation: unnormalised forward DFT (e^{-i}), scaling
 *    by G(k)/M^3, unnormalised inverse DFT (e^{+i}); phi = h^3 sum_j Ht_j W.
 *  - Support: for even P the P points per dimension are
 *    i0 .. i0+P-1 with i0 = floor(x/h) - P/2 + 1 (tensor-product box).
 *  - eta = P L^2 xi^2 / (c^2 pi M^2) with c = 0.95 unless given (Eq. 4.2).
 *  - Positions inside [0, L) are used as given; others are wrapped with
 *    x - L floor(x/L) (reciprocal of L rounded once), corrected once by L, and
 *    set to 0 if still outside.  The cell index is floor(x M/L) (M/L rounded
 *    once), clamped to M-1.
 *    When the oracle is compared with a single-precision GPU path, the
 *    wrap and the cell index are decided in single precision with the same
 *    operations as there (cell_mode = 32); all arithmetic after that integer
 *    decision is FP64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <float.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* Periodic wrap and cell index (reading: see header).                       */
/* ------------------------------------------------------------------------ */

/* Double-precision wrap: untouched inside [0, L); otherwise x - L floor(x/L)
 * with the reciprocal 1/L rounded once, each operation rounded (this file is
 * compiled with -ffp-contract=off), then one correction by L either way;
 * anything still outside becomes 0. */
static double wrap64(double x, double L, double invL)
{
    if (x >= 0.0 && x < L) return x;
    double s = x * invL;
    double f = floor(s);
    double p = f * L;
    double w = x - p;
    if (w >= L) w = w - L;
    if (w < 0.0) w = w + L;
    if (!(w >= 0.0 && w < L)) w = 0.0;
    return w;
}

/* Single-precision decision, operation for operation: one multiply by the
 * rounded 1/L, floor, one multiply by L, one subtract, each rounded to
 * float (this file is compiled with -ffp-contract=off). */
static float wrap32(float x, float L, float invL)
{
    if (x >= 0.0f && x < L) return x;
    float s = x * invL;
    float f = floorf(s);
    float p = f * L;
    float w = x - p;
    if (w >= L) w = w - L;
    if (w < 0.0f) w = w + L;
    if (!(w >= 0.0f && w < L)) w = 0.0f;
    return w;
}

/* Wrapped position (FP64) and cell index of one coordinate. */
static void wrap_and_cell(double x, double L, int M, int cell_mode,
                          double *xw, int *cell)
{
    int c;
    if (cell_mode == 32) {
        float Lf = (float)L;
        float invLf = (float)(1.0 / L);
        float invhf = (float)((double)M / L);
        float wf = wrap32((float)x, Lf, invLf);
        float s = wf * invhf;
        c = (int)floorf(s);
        *xw = (double)wf;
    } else {
        double w = wrap64(x, L, 1.0 / L);
        double invh = (double)M / L;
        c = (int)floor(w * invh);
        *xw = w;
    }
    if (c >= M) c = M - 1;
    if (c < 0) c = 0;
    *cell = c;
}

/* ------------------------------------------------------------------------ */
/* O1: classic Ewald sum, Eq. 1.5-1.7.                                       */
/* ------------------------------------------------------------------------ */

/*
 * k-space part (superscript L in Eq. 1.5-1.7).  All k = 2 pi n / L with
 * 0 < |n|^2 <= nmax^2 are summed; n and -n give complex-conjugate terms, so
 * the sums run over the half space (nx > 0, or nx = 0 and ny > 0, or
 * nx = ny = 0 and nz > 0) with weight 2:
 *   S(k)     = sum_n q_n e^{i k.x_n}
 *   f(k)     = e^{-k^2/(4 xi^2)} / k^2
 *   E^L      = (2 pi / L^3) sum_{k!=0} f |S|^2
 *   phi^L_m  = (4 pi / L^3) sum_{k!=0} f Re(e^{i k.x_m} conj(S))
 *   F^L_m    = -dE^L/dx_m = (4 pi q_m / L^3) sum_{k!=0} f k Im(e^{i k.x_m} conj(S))
 * (The last line is the derivative of the energy; Eq. 1.7 prints half of it.)
 */

/* Index of half-cube storage: nx in [0, nmax], ny, nz in [-nmax, nmax]. */
static size_t sidx(int nx, int ny, int nz, int nmax)
{
    const size_t W = (size_t)(2 * nmax + 1);
    return ((size_t)nx * W + (size_t)(ny + nmax)) * W + (size_t)(nz + nmax);
}

static int in_half_sphere(int nx, int ny, int nz, int nmax)
{
    int n2 = nx * nx + ny * ny + nz * nz;
    if (n2 == 0 || n2 > nmax * nmax) return 0;
    if (nx == 0 && (ny < 0 || (ny == 0 && nz < 0))) return 0;
    return 1;
}

/* e^{i 2 pi n x / L}, n in [-nmax, nmax], of one coordinate, by direct cos/sin. */
static void phase_row(double x, double L, int nmax, double *re, double *im)
{
    for (int n = -nmax; n <= nmax; ++n) {
        double a = 2.0 * M_PI * n * x / L;
        re[n + nmax] = cos(a);
        im[n + nmax] = sin(a);
    }
}

/* Structure factor S(k) over the half cube (zero outside the half sphere).
 * Sr, Si have (nmax+1)(2nmax+1)^2 entries.  Returns -1 on allocation failure. */
int oracle_ewald_structure(int64_t N, const double *x, const double *q,
                           double L, int nmax, double *Sr, double *Si)
{
    const int W = 2 * nmax + 1;
    const size_t S = (size_t)(nmax + 1) * W * W;
    memset(Sr, 0, sizeof(double) * S);
    memset(Si, 0, sizeof(double) * S);
    const int64_t CH = 2048;
    double *tr = (double *)malloc(sizeof(double) * (size_t)CH * 3 * W);
    double *ti = (double *)malloc(sizeof(double) * (size_t)CH * 3 * W);
    if (!tr || !ti) { free(tr); free(ti); return -1; }
    for (int64_t c0 = 0; c0 < N; c0 += CH) {
        int64_t cn = (N - c0 < CH) ? N - c0 : CH;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < cn; ++i)
            for (int d = 0; d < 3; ++d)
                phase_row(x[3 * (c0 + i) + d], L, nmax,
                          tr + ((size_t)i * 3 + d) * W, ti + ((size_t)i * 3 + d) * W);
        /* each (nx, ny) column is owned by one thread: no write conflicts */
#pragma omp parallel for schedule(dynamic, 1)
        for (int col = 0; col < (nmax + 1) * W; ++col) {
            int nx = col / W, ny = col % W - nmax;
            if (nx * nx + ny * ny > nmax * nmax) continue;
            int nzmax = (int)floor(sqrt((double)(nmax * nmax - nx * nx - ny * ny)));
            for (int64_t i = 0; i < cn; ++i) {
                const double *xr = tr + (size_t)i * 3 * W, *xi_ = ti + (size_t)i * 3 * W;
                double ar = xr[nx + nmax], ai = xi_[nx + nmax];
                double br = xr[W + ny + nmax], bi = xi_[W + ny + nmax];
                double qq = q[c0 + i];
                double pr = qq * (ar * br - ai * bi), pim = qq * (ar * bi + ai * br);
                for (int nz = -nzmax; nz <= nzmax; ++nz) {
                    double zr = xr[2 * W + nz + nmax], zi = xi_[2 * W + nz + nmax];
                    size_t k = sidx(nx, ny, nz, nmax);
                    Sr[k] += pr * zr - pim * zi;
                    Si[k] += pr * zi + pim * zr;
                }
            }
        }
    }
    free(tr); free(ti);
    return 0;
}

/* E^L from the structure factor. */
double oracle_ewald_energy(const double *Sr, const double *Si, double L, double xi, int nmax)
{
    const double t = 2.0 * M_PI / L;
    double e = 0.0;
    for (int nx = 0; nx <= nmax; ++nx)
        for (int ny = -nmax; ny <= nmax; ++ny)
            for (int nz = -nmax; nz <= nmax; ++nz) {
                if (!in_half_sphere(nx, ny, nz, nmax)) continue;
                double k2 = t * t * ((double)nx * nx + (double)ny * ny + (double)nz * nz);
                double f = exp(-k2 / (4.0 * xi * xi)) / k2;
                size_t i = sidx(nx, ny, nz, nmax);
                e += 2.0 * f * (Sr[i] * Sr[i] + Si[i] * Si[i]);
            }
    return 2.0 * M_PI / (L * L * L) * e;
}

/* phi^L and F^L at T target positions xt (charges qt) from the structure factor. */
void oracle_ewald_eval(int64_t T, const double *xt, const double *qt,
                       const double *Sr, const double *Si,
                       double L, double xi, int nmax, double *phi, double *F)
{
    const int W = 2 * nmax + 1;
    const double t = 2.0 * M_PI / L;
    const double V = L * L * L;
#pragma omp parallel
    {
        double *er = (double *)malloc(sizeof(double) * 3 * W);
        double *ei = (double *)malloc(sizeof(double) * 3 * W);
#pragma omp for schedule(dynamic, 4)
        for (int64_t m = 0; m < T; ++m) {
            for (int d = 0; d < 3; ++d)
                phase_row(xt[3 * m + d], L, nmax, er + d * W, ei + d * W);
            double ph = 0.0, fx = 0.0, fy = 0.0, fz = 0.0;
            for (int nx = 0; nx <= nmax; ++nx)
                for (int ny = -nmax; ny <= nmax; ++ny) {
                    if (nx * nx + ny * ny > nmax * nmax) continue;
                    double ar = er[nx + nmax], ai = ei[nx + nmax];
                    double br = er[W + ny + nmax], bi = ei[W + ny + nmax];
                    double pr = ar * br - ai * bi, pim = ar * bi + ai * br;
                    for (int nz = -nmax; nz <= nmax; ++nz) {
                        if (!in_half_sphere(nx, ny, nz, nmax)) continue;
                        double k2 = t * t * ((double)nx * nx + (double)ny * ny + (double)nz * nz);
                        double f = exp(-k2 / (4.0 * xi * xi)) / k2;
                        double zr = er[2 * W + nz + nmax], zi = ei[2 * W + nz + nmax];
                        double gr = pr * zr - pim * zi, gi = pr * zi + pim * zr; /* e^{i k.x_m} */
                        size_t i = sidx(nx, ny, nz, nmax);
                        double re = gr * Sr[i] + gi * Si[i];   /* Re(e^{ik.x} conj S) */
                        double imv = gi * Sr[i] - gr * Si[i];  /* Im(e^{ik.x} conj S) */
                        ph += 2.0 * f * re;
                        fx += 2.0 * f * t * nx * imv;
                        fy += 2.0 * f * t * ny * imv;
                        fz += 2.0 * f * t * nz * imv;
                    }
                }
            phi[m] = 4.0 * M_PI / V * ph;
            F[3 * m] = 4.0 * M_PI * qt[m] / V * fx;
            F[3 * m + 1] = 4.0 * M_PI * qt[m] / V * fy;
            F[3 * m + 2] = 4.0 * M_PI * qt[m] / V * fz;
        }
        free(er); free(ei);
    }
}

/* All of the above for every particle.  Returns -1 on allocation failure. */
int oracle_ewald_kspace(int64_t N, const double *x, const double *q,
                        double L, double xi, int nmax,
                        double *E, double *phi, double *F)
{
    const int W = 2 * nmax + 1;
    const size_t S = (size_t)(nmax + 1) * W * W;
    double *Sr = (double *)malloc(sizeof(double) * S);
    double *Si = (double *)malloc(sizeof(double) * S);
    if (!Sr || !Si) { free(Sr); free(Si); return -1; }
    if (oracle_ewald_structure(N, x, q, L, nmax, Sr, Si)) { free(Sr); free(Si); return -1; }
    *E = oracle_ewald_energy(Sr, Si, L, xi, nmax);
    oracle_ewald_eval(N, x, q, Sr, Si, L, xi, nmax, phi, F);
    free(Sr); free(Si);
    return 0;
}

/*
 * Real-space part (superscript S in Eq. 1.5-1.7) by an explicit image sum
 * over every p in Z^3 with |x_m - x_n + p L| <= rc (the m == n, p == 0 term
 * excluded), and the self term -2 xi / sqrt(pi) q_m (Eq. 1.5).
 *   phi^S_m = sum_n sum'_p q_n erfc(xi r) / r
 *   F^S_m   = q_m sum_n sum'_p q_n (2 xi/sqrt(pi) e^{-xi^2 r^2} + erfc(xi r)/r) r_vec / r^2
 *   E^S     = 1/2 sum_m q_m phi^S_m,  E^self = -xi/sqrt(pi) sum_m q_m^2
 * phi and F receive the real-space part; phi_self receives the self term.
 */
/* The real-space potential and force of oracle_ewald_real at T target
 * particles idx[t] only (same images, same cut-off, same terms; the self
 * term not included): for checks of large systems on a sample. */
void oracle_ewald_real_at(int64_t N, const double *x, const double *q,
                          double L, double xi, double rc, int64_t T,
                          const int64_t *idx, double *phi, double *F)
{
    const int pmax = (int)ceil(rc / L) + 1;
    const double twoxi_sqrtpi = 2.0 * xi / sqrt(M_PI);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < T; ++t) {
        const int64_t m = idx[t];
        double ph = 0.0, fx = 0.0, fy = 0.0, fz = 0.0;
        for (int64_t n = 0; n < N; ++n)
            for (int px = -pmax; px <= pmax; ++px)
                for (int py = -pmax; py <= pmax; ++py)
                    for (int pz = -pmax; pz <= pmax; ++pz) {
                        if (n == m && px == 0 && py == 0 && pz == 0) continue;
                        double dx = x[3 * m] - x[3 * n] + px * L;
                        double dy = x[3 * m + 1] - x[3 * n + 1] + py * L;
                        double dz = x[3 * m + 2] - x[3 * n + 2] + pz * L;
                        double r2 = dx * dx + dy * dy + dz * dz;
                        if (r2 > rc * rc) continue;
                        double r = sqrt(r2);
                        double ec = erfc(xi * r) / r;
                        ph += q[n] * ec;
                        double s = q[n] * (twoxi_sqrtpi * exp(-xi * xi * r2) + ec) / r2;
                        fx += s * dx; fy += s * dy; fz += s * dz;
                    }
        phi[t] = ph;
        F[3 * t] = q[m] * fx; F[3 * t + 1] = q[m] * fy; F[3 * t + 2] = q[m] * fz;
    }
}

void oracle_ewald_real(int64_t N, const double *x, const double *q,
                       double L, double xi, double rc,
                       double *E_real, double *E_self,
                       double *phi, double *phi_self, double *F)
{
    const int pmax = (int)ceil(rc / L) + 1;
    const double twoxi_sqrtpi = 2.0 * xi / sqrt(M_PI);
    double Er = 0.0, Es = 0.0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : Er)
    for (int64_t m = 0; m < N; ++m) {
        double ph = 0.0, fx = 0.0, fy = 0.0, fz = 0.0;
        for (int64_t n = 0; n < N; ++n)
            for (int px = -pmax; px <= pmax; ++px)
                for (int py = -pmax; py <= pmax; ++py)
                    for (int pz = -pmax; pz <= pmax; ++pz) {
                        if (n == m && px == 0 && py == 0 && pz == 0) continue;
                        double dx = x[3 * m] - x[3 * n] + px * L;
                        double dy = x[3 * m + 1] - x[3 * n + 1] + py * L;
                        double dz = x[3 * m + 2] - x[3 * n + 2] + pz * L;
                        double r2 = dx * dx + dy * dy + dz * dz;
                        if (r2 > rc * rc) continue;
                        double r = sqrt(r2);
                        double ec = erfc(xi * r) / r;
                        ph += q[n] * ec;
                        double s = q[n] * (twoxi_sqrtpi * exp(-xi * xi * r2) + ec) / r2;
                        fx += s * dx; fy += s * dy; fz += s * dz;
                    }
        phi[m] = ph;
        F[3 * m] = q[m] * fx; F[3 * m + 1] = q[m] * fy; F[3 * m + 2] = q[m] * fz;
        Er += 0.5 * q[m] * ph;
    }
    for (int64_t m = 0; m < N; ++m) {
        phi_self[m] = -twoxi_sqrtpi * q[m];
        Es += -xi / sqrt(M_PI) * q[m] * q[m];
    }
    *E_real = Er;
    *E_self = Es;
}

/* ------------------------------------------------------------------------ */
/* O2: the SE k-space method, Sec. 3.                                        */
/* ------------------------------------------------------------------------ */

/* Shape parameters (Sec. 3 after Eq. 3.9, and Eq. 4.2).  eta_in > 0 overrides
 * the rule eta = P L^2 xi^2 / (c^2 pi M^2).  out[0..5] = h, w, eta, alpha,
 * c_g, m with alpha = 2 xi^2 / eta and c_g = (2 xi^2 / (pi eta))^{3/2}. */
void oracle_se_params(double L, double xi, int M, int P, double c, double eta_in,
                      double *out)
{
    double h = L / M;
    double w = P * h / 2.0;
    double m = c * sqrt(M_PI * P);
    double eta = (eta_in > 0.0) ? eta_in : (2.0 * w * xi / m) * (2.0 * w * xi / m);
    double alpha = 2.0 * xi * xi / eta;
    double cg = pow(2.0 * xi * xi / (M_PI * eta), 1.5);
    out[0] = h; out[1] = w; out[2] = eta; out[3] = alpha; out[4] = cg; out[5] = m;
}

/* One-dimensional direct DFT along one axis of a complex M^3 array stored
 * (ix, iy, iz) with iz fastest; sign = -1 forward (e^{-i}), +1 inverse.
 * out[k] = sum_j in[j] e^{sign 2 pi i j k / M}; twiddles indexed by (j k) mod M. */
static void dft_axis(double *re, double *im, int M, int axis, int sign)
{
    double *twr = (double *)malloc(sizeof(double) * M);
    double *twi = (double *)malloc(sizeof(double) * M);
    for (int r = 0; r < M; ++r) {
        twr[r] = cos(2.0 * M_PI * r / M);
        twi[r] = sign * sin(2.0 * M_PI * r / M);
    }
    const size_t sx = (size_t)M * M, sy = (size_t)M, sz = 1;
    const size_t stride = axis == 0 ? sx : (axis == 1 ? sy : sz);
#pragma omp parallel
    {
        double *lr = (double *)malloc(sizeof(double) * M);
        double *li = (double *)malloc(sizeof(double) * M);
#pragma omp for schedule(static)
        for (int64_t line = 0; line < (int64_t)M * M; ++line) {
            int u = (int)(line / M), v = (int)(line % M);
            size_t base;
            if (axis == 0) base = (size_t)u * sy + (size_t)v * sz;
            else if (axis == 1) base = (size_t)u * sx + (size_t)v * sz;
            else base = (size_t)u * sx + (size_t)v * sy;
            for (int k = 0; k < M; ++k) {
                double ar = 0.0, ai = 0.0;
                for (int j = 0; j < M; ++j) {
                    int r = (int)(((int64_t)j * k) % M);
                    double xr = re[base + (size_t)j * stride], xi_ = im[base + (size_t)j * stride];
                    ar += xr * twr[r] - xi_ * twi[r];
                    ai += xr * twi[r] + xi_ * twr[r];
                }
                lr[k] = ar; li[k] = ai;
            }
            for (int k = 0; k < M; ++k) {
                re[base + (size_t)k * stride] = lr[k];
                im[base + (size_t)k * stride] = li[k];
            }
        }
        free(lr); free(li);
    }
    free(twr); free(twi);
}

/* 3-D direct DFT (all three axes), in place. */
void oracle_dft3(double *re, double *im, int M, int sign)
{
    dft_axis(re, im, M, 0, sign);
    dft_axis(re, im, M, 1, sign);
    dft_axis(re, im, M, 2, sign);
}

/* Signed wave number of DFT index n on an M-point grid. */
static int signed_index(int n, int M) { return (2 * n <= M) ? n : n - M; }

/* Spread, Eq. 3.5: H_j = sum_n q_n c_g exp(-alpha |x_j - x_n|^2) over the P^3
 * support box of each particle, with periodic grid indices.  H is M^3 real,
 * iz fastest.  Direct exp at every support point. */
void oracle_se_spread(int64_t N, const double *x, const double *q, double L,
                      int M, int P, double alpha, double cg, int cell_mode,
                      double *H)
{
    const double h = L / M;
    memset(H, 0, sizeof(double) * (size_t)M * M * M);
    for (int64_t n = 0; n < N; ++n) {
        double xw[3];
        int i0[3];
        for (int d = 0; d < 3; ++d) {
            int c;
            wrap_and_cell(x[3 * n + d], L, M, cell_mode, &xw[d], &c);
            i0[d] = c - P / 2 + 1;
        }
        for (int a = 0; a < P; ++a) {
            double dx = (i0[0] + a) * h - xw[0];
            int jx = ((i0[0] + a) % M + M) % M;
            for (int b = 0; b < P; ++b) {
                double dy = (i0[1] + b) * h - xw[1];
                int jy = ((i0[1] + b) % M + M) % M;
                for (int c = 0; c < P; ++c) {
                    double dz = (i0[2] + c) * h - xw[2];
                    int jz = ((i0[2] + c) % M + M) % M;
                    double r2 = dx * dx + dy * dy + dz * dz;
                    H[((size_t)jx * M + jy) * M + jz] += q[n] * cg * exp(-alpha * r2);
                }
            }
        }
    }
}

/* Modified Green's function of Eq. 3.6 with the 4 pi of Eq. 3.7:
 * G(k) = 4 pi e^{-(1-eta) k^2 / (4 xi^2)} / k^2, G(0) = 0. */
static double green(int nx, int ny, int nz, int M, double L, double xi, double eta)
{
    int sx = signed_index(nx, M), sy = signed_index(ny, M), sz = signed_index(nz, M);
    if (sx == 0 && sy == 0 && sz == 0) return 0.0;
    double t = 2.0 * M_PI / L;
    double k2 = t * t * ((double)sx * sx + (double)sy * sy + (double)sz * sz);
    return 4.0 * M_PI * exp(-(1.0 - eta) * k2 / (4.0 * xi * xi)) / k2;
}

/* Scale step (Eq. 3.6) between the two transforms: Hhat <- G/M^3 Hhat,
 * and the grid energy E_grid = h^3/(2 M^3) sum_k G |DFT(H)_k|^2. */
void oracle_se_scale(double *re, double *im, int M, double L, double xi,
                     double eta, double *E_grid)
{
    const double M3 = (double)M * M * M;
    const double h = L / M;
    double e = 0.0;
    for (int nx = 0; nx < M; ++nx)
        for (int ny = 0; ny < M; ++ny)
            for (int nz = 0; nz < M; ++nz) {
                size_t i = ((size_t)nx * M + ny) * M + nz;
                double G = green(nx, ny, nz, M, L, xi, eta);
                e += G * (re[i] * re[i] + im[i] * im[i]);
                re[i] *= G / M3;
                im[i] *= G / M3;
            }
    *E_grid = h * h * h / (2.0 * M3) * e;
}

/* Gather, Eq. 3.9 and the derivative of the energy (reading of Eq. 3.13):
 *   phi_m = h^3 sum_j Ht_j c_g exp(-alpha |x_j - x_m|^2)
 *   F_m   = -2 alpha h^3 q_m sum_j (x_j - x_m) Ht_j c_g exp(-alpha |x_j - x_m|^2)
 * with x_j - x_m the unwrapped offset inside the support box. */
void oracle_se_gather(int64_t N, const double *x, const double *q, double L,
                      int M, int P, double alpha, double cg, int cell_mode,
                      const double *Ht, double *phi, double *F)
{
    const double h = L / M;
    const double h3 = h * h * h;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t n = 0; n < N; ++n) {
        double xw[3];
        int i0[3];
        for (int d = 0; d < 3; ++d) {
            int c;
            wrap_and_cell(x[3 * n + d], L, M, cell_mode, &xw[d], &c);
            i0[d] = c - P / 2 + 1;
        }
        double s = 0.0, fx = 0.0, fy = 0.0, fz = 0.0;
        for (int a = 0; a < P; ++a) {
            double dx = (i0[0] + a) * h - xw[0];
            int jx = ((i0[0] + a) % M + M) % M;
            for (int b = 0; b < P; ++b) {
                double dy = (i0[1] + b) * h - xw[1];
                int jy = ((i0[1] + b) % M + M) % M;
                for (int c = 0; c < P; ++c) {
                    double dz = (i0[2] + c) * h - xw[2];
                    int jz = ((i0[2] + c) % M + M) % M;
                    double r2 = dx * dx + dy * dy + dz * dz;
                    double v = Ht[((size_t)jx * M + jy) * M + jz] * cg * exp(-alpha * r2);
                    s += v;
                    fx += dx * v; fy += dy * v; fz += dz * v;
                }
            }
        }
        phi[n] = h3 * s;
        F[3 * n] = -2.0 * alpha * h3 * q[n] * fx;
        F[3 * n + 1] = -2.0 * alpha * h3 * q[n] * fy;
        F[3 * n + 2] = -2.0 * alpha * h3 * q[n] * fz;
    }
}

/* Differentiation by i k in Fourier space (Sec. 2.3, the first of the three
 * ways to obtain the force): a full M^3 spectrum (iz fastest) is multiplied
 * by i k_d, k_d = 2 pi n_d / L with n_d the signed index along axis d.  For
 * an even M the Nyquist index n_d = M/2 stands for both +M/2 and -M/2; it
 * gets k_d = 0 (reading: the derivative of that mode is not defined on the
 * grid, and 0 keeps the derivative of a real grid real). */
void oracle_spectral_derivative(double *re, double *im, int M, double L, int axis)
{
    const double t = 2.0 * M_PI / L;
    for (int nx = 0; nx < M; ++nx)
        for (int ny = 0; ny < M; ++ny)
            for (int nz = 0; nz < M; ++nz) {
                int n = axis == 0 ? nx : (axis == 1 ? ny : nz);
                int sn = (2 * n == M) ? 0 : signed_index(n, M);
                double k = t * sn;
                size_t i = ((size_t)nx * M + ny) * M + nz;
                double a = re[i], b = im[i];
                re[i] = -k * b;
                im[i] = k * a;
            }
}

/*
 * SE k-space evaluation with forces by ik differentiation (Sec. 2.3): spread,
 * DFT and scaling as oracle_se_kspace; then, per axis d, the scaled spectrum
 * times i k_d, inverse DFT (the d-derivative of the smoothed potential grid),
 * and the gather with the same window as the spread (Eq. 3.9):
 *   F_m,d = -q_m h^3 sum_j (d_d Ht)_j c_g exp(-alpha |x_j - x_m|^2),
 * i.e. F = -q grad phi with the derivative taken on the grid instead of on
 * the window.  phi and E as in oracle_se_kspace.
 */
int oracle_se_kspace_ik(int64_t N, const double *x, const double *q,
                        double L, double xi, int M, int P, double c, double eta_in,
                        int cell_mode, double *E, double *phi, double *F)
{
    double prm[6];
    oracle_se_params(L, xi, M, P, c, eta_in, prm);
    const double eta = prm[2], alpha = prm[3], cg = prm[4];
    const size_t M3 = (size_t)M * M * M;
    double *re = (double *)malloc(sizeof(double) * M3);
    double *im = (double *)calloc(M3, sizeof(double));
    double *dr = (double *)malloc(sizeof(double) * M3);
    double *di = (double *)malloc(sizeof(double) * M3);
    double *gd = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    double *Fs = (double *)malloc(sizeof(double) * 3 * (size_t)(N > 0 ? N : 1));
    if (!re || !im || !dr || !di || !gd || !Fs) {
        free(re); free(im); free(dr); free(di); free(gd); free(Fs);
        return -1;
    }
    oracle_se_spread(N, x, q, L, M, P, alpha, cg, cell_mode, re);
    oracle_dft3(re, im, M, -1);
    double eg = 0.0;
    oracle_se_scale(re, im, M, L, xi, eta, &eg);
    for (int d = 0; d < 3; ++d) {
        memcpy(dr, re, sizeof(double) * M3);
        memcpy(di, im, sizeof(double) * M3);
        oracle_spectral_derivative(dr, di, M, L, d);
        oracle_dft3(dr, di, M, +1);
        /* the phi output of the gather on the derivative grid is h^3 sum D W */
        oracle_se_gather(N, x, q, L, M, P, alpha, cg, cell_mode, dr, gd, Fs);
        for (int64_t n = 0; n < N; ++n) F[3 * n + d] = -q[n] * gd[n];
    }
    oracle_dft3(re, im, M, +1);
    oracle_se_gather(N, x, q, L, M, P, alpha, cg, cell_mode, re, phi, Fs);
    double e = 0.0;
    for (int64_t n = 0; n < N; ++n) e += 0.5 * q[n] * phi[n];
    *E = e;
    free(re); free(im); free(dr); free(di); free(gd); free(Fs);
    return 0;
}

/*
 * The whole SE k-space evaluation (Algorithm 1 with the SE formulas of
 * Table 2): spread, DFT, scale, inverse DFT, gather, E = 1/2 sum q phi.
 * Optional outputs (pass NULL to skip): H (spread grid), Ht (the scaled and
 * back-transformed grid), E_grid (energy from the grid, Eq. 3.6 with
 * Parseval).  eta <= 0 selects Eq. 4.2 with shape constant c.
 */
int oracle_se_kspace(int64_t N, const double *x, const double *q,
                     double L, double xi, int M, int P, double c, double eta_in,
                     int cell_mode,
                     double *E, double *phi, double *F,
                     double *H_out, double *Ht_out, double *E_grid)
{
    double prm[6];
    oracle_se_params(L, xi, M, P, c, eta_in, prm);
    const double eta = prm[2], alpha = prm[3], cg = prm[4];
    const size_t M3 = (size_t)M * M * M;
    double *re = (double *)malloc(sizeof(double) * M3);
    double *im = (double *)calloc(M3, sizeof(double));
    if (!re || !im) { free(re); free(im); return -1; }
    oracle_se_spread(N, x, q, L, M, P, alpha, cg, cell_mode, re);
    if (H_out) memcpy(H_out, re, sizeof(double) * M3);
    oracle_dft3(re, im, M, -1);
    double eg = 0.0;
    oracle_se_scale(re, im, M, L, xi, eta, &eg);
    oracle_dft3(re, im, M, +1);
    /* the inverse transform of a Hermitian spectrum is real; im holds rounding only */
    if (Ht_out) memcpy(Ht_out, re, sizeof(double) * M3);
    oracle_se_gather(N, x, q, L, M, P, alpha, cg, cell_mode, re, phi, F);
    double e = 0.0;
    for (int64_t n = 0; n < N; ++n) e += 0.5 * q[n] * phi[n];
    *E = e;
    if (E_grid) *E_grid = eg;
    free(re); free(im);
    return 0;
}
