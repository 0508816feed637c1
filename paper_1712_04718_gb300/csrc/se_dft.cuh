// se_dft.cuh -- register-tiled direct DFTs on data in shared memory, for the
// single-precision pipeline (M <= 128).  Each routine is a small complex
// matrix product: output (k, c) = sum_j input(j, c) w^{j k}, w = e^{sign 2 pi i / M},
// with a TK x TC tile of outputs per thread (independent accumulators, the
// inputs and twiddles of one j reused TK and TC times).  Twiddles come from
// the table tw[r] = (cos, sin)(2 pi r / M), r = (j k) mod M kept incrementally.
#pragma once
#include <cuda_runtime.h>

#include "se_kernels.cuh"

namespace se {

// Complex to complex.  X(j, c) = X[j*xj + c*xc], Y(k, c) = Y[k*yk + c*yc].
template <int TK, int TC>
__device__ __forceinline__ void dft_c2c(const float2* __restrict__ X, int xj, int xc,
                                        float2* __restrict__ Y, int yk, int yc, int J, int K,
                                        int C, const float2* __restrict__ tw, int M, float sign) {
    const int nk = (K + TK - 1) / TK, nc = (C + TC - 1) / TC;
    const FDiv fnc = fdiv_of(nc);
    for (int t = threadIdx.x; t < nk * nc; t += blockDim.x) {
        const int tq = fdiv(t, fnc);
        const int k0 = tq * TK, c0 = (t - tq * nc) * TC;
        float ar[TK][TC], ai[TK][TC];
        int r[TK];
#pragma unroll
        for (int a = 0; a < TK; ++a) {
            r[a] = 0;
#pragma unroll
            for (int b = 0; b < TC; ++b) ar[a][b] = ai[a][b] = 0.f;
        }
        for (int j = 0; j < J; ++j) {
            float2 x[TC];
#pragma unroll
            for (int b = 0; b < TC; ++b)
                x[b] = (c0 + b < C) ? X[j * xj + (c0 + b) * xc] : make_float2(0.f, 0.f);
#pragma unroll
            for (int a = 0; a < TK; ++a) {
                const float2 w = tw[r[a]];
                const float ws = sign * w.y;
#pragma unroll
                for (int b = 0; b < TC; ++b) {
                    ar[a][b] = fmaf(x[b].x, w.x, fmaf(-x[b].y, ws, ar[a][b]));
                    ai[a][b] = fmaf(x[b].x, ws, fmaf(x[b].y, w.x, ai[a][b]));
                }
                r[a] += (k0 + a < K) ? k0 + a : 0;   // rows past K: stay at r = 0
                if (r[a] >= M) r[a] -= M;
            }
        }
#pragma unroll
        for (int a = 0; a < TK; ++a)
#pragma unroll
            for (int b = 0; b < TC; ++b)
                if (k0 + a < K && c0 + b < C)
                    Y[(k0 + a) * yk + (c0 + b) * yc] = make_float2(ar[a][b], ai[a][b]);
    }
}

// Real to complex, forward (e^{-i}): Y(k, c) = sum_j X(j, c) e^{-2 pi i j k / M}, k < K.
template <int TK, int TC>
__device__ __forceinline__ void dft_r2c(const float* __restrict__ X, int xj, int xc,
                                        float2* __restrict__ Y, int yk, int yc, int J, int K,
                                        int C, const float2* __restrict__ tw, int M) {
    const int nk = (K + TK - 1) / TK, nc = (C + TC - 1) / TC;
    const FDiv fnc = fdiv_of(nc);
    for (int t = threadIdx.x; t < nk * nc; t += blockDim.x) {
        const int tq = fdiv(t, fnc);
        const int k0 = tq * TK, c0 = (t - tq * nc) * TC;
        float ar[TK][TC], ai[TK][TC];
        int r[TK];
#pragma unroll
        for (int a = 0; a < TK; ++a) {
            r[a] = 0;
#pragma unroll
            for (int b = 0; b < TC; ++b) ar[a][b] = ai[a][b] = 0.f;
        }
        for (int j = 0; j < J; ++j) {
            float x[TC];
#pragma unroll
            for (int b = 0; b < TC; ++b) x[b] = (c0 + b < C) ? X[j * xj + (c0 + b) * xc] : 0.f;
#pragma unroll
            for (int a = 0; a < TK; ++a) {
                const float2 w = tw[r[a]];
#pragma unroll
                for (int b = 0; b < TC; ++b) {
                    ar[a][b] = fmaf(x[b], w.x, ar[a][b]);
                    ai[a][b] = fmaf(-x[b], w.y, ai[a][b]);
                }
                r[a] += (k0 + a < K) ? k0 + a : 0;   // rows past K: stay at r = 0
                if (r[a] >= M) r[a] -= M;
            }
        }
#pragma unroll
        for (int a = 0; a < TK; ++a)
#pragma unroll
            for (int b = 0; b < TC; ++b)
                if (k0 + a < K && c0 + b < C)
                    Y[(k0 + a) * yk + (c0 + b) * yc] = make_float2(ar[a][b], ai[a][b]);
    }
}

// Complex (half spectrum, already multiplied by the Hermitian weights) to
// real, inverse (e^{+i}): Y(k, c) = sum_j Re(X(j, c) e^{+2 pi i j k / M}), k < K.
template <int TK, int TC>
__device__ __forceinline__ void dft_c2r(const float2* __restrict__ X, int xj, int xc,
                                        float* __restrict__ Y, int yk, int yc, int J, int K,
                                        int C, const float2* __restrict__ tw, int M) {
    const int nk = (K + TK - 1) / TK, nc = (C + TC - 1) / TC;
    const FDiv fnc = fdiv_of(nc);
    for (int t = threadIdx.x; t < nk * nc; t += blockDim.x) {
        const int tq = fdiv(t, fnc);
        const int k0 = tq * TK, c0 = (t - tq * nc) * TC;
        float ar[TK][TC];
        int r[TK];
#pragma unroll
        for (int a = 0; a < TK; ++a) {
            r[a] = 0;
#pragma unroll
            for (int b = 0; b < TC; ++b) ar[a][b] = 0.f;
        }
        for (int j = 0; j < J; ++j) {
            float2 x[TC];
#pragma unroll
            for (int b = 0; b < TC; ++b)
                x[b] = (c0 + b < C) ? X[j * xj + (c0 + b) * xc] : make_float2(0.f, 0.f);
#pragma unroll
            for (int a = 0; a < TK; ++a) {
                const float2 w = tw[r[a]];
#pragma unroll
                for (int b = 0; b < TC; ++b) ar[a][b] = fmaf(x[b].x, w.x, fmaf(-x[b].y, w.y, ar[a][b]));
                r[a] += (k0 + a < K) ? k0 + a : 0;   // rows past K: stay at r = 0
                if (r[a] >= M) r[a] -= M;
            }
        }
#pragma unroll
        for (int a = 0; a < TK; ++a)
#pragma unroll
            for (int b = 0; b < TC; ++b)
                if (k0 + a < K && c0 + b < C) Y[(k0 + a) * yk + (c0 + b) * yc] = ar[a][b];
    }
}

// ---------------------------------------------------------------------------
// Factored complex DFT (Cooley-Tukey with M = M1 M2): with j = j1 + M1 j2 and
// k = k2 + M2 k1,
//   Y(k2 + M2 k1) = sum_{j1} w^{M2 j1 k1} [ w^{j1 k2} sum_{j2} X(j1 + M1 j2) w^{M1 j2 k2} ],
// i.e. M1 DFTs of length M2, a twiddle, and M2 DFTs of length M1: M1 + M2
// terms per output instead of M.  Both stages are dft_stage calls.

// One stage: for every column col < ncol and k < K,
//   out[oo(col) + k ok] = pt(col, k) sum_{j < J} in[io(col) + j ij] w^{f j k},
// w = e^{sign 2 pi i / M}, io(col) = (col / cd) is1 + (col % cd) is2 (oo the
// same with os1, os2) and pt = w^{(col / cd) k} when post is set, else 1.
// M is the transform's length; the twiddles are read at index r << tsh of
// the table (template tsh = 1: a length-M/2 transform from the length-M table).
struct StageDesc {
    int ij, is1, is2;
    int ok, os1, os2;
    int J, K, ncol, cd, f, post;
};

template <int TK, int TC, int tsh = 0>
__device__ __forceinline__ void dft_stage(const float2* __restrict__ in, float2* __restrict__ out,
                                          const StageDesc d, const float2* __restrict__ tw, int M,
                                          float sign) {
    const int nk = (d.K + TK - 1) / TK, nc = (d.ncol + TC - 1) / TC;
    const FDiv fnc = fdiv_of(nc), fcd = fdiv_of(d.cd);
    for (int t = threadIdx.x; t < nk * nc; t += blockDim.x) {
        const int tq = fdiv(t, fnc);
        const int k0 = tq * TK, c0 = (t - tq * nc) * TC;
        int io[TC], oo[TC], hq[TC];
        bool cv[TC];
#pragma unroll
        for (int b = 0; b < TC; ++b) {
            const int col = c0 + b;
            cv[b] = col < d.ncol;
            const int q = cv[b] ? fdiv(col, fcd) : 0, r = cv[b] ? col - q * d.cd : 0;
            hq[b] = q;
            io[b] = q * d.is1 + r * d.is2;
            oo[b] = q * d.os1 + r * d.os2;
        }
        float ar[TK][TC], ai[TK][TC];
        int rr[TK], st[TK];
#pragma unroll
        for (int a = 0; a < TK; ++a) {
            rr[a] = 0;
            st[a] = (k0 + a < d.K) ? d.f * (k0 + a) : 0;   // < M for every stage
#pragma unroll
            for (int b = 0; b < TC; ++b) ar[a][b] = ai[a][b] = 0.f;
        }
        for (int j = 0; j < d.J; ++j) {
            float2 x[TC];
#pragma unroll
            for (int b = 0; b < TC; ++b)
                x[b] = cv[b] ? in[io[b] + j * d.ij] : make_float2(0.f, 0.f);
#pragma unroll
            for (int a = 0; a < TK; ++a) {
                const float2 w = tw[rr[a] << tsh];
                const float ws = sign * w.y;
#pragma unroll
                for (int b = 0; b < TC; ++b) {
                    ar[a][b] = fmaf(x[b].x, w.x, fmaf(-x[b].y, ws, ar[a][b]));
                    ai[a][b] = fmaf(x[b].x, ws, fmaf(x[b].y, w.x, ai[a][b]));
                }
                rr[a] += st[a];
                if (rr[a] >= M) rr[a] -= M;
            }
        }
#pragma unroll
        for (int a = 0; a < TK; ++a)
#pragma unroll
            for (int b = 0; b < TC; ++b) {
                if (!(k0 + a < d.K && cv[b])) continue;
                float re = ar[a][b], im = ai[a][b];
                if (d.post) {
                    const float2 w = tw[(hq[b] * (k0 + a)) << tsh];   // j1 k2 < M1 M2 = M
                    const float ws = sign * w.y;
                    const float r2 = fmaf(re, w.x, -im * ws);
                    im = fmaf(re, ws, im * w.x);
                    re = r2;
                }
                out[oo[b] + (k0 + a) * d.ok] = make_float2(re, im);
            }
    }
}

// M1: the largest divisor of M not above sqrt(M) (1 when M is prime), which
// makes M1 + M / M1 smallest.
__host__ __device__ inline int dft_split(int M) {
    int best = 1;
    for (int a = 2; a * a <= M; ++a)
        if (M % a == 0) best = a;
    return best;
}

// Y(k, c) = sum_j X(j, c) w^{j k} for C columns, j, k < M, through the
// factored form with the scratch Z (M x C complex, distinct from X and Y).
// Called by the whole block; X must be ready (synchronised) before the call,
// and Y is complete after the caller's next barrier.
template <int TK = 2, int TC = 2>
__device__ __forceinline__ void dft_c2c_fact(const float2* __restrict__ X, int xj, int xc,
                                             float2* __restrict__ Y, int yk, int yc, int C,
                                             float2* __restrict__ Z,
                                             const float2* __restrict__ tw, int M, float sign) {
    const int M1 = dft_split(M), M2 = M / M1;
    if (M1 == 1) {
        dft_stage<TK, TC>(X, Y, StageDesc{xj, 0, xc, yk, 0, yc, M, M, C, C, 1, 0}, tw, M, sign);
        return;
    }
    dft_stage<TK, TC>(X, Z, StageDesc{M1 * xj, xj, xc, C, M2 * C, 1, M2, M2, M1 * C, C, M1, 1},
                      tw, M, sign);
    __syncthreads();
    dft_stage<TK, TC>(Z, Y, StageDesc{M2 * C, C, 1, M2 * yk, yk, yc, M1, M1, M2 * C, C, M2, 0},
                      tw, M, sign);
}

// ---------------------------------------------------------------------------
// Real transforms of even length M through a complex transform of length
// N = M / 2 (the classical packing of two real samples into one complex
// one), factored as above: N (N1 + N2) complex terms per row instead of the
// M (M/2 + 1) real-by-complex terms of dft_r2c / dft_c2r, which pays for
// the packing pass and its barriers when N factors (dft_split(N) > 1).  P
// and Q are scratch of N x C complex each, distinct from one another and
// from Y of the forward transform; Q may share storage with X of the
// forward transform (X is dead once packed) or with Y of the inverse one (Y
// is written last), so none of these carries __restrict__.  Called by the
// whole block with X ready; Y is complete after the caller's next barrier.

// The length-N transform of the C columns of P (P(n, c) = P[n C + c]) into
// P, through Q (sign: -1 forward, +1 inverse).
template <int TK, int TC>
__device__ __forceinline__ void dft_half_pq(float2* P, float2* Q, int C, int N,
                                            const float2* __restrict__ tw, float sign) {
    const int N1 = dft_split(N), N2 = N / N1;
    if (N1 == 1) {
        dft_stage<TK, TC, 1>(P, Q, StageDesc{C, 0, 1, C, 0, 1, N, N, C, C, 1, 0}, tw, N, sign);
        __syncthreads();
        for (int e = threadIdx.x; e < N * C; e += blockDim.x) P[e] = Q[e];
        return;
    }
    dft_stage<TK, TC, 1>(P, Q, StageDesc{N1 * C, C, 1, C, N2 * C, 1, N2, N2, N1 * C, C, N1, 1},
                         tw, N, sign);
    __syncthreads();
    dft_stage<TK, TC, 1>(Q, P, StageDesc{N2 * C, C, 1, N2 * C, C, 1, N1, N1, N2 * C, C, N2, 0},
                         tw, N, sign);
}

// Real to complex, forward: Y(k, c) = sum_{j<M} X(j, c) e^{-2 pi i j k / M},
// k <= N.  With z(n) = x(2n) + i x(2n+1) and Z its length-N transform,
// Y(k) = E(k) + w^k O(k), w = e^{-2 pi i / M}, where E = (Z(k) + conj Z(N-k)) / 2
// and O = -i (Z(k) - conj Z(N-k)) / 2 are the transforms of the even and odd
// samples (indices mod N).
template <int TK, int TC>
__device__ __forceinline__ void dft_r2c_half(const float* X, int xj, int xc, float2* __restrict__ Y,
                                             int yk, int yc, int C, float2* P, float2* Q,
                                             const float2* __restrict__ tw, int M) {
    const int N = M / 2;
    const FDiv fC = fdiv_of(max(C, 1));
    for (int e = threadIdx.x; e < N * C; e += blockDim.x) {
        const int n = fdiv(e, fC), c = e - n * C;
        const float* x = X + (size_t)(2 * n) * xj + (size_t)c * xc;
        P[e] = make_float2(x[0], x[xj]);
    }
    __syncthreads();
    dft_half_pq<TK, TC>(P, Q, C, N, tw, -1.0f);
    __syncthreads();
    for (int e = threadIdx.x; e < (N + 1) * C; e += blockDim.x) {
        const int k = fdiv(e, fC), c = e - k * C;
        const float2 a = P[(k == N ? 0 : k) * C + c];
        const float2 b = P[(k == 0 ? 0 : N - k) * C + c];   // Z(N - k mod N)
        const float er = 0.5f * (a.x + b.x), ei = 0.5f * (a.y - b.y);   // E
        const float orr = 0.5f * (a.y + b.y), oi = -0.5f * (a.x - b.x);   // O
        const float2 w = tw[k];   // (cos, sin)(2 pi k / M); forward: cos - i sin
        Y[(size_t)k * yk + (size_t)c * yc] =
            make_float2(er + fmaf(w.x, orr, w.y * oi), ei + fmaf(w.x, oi, -w.y * orr));
    }
}

// Complex (half spectrum) to real, inverse: Y(j, c) = Re sum_{k<=N} A(k, c)
// e^{+2 pi i j k / M}, j < M, where A(k) = X(k) times hw^{-1} for 0 < k < N
// (hw = 1/2 when X already carries the Hermitian weights 2, hw = 1 when it
// does not).  The conjugate-symmetric spectrum F with F(k) = hw X(k),
// F(M-k) = conj F(k) (0 < k < N), F(0) = Re X(0), F(N) = Re X(N) has the
// same real transform; its even and odd samples are the real and imaginary
// parts of the length-N inverse transform of
//   Z(k) = (F(k) + F(k+N)) + i w^k (F(k) - F(k+N)),  w = e^{+2 pi i / M}, k < N.
template <int TK, int TC>
__device__ __forceinline__ void dft_c2r_half(const float2* X, int xj, int xc, float* Y,
                                             int yk, int yc, int C, float2* P, float2* Q,
                                             const float2* __restrict__ tw, int M, float hw) {
    const int N = M / 2;
    const FDiv fC = fdiv_of(max(C, 1));
    for (int e = threadIdx.x; e < N * C; e += blockDim.x) {
        const int k = fdiv(e, fC), c = e - k * C;
        float2 f0, f1;   // F(k), F(k + N)
        if (k == 0) {
            f0 = make_float2(X[(size_t)c * xc].x, 0.f);
            f1 = make_float2(X[(size_t)N * xj + (size_t)c * xc].x, 0.f);
        } else {
            const float2 u = X[(size_t)k * xj + (size_t)c * xc];
            const float2 v = X[(size_t)(N - k) * xj + (size_t)c * xc];
            f0 = make_float2(hw * u.x, hw * u.y);
            f1 = make_float2(hw * v.x, -hw * v.y);
        }
        const float sr = f0.x + f1.x, si = f0.y + f1.y;   // F(k) + F(k+N)
        const float dr = f0.x - f1.x, di = f0.y - f1.y;   // F(k) - F(k+N)
        const float2 w = tw[k];                           // e^{+i theta} = cos + i sin
        const float tr = fmaf(w.x, dr, -w.y * di), ti = fmaf(w.x, di, w.y * dr);
        P[e] = make_float2(sr - ti, si + tr);             // + i (w d)
    }
    __syncthreads();
    dft_half_pq<TK, TC>(P, Q, C, N, tw, 1.0f);
    __syncthreads();
    for (int e = threadIdx.x; e < N * C; e += blockDim.x) {
        const int n = fdiv(e, fC), c = e - n * C;
        const float2 z = P[e];
        float* y = Y + (size_t)(2 * n) * yk + (size_t)c * yc;
        y[0] = z.x;
        y[yk] = z.y;
    }
}

// Whether the half-length real transforms serve length M: when they cut
// the multiply-adds of a row at least 2.75-fold (2 M (M/2+1) real-by-complex
// against 4 N (N1 + N2) complex ones).  Measured on the slab transforms:
// M = 84 (3.3-fold) 19 % faster, M = 52 (1.8-fold, 2-CTA clusters) 11 %
// slower, the packing pass and its barriers outweighing the saved terms.
// Build with -DSE_DFT_HALF=0 for the direct ones everywhere.
#ifndef SE_DFT_HALF
#define SE_DFT_HALF 1
#endif
constexpr int kDftHalfR4 = 11;   // the 2.75-fold cut, in quarters
// Slab transforms of many systems at once (the ensemble) keep every SM busy:
// there the saved terms pay at a smaller cut (build-time knob, in quarters).
#ifndef SE_DFT_HALF_BATCH_R4
#define SE_DFT_HALF_BATCH_R4 11
#endif
__host__ __device__ inline bool dft_half_ok(int M, int r4 = kDftHalfR4) {
    if (!SE_DFT_HALF || M % 2 != 0 || M < 8) return false;
    const int N = M / 2, N1 = dft_split(N);
    return N1 > 1 && 2 * M * (M / 2 + 1) * 4 >= r4 * 4 * N * (N1 + N / N1);
}

}  // namespace se
