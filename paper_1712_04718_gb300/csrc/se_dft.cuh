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
struct StageDesc {
    int ij, is1, is2;
    int ok, os1, os2;
    int J, K, ncol, cd, f, post;
};

template <int TK, int TC>
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
                const float2 w = tw[rr[a]];
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
                    const float2 w = tw[hq[b] * (k0 + a)];   // j1 k2 < M1 M2 = M
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

}  // namespace se
