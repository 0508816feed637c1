// se_dft.cuh -- register-tiled direct DFTs on data in shared memory, for the
// single-precision pipeline (M <= 128).  Each routine is a small complex
// matrix product: output (k, c) = sum_j input(j, c) w^{j k}, w = e^{sign 2 pi i / M},
// with a TK x TC tile of outputs per thread (independent accumulators, the
// inputs and twiddles of one j reused TK and TC times).  Twiddles come from
// the table tw[r] = (cos, sin)(2 pi r / M), r = (j k) mod M kept incrementally.
#pragma once
#include <cuda_runtime.h>

namespace se {

// Complex to complex.  X(j, c) = X[j*xj + c*xc], Y(k, c) = Y[k*yk + c*yc].
template <int TK, int TC>
__device__ __forceinline__ void dft_c2c(const float2* __restrict__ X, int xj, int xc,
                                        float2* __restrict__ Y, int yk, int yc, int J, int K,
                                        int C, const float2* __restrict__ tw, int M, float sign) {
    const int nk = (K + TK - 1) / TK, nc = (C + TC - 1) / TC;
    for (int t = threadIdx.x; t < nk * nc; t += blockDim.x) {
        const int k0 = (t / nc) * TK, c0 = (t % nc) * TC;
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
    for (int t = threadIdx.x; t < nk * nc; t += blockDim.x) {
        const int k0 = (t / nc) * TK, c0 = (t % nc) * TC;
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
    for (int t = threadIdx.x; t < nk * nc; t += blockDim.x) {
        const int k0 = (t / nc) * TK, c0 = (t % nc) * TC;
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

}  // namespace se
