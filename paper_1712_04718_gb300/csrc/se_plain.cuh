// se_plain.cuh -- the gather with the plain (underived) window, and the
// scaling step of force evaluation by ik differentiation.
//
// Sec. 2.3 of arXiv:1712.04718 names three ways to obtain the force from the
// mesh: multiplication by i k in Fourier space (the most accurate, at the
// price of extra inverse transforms), differences on the mesh, and analytic
// differentiation of the window (the SE default, Sec. 3.1, in se_kernels.cuh).
// This file holds the first:
//   k_scale_ik      Hhat <- G/M^3 Hhat as k_scale, and in addition the three
//                   spectra D_d = i k_d G/M^3 Hhat (d = x, y, z; dstride
//                   complex values apart), whose
//                   inverse transforms are the gradient of the smoothed
//                   potential grid on the mesh;
//   k_gather_plain  phi_m and F_m = -q_m grad phi(x_m) from NG grids with the
//                   same Gaussian window as the spread (Eq. 3.9), no
//                   derivative of the window: NG = 4 reads [Ht, D_x, D_y, D_z]
//                   (ik forces), NG = 1 reads Ht alone (potential only).
// Since the spread and the gather use one window, sum_m F_m = -(h^3/M^3)
// sum_k i k G |Hhat_k|^2, a sum of terms odd in k: ik forces conserve
// momentum to rounding, where the analytic forces do not (Sec. 4).
#pragma once
#include <algorithm>
#include <type_traits>

#include "se_kernels.cuh"

namespace se {

// Signed wave number of index n on an M-point grid for a first derivative:
// the Nyquist index of an even M (n = M/2, whose sign is ambiguous) gets 0,
// so that the differentiated spectrum stays Hermitian and its inverse real.
__device__ __forceinline__ int deriv_index(int n, int M) {
    return (2 * n < M) ? n : ((2 * n == M) ? 0 : n - M);
}

template <typename T, typename C>
__global__ void __launch_bounds__(256)
k_scale_ik(C* __restrict__ cgrid, C* __restrict__ dgrid, long long dstride,
           const double* __restrict__ green, int M, double invM3, double kunit,
           T* __restrict__ zero_grid, double* __restrict__ partials, unsigned* ticket, Acc* acc,
           double e_scale, double* E_out) {
    __shared__ double sbuf[32];
    const int Mh = M / 2 + 1;
    const long long total = (long long)M * M * Mh;
    const long long stride = (long long)gridDim.x * blockDim.x;
    double e = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        const int kz = (int)(i % Mh);
        const long long r = i / Mh;
        const int iy = (int)(r % M), ix = (int)(r / M);
        const double g = green[i];
        C c = cgrid[i];
        const double m2 = (double)c.x * (double)c.x + (double)c.y * (double)c.y;
        e += ((kz == 0 || 2 * kz == M) ? 1.0 : 2.0) * g * m2;
        const double f = g * invM3;
        const T fT = (T)f;
        // i k_d f (a + i b) = k_d f (-b + i a)
        const T fx = (T)(kunit * deriv_index(ix, M) * f);
        const T fy = (T)(kunit * deriv_index(iy, M) * f);
        const T fz = (T)(kunit * deriv_index(kz, M) * f);
        C d;
        d.x = -fx * c.y;
        d.y = fx * c.x;
        dgrid[i] = d;
        d.x = -fy * c.y;
        d.y = fy * c.x;
        dgrid[dstride + i] = d;
        d.x = -fz * c.y;
        d.y = fz * c.x;
        dgrid[2 * dstride + i] = d;
        c.x *= fT;
        c.y *= fT;
        cgrid[i] = c;
    }
    if (zero_grid) {
        const long long n3 = (long long)M * M * M;
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += stride)
            zero_grid[i] = T(0);
    }
    double rs = block_sum(e, sbuf);
    if (threadIdx.x == 0) partials[blockIdx.x] = rs;
    if (!last_block(ticket)) return;
    const double s = sum_partials(partials, gridDim.x, 1, 0, sbuf);
    if (threadIdx.x == 0) {
        acc->e_grid = s;
        if (E_out) *E_out = e_scale * s;
        *ticket = 0u;
    }
}

// Window sums of one particle over NG grids spaced gstride apart, this lane's
// z points only: v[n] = sum_a gx[a] sum_b gy[b] sum_c gz[c] grid_n[a, b, c].
template <typename T, int P, int NG>
__device__ __forceinline__ void plain_accum(const GatherPrep<T, P>& g, const T* __restrict__ grid,
                                            size_t gstride, int M, const T* sE3, T (&v)[NG]) {
    constexpr int D = pick_d(P);
    T acc[NG][D];
#pragma unroll
    for (int n = 0; n < NG; ++n)
#pragma unroll
        for (int j = 0; j < D; ++j) acc[n][j] = T(0);
    T px = g.px0;
#pragma unroll((NG == 1 && P <= 8) ? P : 1)
    for (int a = 0; a < P; ++a) {
        const T gxa = px * sE3[a];
        px *= g.Bx;
        const int jx = wrap_index(g.i0x + a, M);
        T tb[NG][D];
#pragma unroll
        for (int n = 0; n < NG; ++n)
#pragma unroll
            for (int j = 0; j < D; ++j) tb[n][j] = T(0);
#pragma unroll
        for (int b = 0; b < P; ++b) {
            const T* row = grid + ((size_t)jx * M + g.jy[b]) * M;
#pragma unroll
            for (int n = 0; n < NG; ++n)
#pragma unroll
                for (int j = 0; j < D; ++j) tb[n][j] += g.gy[b] * __ldg(row + n * gstride + g.jz[j]);
        }
#pragma unroll
        for (int n = 0; n < NG; ++n)
#pragma unroll
            for (int j = 0; j < D; ++j) acc[n][j] += gxa * tb[n][j];
    }
#pragma unroll
    for (int n = 0; n < NG; ++n)
#pragma unroll
        for (int j = 0; j < D; ++j) v[n] += g.gz[j] * acc[n][j];
}

// phi_m = kc h^3 c_g v0 and, for NG = 4, F_m,d = -q_m kc h^3 c_g v_d: the
// gradient grids are already derivatives, so the window enters underived.
// The energy 1/2 sum q phi is reduced as in k_gather.  Particles and launch
// shape as k_gather (G lanes per particle, warp-synchronous reduction).
template <typename T, int P, int NG>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 && P <= 8) ? 4 : 1)
k_gather_plain(const v4_t<T>* __restrict__ sorted, const int* __restrict__ perm,
               const T* __restrict__ grid, size_t gstride, T* __restrict__ phi,
               T* __restrict__ F, const KParams<T> kp, double* __restrict__ partials,
               unsigned* ticket, Acc* acc, double e_scale, double* E_out) {
    constexpr int D = pick_d(P), G = P / D, GPW = 32 / G;
    constexpr bool kSingle = sizeof(T) == sizeof(float);
    __shared__ double sbuf[32];
    __shared__ df2 sbuf_df[32];
    __shared__ T sE3[P];
    if (threadIdx.x < P) sE3[threadIdx.x] = kp.E3[threadIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gi = lane / G, k = lane - gi * G;
    const int gpb = (blockDim.x >> 5) * GPW;
    int pb = blockIdx.x * gpb + warp * GPW;
    GatherPrep<T, P> g;
    T qq = T(0);
    if (gi < GPW && pb + gi < kp.N) {
        const v4_t<T> v = sorted[pb + gi];
        qq = v.w;
        gather_prep<T, P>(v, kp, k, g);
    }
    pdl_wait();
    __syncthreads();
    double e_loc = 0.0;
    df2 e_df = df_from(0.0f);
    for (; pb < kp.N; pb += gridDim.x * gpb) {
        const int p = pb + gi;
        const bool valid = (gi < GPW) && (p < kp.N);
        T v[NG];
#pragma unroll
        for (int n = 0; n < NG; ++n) v[n] = T(0);
        if (valid) {
            if (pb != blockIdx.x * gpb + warp * GPW) {
                const v4_t<T> pv = sorted[p];
                qq = pv.w;
                gather_prep<T, P>(pv, kp, k, g);
            }
            plain_accum<T, P, NG>(g, grid, gstride, kp.M, sE3, v);
        }
#pragma unroll
        for (int o = 1; o < G; o <<= 1) {
#pragma unroll
            for (int n = 0; n < NG; ++n) {
                const T a = __shfl_down_sync(0xffffffffu, v[n], o);
                if (k + o < G) v[n] += a;
            }
        }
        if (valid && k == 0) {
            const T ph = v[0] * kp.phi_scale;
            const int orig = perm ? perm[p] : p;
            if (phi) phi[orig] = ph;
            if (NG == 4 && F) {
                const T fm = -qq * kp.phi_scale;
                F[3 * orig] = fm * v[1 % NG];
                F[3 * orig + 1] = fm * v[2 % NG];
                F[3 * orig + 2] = fm * v[3 % NG];
            }
            if (kSingle)
                e_df = df_add(e_df, df_from((float)(qq * ph)));
            else
                e_loc += (double)qq * (double)ph;
        }
    }
    if (kSingle) {
        float* pf = reinterpret_cast<float*>(partials);
        const df2 r = block_sum_df(e_df, sbuf_df);
        if (threadIdx.x == 0) {
            pf[2 * blockIdx.x] = r.hi;
            pf[2 * blockIdx.x + 1] = r.lo;
        }
        if (!last_block(ticket) || threadIdx.x >= 32) return;
        const df2 t = warp_sum_partials_df(pf, gridDim.x, 1, 0);
        if (threadIdx.x == 0) {
            const double s = df_to_double(t);
            acc->e_gather = s;
            if (E_out) *E_out = e_scale * s;
            *ticket = 0u;
        }
        return;
    }
    double r = block_sum(e_loc, sbuf);
    if (threadIdx.x == 0) partials[blockIdx.x] = r;
    if (!last_block(ticket)) return;
    const double s = sum_partials(partials, gridDim.x, 1, 0, sbuf);
    if (threadIdx.x == 0) {
        acc->e_gather = s;
        if (E_out) *E_out = e_scale * s;
        *ticket = 0u;
    }
}

#ifndef SE_P_LIST
#define SE_P_LIST(X) X(2) X(4) X(6) X(8) X(10) X(12) X(14) X(16) X(18) X(20) X(22) X(24) X(26) X(28) X(30) X(32)
#endif

template <typename T>
cudaError_t launch_scale_ik(void* cgrid, void* dgrid, size_t dstride, const double* green, int M,
                            double L, T* zero_grid, double* partials, unsigned* ticket, Acc* acc,
                            double e_scale, double* E_out, cudaStream_t s) {
    using C = typename std::conditional<std::is_same<T, float>::value, float2, double2>::type;
    const long long total = (long long)M * M * (M / 2 + 1);
    const int blocks = (int)std::max(1LL, std::min((total + 255) / 256, (long long)kMaxPartials));
    const double invM3 = 1.0 / ((double)M * M * M);
    const double kunit = 2.0 * 3.14159265358979323846 / L;
    if (dstride < (size_t)total) return cudaErrorInvalidValue;
    k_scale_ik<T, C><<<blocks, 256, 0, s>>>((C*)cgrid, (C*)dgrid, (long long)dstride, green, M,
                                             invM3, kunit, zero_grid, partials, ticket, acc,
                                             e_scale, E_out);
    return cudaGetLastError();
}

template <typename T, int P, int NG>
cudaError_t gather_plain_P(const v4_t<T>* sorted, const int* perm, const T* grid, size_t gstride,
                           T* phi, T* F, const KParams<T>& kp, double* partials, unsigned* ticket,
                           Acc* acc, double e_scale, double* E_out, bool pdl, cudaStream_t s) {
    constexpr int GPW = 32 / (P / pick_d(P));
    const int gpb = 8 * GPW;
    const int blocks = std::max(1, std::min((kp.N + gpb - 1) / gpb, kMaxPartials));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(256);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = pdl ? attr : nullptr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k_gather_plain<T, P, NG>, sorted, perm, grid, gstride, phi, F,
                              kp, partials, ticket, acc, e_scale, E_out);
}

template <typename T>
cudaError_t launch_gather_plain(int ng, const v4_t<T>* sorted, const int* perm, const T* grid,
                                size_t gstride, T* phi, T* F, const KParams<T>& kp,
                                double* partials, unsigned* ticket, Acc* acc, double e_scale,
                                double* E_out, bool pdl, cudaStream_t s) {
    if (ng != 1 && ng != 4) return cudaErrorInvalidValue;
    switch (kp.P) {
#define SE_CASE(PP)                                                                             \
    case PP:                                                                                    \
        return ng == 1 ? gather_plain_P<T, PP, 1>(sorted, perm, grid, gstride, phi, F, kp,      \
                                                  partials, ticket, acc, e_scale, E_out, pdl, s) \
                       : gather_plain_P<T, PP, 4>(sorted, perm, grid, gstride, phi, F, kp,      \
                                                  partials, ticket, acc, e_scale, E_out, pdl, s);
        SE_P_LIST(SE_CASE)
#undef SE_CASE
        default: return cudaErrorInvalidValue;
    }
}

#define SE_PLAIN_INSTANTIATE(T)                                                                 \
    template cudaError_t launch_scale_ik<T>(void*, void*, size_t, const double*, int, double,   \
                                            T*, double*, unsigned*, Acc*, double, double*,      \
                                            cudaStream_t);                                      \
    template cudaError_t launch_gather_plain<T>(int, const v4_t<T>*, const int*, const T*,      \
                                                size_t, T*, T*, const KParams<T>&, double*,     \
                                                unsigned*, Acc*, double, double*, bool,         \
                                                cudaStream_t);

}  // namespace se
