// se_launch.cuh -- host launchers of the SE kernels, dispatching the support
// size P (even, 2..32) to the compile-time kernel instances.
#pragma once
#include <algorithm>

#include "se_kernels.cuh"

namespace se {

#ifndef SE_P_LIST
#define SE_P_LIST(X) X(2) X(4) X(6) X(8) X(10) X(12) X(14) X(16) X(18) X(20) X(22) X(24) X(26) X(28) X(30) X(32)
#endif
#define SE_FOR_EACH_P(X) \
    SE_P_LIST(X)

constexpr int kThreads = 256;

template <typename T>
cudaError_t launch_bin(const T* xyz, const T* q, const KParams<T>& kp, int* tile_count,
                       int* slot, int* tile_of, int* tile_start, double* partials,
                       unsigned* ticket, Acc* acc, cudaStream_t s) {
    int blocks = std::max(1, std::min((kp.N + kThreads - 1) / kThreads, kMaxPartials));
    k_bin<T><<<blocks, kThreads, 0, s>>>(xyz, q, kp, tile_count, slot, tile_of, tile_start,
                                         partials, ticket, acc);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scatter(const T* xyz, const T* q, const KParams<T>& kp, const int* slot,
                           const int* tile_of, const int* tile_start, v4_t<T>* sorted,
                           int* perm, cudaStream_t s) {
    if (kp.N == 0) return cudaSuccess;
    int blocks = std::min((kp.N + kThreads - 1) / kThreads, 8192);
    k_scatter<T><<<blocks, kThreads, 0, s>>>(xyz, q, kp, slot, tile_of, tile_start, sorted, perm);
    return cudaGetLastError();
}

template <typename T, int P, bool COMP>
cudaError_t spread_tiled_P(const v4_t<T>* sorted, const int* tile_start, T* grid,
                           const KParams<T>& kp, cudaStream_t s) {
    const size_t R = (size_t)kp.tile + P - 1;
    const size_t plane = R * R * sizeof(T) * (COMP ? 2 : 1);
    const int slab = (int)std::min(R, kSmemBudget / plane);
    if (slab < 1) return cudaErrorInvalidValue;
    const size_t bytes = (size_t)slab * plane;
    cudaError_t e = cudaFuncSetAttribute(k_spread_tiled<T, P, COMP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmemBudget);
    if (e != cudaSuccess) return e;
    k_spread_tiled<T, P, COMP><<<kp.ntiles, kThreads, bytes, s>>>(sorted, tile_start, grid, kp, slab);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_spread_tiled(const v4_t<T>* sorted, const int* tile_start, T* grid,
                                const KParams<T>& kp, bool comp, cudaStream_t s) {
    switch (kp.P) {
#define SE_CASE(PP) \
    case PP: return comp ? spread_tiled_P<T, PP, true>(sorted, tile_start, grid, kp, s) \
                         : spread_tiled_P<T, PP, false>(sorted, tile_start, grid, kp, s);
        SE_FOR_EACH_P(SE_CASE)
#undef SE_CASE
        default: return cudaErrorInvalidValue;
    }
}

template <typename T, int P>
cudaError_t spread_direct_P(const v4_t<T>* sorted, T* grid, const KParams<T>& kp, cudaStream_t s) {
    if (kp.N == 0) return cudaSuccess;
    constexpr int GPW = 32 / (P / pick_d(P));
    const int gpb = (kThreads / 32) * GPW;
    const int blocks = std::min((kp.N + gpb - 1) / gpb, 152 * 32);
    k_spread_direct<T, P><<<blocks, kThreads, 0, s>>>(sorted, grid, kp);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_spread_direct(const v4_t<T>* sorted, T* grid, const KParams<T>& kp,
                                 cudaStream_t s) {
    switch (kp.P) {
#define SE_CASE(PP) case PP: return spread_direct_P<T, PP>(sorted, grid, kp, s);
        SE_FOR_EACH_P(SE_CASE)
#undef SE_CASE
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t launch_scale(void* cgrid, const double* green, int M, T* zero_grid,
                         double* partials, unsigned* ticket, Acc* acc, double e_scale,
                         double* E_out, cudaStream_t s) {
    using C = typename std::conditional<std::is_same<T, float>::value, float2, double2>::type;
    const long long total = (long long)M * M * (M / 2 + 1);
    const int blocks = (int)std::max(1LL, std::min((total + kThreads - 1) / kThreads,
                                                   (long long)kMaxPartials));
    const double invM3 = 1.0 / ((double)M * M * M);
    k_scale<T, C><<<blocks, kThreads, 0, s>>>((C*)cgrid, green, M, invM3, zero_grid, partials,
                                              ticket, acc, e_scale, E_out);
    return cudaGetLastError();
}

template <typename T, int P>
cudaError_t gather_P(const v4_t<T>* sorted, const int* perm, const T* grid, T* phi, T* F,
                     const KParams<T>& kp, double* partials, unsigned* ticket, Acc* acc,
                     double e_scale, double* E_out, const double* adj, cudaStream_t s) {
    constexpr int GPW = 32 / (P / pick_d(P));
    const int gpb = (gather_threads<T, P>() / 32) * GPW;
    const int blocks = std::max(1, std::min((kp.N + gpb - 1) / gpb, kMaxPartials));
    k_gather<T, P><<<blocks, gather_threads<T, P>(), 0, s>>>(sorted, perm, grid, phi, F, kp, partials, ticket,
                                               acc, e_scale, E_out, adj);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gather(const v4_t<T>* sorted, const int* perm, const T* grid, T* phi,
                          T* F, const KParams<T>& kp, double* partials, unsigned* ticket,
                          Acc* acc, double e_scale, double* E_out, const double* adj,
                          cudaStream_t s) {
    switch (kp.P) {
#define SE_CASE(PP) \
    case PP: return gather_P<T, PP>(sorted, perm, grid, phi, F, kp, partials, ticket, acc, e_scale, E_out, adj, s);
        SE_FOR_EACH_P(SE_CASE)
#undef SE_CASE
        default: return cudaErrorInvalidValue;
    }
}

#define SE_INSTANTIATE(T)                                                                       \
    template cudaError_t launch_bin<T>(const T*, const T*, const KParams<T>&, int*, int*, int*,  \
                                       int*, double*, unsigned*, Acc*, cudaStream_t);            \
    template cudaError_t launch_scatter<T>(const T*, const T*, const KParams<T>&, const int*,    \
                                           const int*, const int*, v4_t<T>*, int*, cudaStream_t); \
    template cudaError_t launch_spread_tiled<T>(const v4_t<T>*, const int*, T*,                 \
                                                const KParams<T>&, bool, cudaStream_t);         \
    template cudaError_t launch_spread_direct<T>(const v4_t<T>*, T*, const KParams<T>&,         \
                                                 cudaStream_t);                                 \
    template cudaError_t launch_scale<T>(void*, const double*, int, T*, double*, unsigned*,     \
                                         Acc*, double, double*, cudaStream_t);                  \
    template cudaError_t launch_gather<T>(const v4_t<T>*, const int*, const T*, T*, T*,         \
                                          const KParams<T>&, double*, unsigned*, Acc*, double,  \
                                          double*, const double*, cudaStream_t);

}  // namespace se
