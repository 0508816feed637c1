// se_fast_launch.cuh -- host launchers of the single-precision pipeline
// (se_fast.cuh).  Every kernel after the first is launched with programmatic
// stream serialization: it may be scheduled while its predecessor drains and
// waits for that predecessor's results in griddepcontrol.wait.
#pragma once
#include <algorithm>

#include "se_fast.cuh"
#include "se_launch.cuh"

namespace se {

inline int fast_bin_blocks(const KParams<float>& kp) {
    const long long b = ((long long)kp.N + 255) / 256;
    return (int)std::max<long long>(1, std::min<long long>(b, kMaxPartials));
}

// Dynamic shared memory (at least `need`) with which no more than per_sm CTAs
// fit on an SM: the SM's shared memory over per_sm + 1/2 CTAs, less the
// per-CTA reservation and 1 KB for static shared memory.  A grid scheduled
// early, while its predecessor drains, is otherwise packed onto the SMs that
// have room; with the cap it spreads over all SMs.
inline size_t smem_cap_per_sm(size_t need, int per_sm) {
    int dev = 0, sm_bytes = 0, reserved = 0;
    if (per_sm < 1 || cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sm_bytes, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess)
        return need;
    const long long floor_b = (long long)(sm_bytes / (per_sm + 0.5)) - reserved - 1024;
    return floor_b > (long long)need ? (size_t)floor_b : need;
}

inline int sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return n;
}

template <int P>
cudaError_t fast_spread_P(const KParams<float>& kp, const FastBufs& b, int nbin, cudaStream_t s) {
    const size_t R = (size_t)kp.tile + P - 1;
    // one 32-bit accumulator per point, rows padded to the region stride
    const size_t plane = R * (size_t)region_stride<P>((int)R) * sizeof(unsigned);
    const int slab = (int)std::min(R, kSmemBudget / plane);
    if (slab < 1) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_fspread<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmemBudget);
    if (e != cudaSuccess) return e;
    // scheduled early (dependent launch) with at most ceil(grid / SMs) CTAs
    // per SM, up to the 5 that the kernel's registers allow
    const int grid = kp.ntiles + kOverflowBlocks, nsm = sm_count();
    const int per_sm = nsm > 0 ? (grid + nsm - 1) / nsm : 0;
    const size_t dyn = (P <= 8 && per_sm >= 1 && per_sm <= 5)
                           ? smem_cap_per_sm((size_t)slab * plane, per_sm)
                           : (size_t)slab * plane;
    return launch_ex(k_fspread<P>, grid, kThreads, dyn, s, true, (const f4*)b.bucket, b.cap, b.tile_count,
                     b.tile_n, (const int*)b.over_idx,
                     (int*)(b.tickets + 4), (const f4*)b.wrapped, (unsigned long long*)b.g64, kp,
                     (const double*)b.partials, nbin, b.tickets + 3, b.acc, slab);
}

template <int P>
cudaError_t fast_direct_P(const float* xyz, const float* q, const KParams<float>& kp,
                          const FastBufs& b, cudaStream_t s) {
    constexpr int GPW = 32 / (P / pick_d(P));
    const int gpb = (kThreads / 32) * GPW;
    const int blocks = std::max(1, std::min((kp.N + gpb - 1) / gpb, kMaxPartials));
    return launch_ex(k_fdirect<P>, blocks, kThreads, 0, s, false, xyz, q, kp, (float*)b.g64,
                     (f4*)b.wrapped, b.partials, b.tickets + 0, b.acc);
}

cudaError_t fast_spread(const float* xyz, const float* q, const KParams<float>& kp,
                        const FastBufs& b, cudaStream_t s, bool marks, void (*mark)(void*, int),
                        void* ctx) {
    if (b.unsorted) {
        if (marks) {
            mark(ctx, 0);
            mark(ctx, 1);
        }
        switch (kp.P) {
#define SE_CASE(PP) case PP: return fast_direct_P<PP>(xyz, q, kp, b, s);
            SE_FOR_EACH_P(SE_CASE)
#undef SE_CASE
            default: return cudaErrorInvalidValue;
        }
    }
    const int nbin = fast_bin_blocks(kp);
    cudaError_t e = launch_ex(k_fbin<float>, nbin, kThreads, 0, s, false, xyz, q, kp, b.tile_count,
                              (f4*)b.bucket, b.bucket_idx, b.cap, b.over_idx, (int*)(b.tickets + 4),
                              (f4*)b.wrapped, b.partials);
    if (e != cudaSuccess) return e;
    if (marks) {
        mark(ctx, 0);
        mark(ctx, 1);
    }
    switch (kp.P) {
#define SE_CASE(PP) case PP: return fast_spread_P<PP>(kp, b, nbin, s);
        SE_FOR_EACH_P(SE_CASE)
#undef SE_CASE
        default: return cudaErrorInvalidValue;
    }
}

// 2-CTA clusters per x-slab when every CTA gets an SM of its own (build
// with -DSE_SLAB_CL_PER_SM=n to allow n cluster CTAs per SM)
#ifndef SE_SLAB_CL_PER_SM
#define SE_SLAB_CL_PER_SM 1
#endif
inline bool slab_clusters(int M) {
    const int nsm = sm_count();
    return nsm > 0 && 2 * (M + 1) <= SE_SLAB_CL_PER_SM * nsm;
}

cudaError_t fast_inverse(const KParams<float>& kp, const FastBufs& b, double e_scale,
                         double* E_grid, cudaStream_t s) {
    const int M = kp.M, Mh = M / 2 + 1;
    const int nch = (Mh + kXpassKC - 1) / kXpassKC;
    const float2* tw = (const float2*)b.tw;
    const float2* C = (const float2*)b.cgrid;
    const int nsm = sm_count();
    cudaError_t e;
    if (!slab_clusters(M)) {
        const size_t slab = std::max(slab_smem_bytes(M), kSlabSmemFloor);
        auto kinv = dft_half_ok(M) ? k_slab_inv<true> : k_slab_inv<false>;
        e = cudaFuncSetAttribute(kinv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)slab);
        if (e != cudaSuccess) return e;
        return launch_ex(kinv, M + 1, kSlabNCThreads, slab, s, true, C, b.rgrid, tw, M,
                         (const double*)(b.partials + 5 * kMaxPartials), M * nch, b.acc, e_scale,
                         E_grid);
    }
    const int per_sm = nsm > 0 ? (kSlabCL * (M + 1) + nsm - 1) / nsm : 1;
    const size_t cl = smem_cap_per_sm(slabcl_layout(M).total, per_sm);
    auto kinvcl = dft_half_ok(M) ? k_slab_inv_cl<true> : k_slab_inv_cl<false>;
    e = cudaFuncSetAttribute(kinvcl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cl);
    if (e != cudaSuccess) return e;
    return launch_cluster(kinvcl, kSlabCL * (M + 1), kSlabThreads, cl, kSlabCL, s, true, C,
                          b.rgrid, tw, M, (const double*)(b.partials + 5 * kMaxPartials), M * nch,
                          b.acc, e_scale, E_grid);
}

bool fast_slab_gather_ok(int M) {
    int dev = 0, optin = 0;
    if (M < 2 || M > kFastMaxM || cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return false;
    return sg_smem_bytes(M) <= (size_t)optin;
}

cudaError_t fast_grid_energy(const KParams<float>& kp, const FastBufs& b, double e_scale,
                             double* E_out, cudaStream_t s) {
    const int Mh = kp.M / 2 + 1;
    const int nch = (Mh + kXpassKC - 1) / kXpassKC;
    return launch_ex(k_grid_energy, 1, kThreads, 0, s, true,
                     (const double*)(b.partials + 5 * kMaxPartials), kp.M * nch, b.acc, e_scale,
                     E_out);
}

template <int P>
cudaError_t fast_gather_slab_P(const KParams<float>& kp, const FastBufs& b, float* phi, float* F,
                               double* partials, unsigned* ticket, double e_scale, double* E_out,
                               const double* adj, cudaStream_t s) {
    const int M = kp.M, Mh = M / 2 + 1;
    const int nch = (Mh + kXpassKC - 1) / kXpassKC;
    const int nsm = sm_count();
    // at most ceil(2 (M + 1) / SMs) CTAs per SM, whatever else is resident
    // when the grid is scheduled early
    const int per_sm = nsm > 0 ? (kSlabCL * (M + 1) + nsm - 1) / nsm : 1;
    const size_t cl = smem_cap_per_sm(sg_smem_bytes(M), per_sm);
    const bool forces = F != nullptr || adj != nullptr;
    void (*kern)(const float2*, const float2*, const KParams<float>, const double*, int, Acc*, double,
                 double*, const f4*, const int*, int, const int*, const int*, const f4*, float4*) =
        forces ? k_sinv_gather_cl<P, true> : k_sinv_gather_cl<P, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cl);
    if (e != cudaSuccess) return e;
    e = launch_cluster(kern, kSlabCL * (M + 1), kSlabThreads, cl, kSlabCL, s, true,
                       (const float2*)b.cgrid, (const float2*)b.tw, kp,
                       (const double*)(b.partials + 5 * kMaxPartials), M * nch, b.acc, 0.0,
                       (double*)nullptr, (const f4*)b.bucket, (const int*)b.bucket_idx, b.cap,
                       (const int*)b.tile_n, (const int*)b.over_idx, (const f4*)b.wrapped,
                       (float4*)b.part);
    if (e != cudaSuccess) return e;
    const int blocks = std::max(1, std::min((kp.N + kThreads - 1) / kThreads, kMaxPartials));
    return launch_ex(k_gfinish<P>, blocks, kThreads, 0, s, true, (const float4*)b.part,
                     (const f4*)b.wrapped, phi, F, kp, partials, ticket, b.acc, e_scale, E_out, adj);
}

cudaError_t fast_gather_slab(const KParams<float>& kp, const FastBufs& b, float* phi, float* F,
                             double* partials, unsigned* ticket, double e_scale, double* E_out,
                             const double* adj, cudaStream_t s) {
    switch (kp.P) {
#define SE_CASE(PP) \
    case PP: return fast_gather_slab_P<PP>(kp, b, phi, F, partials, ticket, e_scale, E_out, adj, s);
        SE_FOR_EACH_P(SE_CASE)
#undef SE_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t fast_transform(const KParams<float>& kp, const FastBufs& b, double e_scale,
                           double* E_grid, cudaStream_t s, bool marks, void (*mark)(void*, int),
                           void* ctx, bool inverse) {
    const int M = kp.M, Mh = M / 2 + 1;
    const int nch = (Mh + kXpassKC - 1) / kXpassKC;
    const float2* tw = (const float2*)b.tw;
    float2* C = (float2*)b.cgrid;
    const int nsm = sm_count();
    cudaError_t e;
    // 2-CTA clusters per x-slab when every CTA gets an SM of its own;
    // otherwise one CTA per slab (a cap of two CTAs per SM would let an early
    // placement pack them onto half the SMs)
    const bool clusters = slab_clusters(M);
    // at least half an SM's shared memory: one slab CTA per SM, whatever else
    // is resident when the grid is scheduled early
    const size_t slab = std::max(slab_smem_bytes(M), kSlabSmemFloor);
    if (b.unsorted || !clusters) {
        if (b.unsorted) {
            auto kf = dft_half_ok(M) ? k_slab_fwd_f<true> : k_slab_fwd_f<false>;
            e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)slab);
            if (e != cudaSuccess) return e;
            e = launch_ex(kf, M, kSlabNCThreads, slab, s, true, (float*)b.g64, C, tw, M);
        } else {
            auto kfx = dft_half_ok(M) ? k_slab_fwd<true> : k_slab_fwd<false>;
            e = cudaFuncSetAttribute(kfx, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)slab);
            if (e != cudaSuccess) return e;
            e = launch_ex(kfx, M, kSlabNCThreads, slab, s, true, b.g64, C, tw, M,
                          (const Acc*)b.acc);
        }
    } else {
        // 2-CTA clusters per x-slab, at most ceil(2M / SMs) CTAs per SM
        const int per_sm = nsm > 0 ? (kSlabCL * M + nsm - 1) / nsm : 1;
        const size_t cl = smem_cap_per_sm(slabcl_layout(M).total, per_sm);
        auto kcl = dft_half_ok(M) ? k_slab_fwd_cl<true> : k_slab_fwd_cl<false>;
        e = cudaFuncSetAttribute(kcl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cl);
        if (e != cudaSuccess) return e;
        e = launch_cluster(kcl, kSlabCL * M, kSlabThreads, cl, kSlabCL, s, true,
                           b.g64, C, tw, M, (const Acc*)b.acc);
    }
    if (e != cudaSuccess) return e;
    if (marks) mark(ctx, 3);
    const float invM3 = (float)(1.0 / ((double)M * M * M));
    e = launch_ex(k_xpass, M * nch, kThreads, 0, s, true, C, tw, b.green_f, M, invM3,
                  b.partials + 5 * kMaxPartials);
    if (e != cudaSuccess) return e;
    if (marks) mark(ctx, 4);
    if (inverse) e = fast_inverse(kp, b, e_scale, E_grid, s);
    if (e != cudaSuccess) return e;
    if (marks) mark(ctx, 5);
    return cudaSuccess;
}

template <int P>
cudaError_t fast_gather_P(const KParams<float>& kp, const FastBufs& b, float* phi, float* F,
                          double* partials, unsigned* ticket, double e_scale, double* E_out,
                          const double* adj, cudaStream_t s) {
    const size_t R = (size_t)kp.tile + P - 1;
    const size_t bytes = R * R * (size_t)region_stride<P>((int)R) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_fgather<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bytes);
    if (e != cudaSuccess) return e;
    return launch_ex(k_fgather<P>, kp.ntiles + kOverflowBlocks, kThreads, bytes, s, true,
                     (const f4*)b.bucket, (const int*)b.bucket_idx, b.cap, (const int*)b.tile_n,
                     (const int*)b.over_idx, (const f4*)b.wrapped, (const float*)b.rgrid, phi, F,
                     kp, partials, ticket, b.acc, e_scale, E_out, adj);
}

// The tile gather pays when a tile's particles read many more grid values
// than its region holds (mean particles per tile x P^3 >= 8 x region): the
// region is then loaded once instead of every particle reading L2.  It needs
// the region within kTileGatherSmem and a CTA count within the energy
// partials' space.
bool fast_gather_tiled(const KParams<float>& kp) {
    const double R = (double)kp.tile + kp.P - 1;
    const double RS = kp.P <= 16 ? kp.P + 15 : R;   // region_stride
    const double per_tile = (double)kp.N / kp.ntiles;
    return R * R * RS * sizeof(float) <= (double)kTileGatherSmem &&
           kp.ntiles + kOverflowBlocks <= 4 * kMaxPartials &&
           per_tile * kp.P * kp.P * kp.P >= 8.0 * R * R * R;
}

cudaError_t fast_gather(const KParams<float>& kp, const FastBufs& b, float* phi, float* F,
                        double* partials, unsigned* ticket, double e_scale, double* E_out,
                        const double* adj, cudaStream_t s) {
    switch (kp.P) {
#define SE_CASE(PP) \
    case PP: return fast_gather_P<PP>(kp, b, phi, F, partials, ticket, e_scale, E_out, adj, s);
        SE_FOR_EACH_P(SE_CASE)
#undef SE_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t fast_to_real(const FastBufs& b, int M, float* dst, cudaStream_t s) {
    const long long n = (long long)M * M * M;
    const int blocks = (int)std::max(1LL, std::min((n + 255) / 256, 4096LL));
    return launch_ex(k_fx_to_real, blocks, kThreads, 0, s, false, (const long long*)b.g64, dst, n,
                     (const Acc*)b.acc);
}

template <int P>
cudaError_t gather_pdl_P(const f4* sorted, const int* perm, const float* grid, float* phi,
                         float* F, const KParams<float>& kp, double* partials, unsigned* ticket,
                         Acc* acc, double e_scale, double* E_out, const double* adj,
                         cudaStream_t s) {
    constexpr int GPW = 32 / (P / pick_d(P));
    const int gpb = (gather_threads<float, P>() / 32) * GPW;
    const int blocks = std::max(1, std::min((kp.N + gpb - 1) / gpb, kMaxPartials));
    return launch_ex(k_gather<float, P>, blocks, gather_threads<float, P>(), 0, s, true, sorted, perm, grid, phi, F,
                     kp, partials, ticket, acc, e_scale, E_out, adj);
}

cudaError_t launch_gather_pdl(const f4* sorted, const int* perm, const float* grid, float* phi,
                              float* F, const KParams<float>& kp, double* partials,
                              unsigned* ticket, Acc* acc, double e_scale, double* E_out,
                              const double* adj, cudaStream_t s) {
    switch (kp.P) {
#define SE_CASE(PP) \
    case PP: return gather_pdl_P<PP>(sorted, perm, grid, phi, F, kp, partials, ticket, acc, e_scale, E_out, adj, s);
        SE_FOR_EACH_P(SE_CASE)
#undef SE_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace se

#ifdef SE_TRACE
// Copy the phase stamps of the traced kernels to the host (build with -DSE_TRACE).
extern "C" int se_trace_read(unsigned long long* host, size_t bytes) {
    if (bytes < sizeof(se::se_trace_buf)) return -1;
    return cudaMemcpyFromSymbol(host, se::se_trace_buf, sizeof(se::se_trace_buf)) == cudaSuccess ? 0 : -2;
}
extern "C" int se_trace_clear(void) {
    static unsigned long long zero[se::kTraceKernels][se::kTraceBlocks][se::kTracePhases];
    return cudaMemcpyToSymbol(se::se_trace_buf, zero, sizeof(zero)) == cudaSuccess ? 0 : -2;
}
#endif
