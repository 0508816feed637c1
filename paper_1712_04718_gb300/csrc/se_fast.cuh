// se_fast.cuh -- the single-precision SE pipeline for grids up to 128^3:
// six short kernels chained by programmatic dependent launch, no cuFFT.
//
//   k_fbin      tile of each particle and a slot in the tile's bucket (a
//               fixed-capacity list; full buckets spill to an overflow list),
//               q sums and max |q|
//   k_fspread   Eq. 3.5, one CTA per tile: 32-bit fixed-point sums in shared
//               memory at a per-tile scale (one native 32-bit atomic per
//               weight), flushed exactly into the 64-bit fixed-point grid with
//               global integer reductions: the grid is the same for any order
//               of the additions; a few more CTAs add the overflow list with
//               global 64-bit atomics
//   k_slab_fwd  per x-slab: forward DFT along z (real to complex; the
//               fixed-point grid is converted to float here and cleared for
//               the next evaluation), then along y;
//               k_slab_fwd_cl the same on a 2-CTA cluster per slab
//   k_xpass     forward DFT along x, scaling by G(k)/M^3 (Eq. 3.6) with the
//               grid energy partials, inverse DFT along x
//   k_slab_inv  per x-slab: inverse DFT along y, then along z (complex to real);
//               one more CTA sums the grid energy; k_slab_inv_cl the same on a
//               2-CTA cluster per slab
//   (k_gather from se_kernels.cuh reads the real grid)
//
// Unsorted variant: k_fdirect replaces k_fbin and k_fspread by
// one kernel that adds every weight straight into a float grid with global
// reductions; k_slab_fwd_f reads that grid and clears it for the next call.
//
// The 1-D transforms (M <= 128) are small complex matrix products with
// register tiles (se_dft.cuh): the complex ones factored as M = M1 M2
// (Cooley-Tukey, two stages), the real-to-complex and complex-to-real ones
// direct; twiddles e^{-2 pi i r/M} from a table in shared memory.
#pragma once
#include <cooperative_groups.h>

#include <type_traits>

#include "se_dft.cuh"
#include "se_kernels.cuh"

namespace se {

constexpr int kFastKC = 8;        // spectrum columns per block in the y and x passes
#ifndef SE_XPASS_KC
#define SE_XPASS_KC 8
#endif
constexpr int kXpassKC = SE_XPASS_KC;   // kz columns per block of the single-system x pass
constexpr int kLoadBatch = 8;     // global loads per thread issued together in the transforms

// cudaLaunchKernelEx with programmatic stream serialization (pdl = true): the
// kernel may be scheduled while its predecessor drains and waits for that
// predecessor's results in griddepcontrol.wait.
template <typename... KArgs, typename... Args>
cudaError_t launch_ex(void (*kern)(KArgs...), int grid, int block, size_t smem, cudaStream_t s,
                      bool pdl, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = pdl ? attr : nullptr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// The same with a thread-block cluster of csize CTAs along x.
template <typename... KArgs, typename... Args>
cudaError_t launch_cluster(void (*kern)(KArgs...), int grid, int block, size_t smem, int csize,
                           cudaStream_t s, bool pdl, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 2 : 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// ---------------------------------------------------------------------------
// Tile buckets: particle slot s of tile t lives at bucket[t * cap + s].  The
// bin kernel takes a slot with an atomic on the tile's count and writes the
// particle there directly (no scan, no second pass); slots past cap go to an
// overflow list that the spread kernel adds with global fixed-point atomics
// (integer additions: the grid does not depend on their order).
template <typename T>
__global__ void __launch_bounds__(256)
k_fbin(const T* __restrict__ xyz, const T* __restrict__ q, const KParams<T> kp,
       int* __restrict__ tile_count, v4_t<T>* __restrict__ bucket, int* __restrict__ bucket_idx,
       int cap, int* __restrict__ over_idx, int* __restrict__ n_over, v4_t<T>* __restrict__ wrapped,
       double* __restrict__ partials) {
    SE_STAMP(0, 0);
    pdl_wait();
    pdl_launch_next();
    SE_STAMP(0, 1);
    __shared__ df2 sbuf[32];
    __shared__ int sbad;
    if (threadIdx.x == 0) sbad = 0;
    SE_STAMP(0, 2);
    df2 sq = df_from(0.0f), sa = df_from(0.0f);
    float qmax = 0.0f;
    int bad = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kp.N; i += gridDim.x * blockDim.x) {
        const T x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2], qq = q[i];
        if (!(isfinite(x) && isfinite(y) && isfinite(z) && isfinite(qq))) bad += 1;
        v4_t<T> v;
        v.x = wrap_coord(x, kp.L, kp.invL);
        v.y = wrap_coord(y, kp.L, kp.invL);
        v.z = wrap_coord(z, kp.L, kp.invL);
        v.w = qq;
        T t;
        const int cx = cell_of(v.x, kp.invh, kp.M, &t);
        const int cy = cell_of(v.y, kp.invh, kp.M, &t);
        const int cz = cell_of(v.z, kp.invh, kp.M, &t);
        const int tile = ((cx / kp.tile) * kp.nT + cy / kp.tile) * kp.nT + cz / kp.tile;
        const int s = atomicAdd(tile_count + tile, 1);
        if (s < cap) {
            bucket[(size_t)tile * cap + s] = v;
            bucket_idx[(size_t)tile * cap + s] = i;
        } else {
            const int o = atomicAdd(n_over, 1);
            if (o < kp.N) over_idx[o] = i;
        }
        wrapped[i] = v;
        sq = df_add(sq, df_from((float)qq));
        sa = df_add(sa, df_from(fabsf((float)qq)));
        qmax = fmaxf(qmax, fabsf((float)qq));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) qmax = fmaxf(qmax, __shfl_xor_sync(0xffffffffu, qmax, o));
    __shared__ unsigned smax;
    if (threadIdx.x == 0) smax = 0u;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) atomicMax(&smax, __float_as_uint(qmax));   // |q| >= 0: bits order as values
    SE_STAMP(0, 3);
    if (bad) atomicAdd(&sbad, bad);
    const df2 r0 = block_sum_df(sq, sbuf);
    const df2 r1 = block_sum_df(sa, sbuf);
    if (threadIdx.x == 0) {
        // per block: q sum (hi, lo), |q| sum (hi, lo), non-finite count, max |q|
        float* pf = reinterpret_cast<float*>(partials);
        pf[6 * blockIdx.x] = r0.hi;
        pf[6 * blockIdx.x + 1] = r0.lo;
        pf[6 * blockIdx.x + 2] = r1.hi;
        pf[6 * blockIdx.x + 3] = r1.lo;
        pf[6 * blockIdx.x + 4] = __int_as_float(sbad);
        pf[6 * blockIdx.x + 5] = __uint_as_float(smax);
        // the same maximum in a contiguous array, which every spread CTA reads
        reinterpret_cast<unsigned*>(partials + 3 * kMaxPartials)[blockIdx.x] = smax;
    }
    SE_STAMP(0, 4);
}

// Exclusive scan of n ints in shared memory (in place), by one block.
__device__ __forceinline__ void block_scan_smem(int* s, int n) {
    __shared__ int warp_tot[32];
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int b0 = min(n, (int)threadIdx.x * per), b1 = min(n, b0 + per);
    int local = 0;
    for (int k = b0; k < b1; ++k) local += s[k];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int nw = blockDim.x >> 5;
        int v = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
        }
        if (lane < nw) warp_tot[lane] = v;
    }
    __syncthreads();
    int run = incl - local + (warp > 0 ? warp_tot[warp - 1] : 0);
    for (int k = b0; k < b1; ++k) {
        int c = s[k];
        s[k] = run;
        run += c;
    }
    __syncthreads();
}

// Fixed-point scale 2^k for the spread: every weight is at most
// B = c_g max|q| (the Gaussian factors are <= 1), and k = 40 - ceil(log2 B)
// keeps each scaled weight below 2^40.  A sum of n weights stays below
// n 2^40, far inside 64 bits for any particle count.
__device__ __forceinline__ int fx_shift_for(double B) {
    if (!(B > 0.0) || !isfinite(B)) return 40;
    int e = (int)ceil(log2(B));
    int k = 40 - e;
    return k < -60 ? -60 : (k > 100 ? 100 : k);
}

// The same shift from a float bound, with integer operations only: for
// B = m 2^e (m in [0.5, 1)), ceil(log2 B) is e, or e - 1 when m = 0.5.
__device__ __forceinline__ int fx_shift_for_f(float B) {
    if (!(B > 0.0f) || !isfinite(B)) return 40;
    int e;
    const float m = frexpf(B, &e);
    const int k = 40 - (m == 0.5f ? e - 1 : e);
    return k < -60 ? -60 : (k > 100 ? 100 : k);
}

// A scaled weight v (float, |v| < 2^62) rounded to the nearest integer and
// split into the two 32-bit words of its 64-bit two's complement, with FP32
// and 32-bit integer operations only (no 64-bit conversion, which would run
// on the FP64 pipe).  |v| < 2^31: one float-to-int32 conversion, the high
// word is the sign.  |v| >= 2^31: v is already an integer and
// v = hf 2^32 + lf exactly, with hf = floor(v 2^-32) and 0 <= lf < 2^32 a
// multiple of v's ulp, so lf is exact in float.
__device__ __forceinline__ void fx_split(float v, unsigned* vh, unsigned* vl) {
    if (fabsf(v) < 2147483648.0f) {
        const int vi = __float2int_rn(v);
        *vl = (unsigned)vi;
        *vh = (unsigned)(vi >> 31);
    } else {
        const float hf = floorf(v * 2.3283064365386963e-10f);   // 2^-32
        const float lf = fmaf(-hf, 4294967296.0f, v);           // exact
        *vl = __float2uint_rn(lf);
        *vh = (unsigned)__float2int_rn(hf);
    }
}

// Row stride, in values, of a tile's region staged in shared memory (z
// fastest, rows of the region's extent in z): for supports up to 16 a
// compile-time P + 15, the extent of the largest tile edge used with them
// (16), so that in the unrolled support loops every row offset is an
// immediate of the load or atomic and only the plane step is an add; 0 (the
// region's own extent) for larger supports.  Tile edges are at most 16 when
// P <= 16 (the plan and the ensemble keep them there).
template <int P>
__host__ __device__ constexpr int region_pad() { return P <= 16 ? P + 15 : 0; }
template <int P>
__host__ __device__ constexpr int region_stride(int Rz) {
    return region_pad<P>() > 0 ? region_pad<P>() : Rz;
}

// Spread of one tile (Eq. 3.5) into the fixed-point grid g64 (scale fxs =
// 2^k): the n particles parts[0..n) of the tile.  The tile's region is
// accumulated in shared memory as one 32-bit integer per point at the scale
// 2^kt, kt = k - s, s = 10 + ceil(log2 n): every weight is at most
// B = c_g max|q| = 2^(40-k), so a point's sum is at most n B 2^kt <= 2^30 and
// cannot overflow; each weight is rounded once to an integer there (a
// quantum of n 2^-30 B at most) and added with one native 32-bit atomic, and
// the region is flushed exactly into the 64-bit grid by a shift of s bits.
// Integer additions: the grid does not depend on their order.  Called by one
// whole block (uniformly: the early return is per block).
template <int P>
// zeroed: the caller has cleared the first slab's region already; first:
// if non-null, this thread's group's first particle, loaded by the caller.
__device__ __forceinline__ void spread_tile(const f4* __restrict__ parts, int n,
                                            unsigned long long* __restrict__ g64,
                                            const KParams<float>& kp, float fxs, int slab,
                                            int tile, unsigned* acc, float* sE3,
                                            bool zeroed = false, const f4* first = nullptr) {
    constexpr int D = pick_d(P), G = P / D, GPW = 32 / G;
    if (n <= 0) return;
    if (threadIdx.x < P) sE3[threadIdx.x] = kp.E3[threadIdx.x];
    const int nT = kp.nT, M = kp.M, TT = kp.tile;
    const int tz = tile % nT, ty = (tile / nT) % nT, tx = tile / (nT * nT);
    const int t0x = tx * TT, t0y = ty * TT, t0z = tz * TT;
    const int Ry = min(TT, M - t0y) + P - 1, Rz = min(TT, M - t0z) + P - 1;
    const int Rx = min(TT, M - t0x) + P - 1;
    const int RS = region_stride<P>(Rz);   // row stride of the staged region
    const int plane = Ry * RS;
    const int shift = 10 + (n > 1 ? 32 - __clz(n - 1) : 0);   // 10 + ceil(log2 n)
    const float fxt = ldexpf(fxs, -shift);

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gi = lane / G, k = lane - gi * G;
    const bool act = gi < GPW;
    const int ngroups = (blockDim.x >> 5) * GPW;
    const int group = warp * GPW + gi;

    for (int s0 = 0; s0 < Rx; s0 += slab) {
        const int ns = min(slab, Rx - s0);
        const int nel = ns * plane;
        if (!(zeroed && s0 == 0))
            for (int e = threadIdx.x; e < nel; e += blockDim.x) acc[e] = 0u;
        __syncthreads();
        SE_STAMP(2, 2);
        if (act) {
            for (int p = group; p < n; p += ngroups) {
                f4 v;
                if (first && p == group) v = *first;
                else v = parts[p];
                float t;
                const int cx = cell_of(v.x, kp.invh, M, &t);
                const float ux = centre_offset(t, cx);
                const int cy = cell_of(v.y, kp.invh, M, &t);
                const float uy = centre_offset(t, cy);
                const int cz = cell_of(v.z, kp.invh, M, &t);
                const float uz = centre_offset(t, cz);
                const int lx = cx - t0x, ly = cy - t0y, lz = cz - t0z;
                const int alo = max(0, s0 - lx), ahi = min(P, s0 + ns - lx);
                if (alo >= ahi) continue;
                float gy[P];
                fgg<float, P>(uy, kp.beta, kp.E3, gy);
                float gz[D];
                const float qw = v.w * kp.qcg * fxt;
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    const float dz = float(k + j * G) - 0.5f * float(P - 1) - uz;
                    gz[j] = qw * expf(-kp.beta * dz * dz);
                }
                const float Bx = expf(2.0f * kp.beta * ux);
                float px = expf(-kp.beta * ux * (ux + float(P - 1)) + 2.0f * kp.beta * ux * float(alo));
                unsigned* row = acc + ((lx + alo - s0) * Ry + ly) * RS + lz + k;
                // small supports: the z factors folded into the y factors
                // (one multiply per weight); a running row pointer keeps the
                // address of each atomic to one add
                constexpr bool kFold = P * D <= 16;
                float gyz[kFold ? P * D : 1];
                if constexpr (kFold) {
#pragma unroll
                    for (int b = 0; b < P; ++b)
#pragma unroll
                        for (int j = 0; j < D; ++j) gyz[b * D + j] = gy[b] * gz[j];
                }
#pragma unroll 1
                for (int a = alo; a < ahi; ++a) {
                    const float gxa = px * sE3[a];
                    px *= Bx;
                    unsigned* rb = row;
#pragma unroll
                    for (int b = 0; b < P; ++b) {
                        if constexpr (kFold) {
#pragma unroll
                            for (int j = 0; j < D; ++j)
                                atomicAdd(rb + j * G, (unsigned)__float2int_rn(gxa * gyz[b * D + j]));
                        } else {
                            const float wab = gxa * gy[b];
#pragma unroll
                            for (int j = 0; j < D; ++j)
                                atomicAdd(rb + j * G, (unsigned)__float2int_rn(wab * gz[j]));
                        }
                        rb += RS;
                    }
                    row += plane;
                }
            }
        }
        __syncthreads();
        SE_STAMP(2, 3);
        const int ox = t0x - P / 2 + 1 + s0, oy = t0y - P / 2 + 1, oz = t0z - P / 2 + 1;
        const FDiv fRz = fdiv_of(Rz), fRy = fdiv_of(Ry);
        const int nlog = ns * Ry * Rz;   // the region's points, without the row padding
        for (int e = threadIdx.x; e < nlog; e += blockDim.x) {
            const int r = fdiv(e, fRz), rz = e - r * Rz;
            const int w = (int)acc[r * RS + rz];
            if (w != 0) {
                const int rx = fdiv(r, fRy), ry = r - rx * Ry;
                const int gx_ = wrap_index(ox + rx, M), gy_ = wrap_index(oy + ry, M),
                          gz_ = wrap_index(oz + rz, M);
                atomicAdd(g64 + ((size_t)gx_ * M + gy_) * M + gz_,
                          (unsigned long long)((long long)w << shift));
            }
        }
        __syncthreads();
        SE_STAMP(2, 4);
    }
}

// One particle's P^3 weights added straight into the fixed-point grid with
// 64-bit integer atomics (the overflow path of the tile buckets), by the G
// lanes of its group (lane k of the group: z points k, k + G, ...).
template <int P>
__device__ __forceinline__ void spread_particle_fx(const f4& v, unsigned long long* __restrict__ g64,
                                                   const KParams<float>& kp, float fxs,
                                                   const float* sE3, int k) {
    constexpr int D = pick_d(P), G = P / D;
    const int M = kp.M;
    float t;
    const int cx = cell_of(v.x, kp.invh, M, &t);
    const float ux = centre_offset(t, cx);
    const int cy = cell_of(v.y, kp.invh, M, &t);
    const float uy = centre_offset(t, cy);
    const int cz = cell_of(v.z, kp.invh, M, &t);
    const float uz = centre_offset(t, cz);
    float gy[P];
    fgg<float, P>(uy, kp.beta, kp.E3, gy);
    float gz[D];
    int jz[D];
    const float qw = v.w * kp.qcg * fxs;
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const int c = k + j * G;
        const float dz = float(c) - 0.5f * float(P - 1) - uz;
        gz[j] = qw * expf(-kp.beta * dz * dz);
        jz[j] = wrap_index(cz - P / 2 + 1 + c, M);
    }
    const float Bx = expf(2.0f * kp.beta * ux);
    float px = expf(-kp.beta * ux * (ux + float(P - 1)));
#pragma unroll 1
    for (int a = 0; a < P; ++a) {
        const float gxa = px * sE3[a];
        px *= Bx;
        const size_t plane = (size_t)wrap_index(cx - P / 2 + 1 + a, M) * M;
#pragma unroll
        for (int b = 0; b < P; ++b) {
            const float wab = gxa * gy[b];
            unsigned long long* row = g64 + (plane + wrap_index(cy - P / 2 + 1 + b, M)) * M;
#pragma unroll
            for (int j = 0; j < D; ++j) {
                unsigned vh, vl;
                fx_split(wab * gz[j], &vh, &vl);
                atomicAdd(row + jz[j], ((unsigned long long)vh << 32) | (unsigned long long)vl);
            }
        }
    }
}

constexpr int kOverflowBlocks = 8;   // CTAs after the tile CTAs, for the overflow list

// Spread (Eq. 3.5): CTA t < ntiles spreads tile t's bucket through shared
// memory; the last kOverflowBlocks CTAs add the overflow list with global
// atomics, and the last of them to finish clears the overflow count.  Every
// CTA takes the fixed-point scale from the bin kernel's per-block max |q|;
// CTA 0 also publishes the input checks and the scale for the transform.
template <int P>
__global__ void __launch_bounds__(256, P <= 8 ? 5 : 1)
k_fspread(const f4* __restrict__ bucket, int cap, int* __restrict__ tile_count,
          int* __restrict__ tile_n, const int* __restrict__ over_idx, int* __restrict__ n_over,
          const f4* __restrict__ wrapped, unsigned long long* __restrict__ g64,
          const KParams<float> kp, const double* __restrict__ partials, int nbin,
          unsigned* ticket, Acc* __restrict__ acc, int slab) {
    SE_STAMP(2, 0);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned* sacc = reinterpret_cast<unsigned*>(smem_raw);
    __shared__ float sE3[P];
    __shared__ float s_fxs;
    __shared__ int s_n;
    __shared__ unsigned s_qm;
    __shared__ df2 sbuf[32];
    // CTAs 0 .. kOverflowBlocks-1 take the overflow list (scheduled first,
    // they run beside the tiles); the others take tile blockIdx.x - kOverflowBlocks
    const int ovf = (int)blockIdx.x < kOverflowBlocks ? (int)blockIdx.x : -1;
    const int tile = ovf < 0 ? (int)blockIdx.x - kOverflowBlocks : kp.ntiles;
    // before the bin's results are needed: clear the first slab of this
    // tile's region and stage the Gaussian table (the CTA is scheduled early)
    if (ovf < 0) {
        const int nT = kp.nT, TT = kp.tile;
        const int ty = (tile / nT) % nT, tz = tile % nT, tx = tile / (nT * nT);
        const int plane = (min(TT, kp.M - ty * TT) + P - 1) *
                          region_stride<P>(min(TT, kp.M - tz * TT) + P - 1);
        const int nel = min(slab, min(TT, kp.M - tx * TT) + P - 1) * plane;
        for (int e = threadIdx.x; e < nel; e += blockDim.x) sacc[e] = 0u;
    }
    if (threadIdx.x < P) sE3[threadIdx.x] = kp.E3[threadIdx.x];
    if (threadIdx.x == 0) s_qm = 0u;
    pdl_wait();
    pdl_launch_next();
    SE_STAMP(2, 1);
    const float* pf = reinterpret_cast<const float*>(partials);
    // one round trip: max |q| of the bin blocks, this CTA's particle count,
    // and (speculatively: a bucket slot is always valid memory) the first
    // particle of this thread's group
    constexpr int G = P / pick_d(P), GPW = 32 / G;
    const int group = (threadIdx.x >> 5) * GPW + (threadIdx.x & 31) / G;
    f4 first;
    first.x = first.y = first.z = first.w = 0.f;
    if (ovf < 0 && group < cap) first = bucket[(size_t)tile * cap + group];
    unsigned m = 0u;
    const unsigned* qmax_b = reinterpret_cast<const unsigned*>(partials + 3 * kMaxPartials);
    for (int b = threadIdx.x; b < nbin; b += blockDim.x) m = max(m, __ldcg(qmax_b + b));
    int cnt = 0;
    if (threadIdx.x == blockDim.x - 1) cnt = ovf < 0 ? __ldcg(tile_count + tile) : __ldcg(n_over);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) atomicMax(&s_qm, m);
    if (threadIdx.x == blockDim.x - 1) {
        if (ovf < 0) {
            s_n = min(cnt, cap);
            tile_count[tile] = 0;   // consumed: clear for the next evaluation
        } else {
            s_n = min(cnt, kp.N);
        }
        tile_n[tile] = s_n;   // kept for the tile gather (the overflow count at ntiles)
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int k = fx_shift_for_f(kp.qcg * __uint_as_float(s_qm));
        s_fxs = ldexpf(1.0f, k);
        if (blockIdx.x == 0) {
            acc->fx_shift = k;
            acc->fx_scale = ldexpf(1.0f, k);
            acc->fx_inv = ldexpf(1.0f, -k);
        }
    }
    __syncthreads();
    if (blockIdx.x == 0) {
        const df2 a = sum_partials_df(pf, nbin, 3, 0, sbuf);
        const df2 b = sum_partials_df(pf, nbin, 3, 1, sbuf);
        int nbad = 0;
        for (int i = threadIdx.x; i < nbin; i += blockDim.x) nbad += __float_as_int(__ldcg(pf + 6 * i + 4));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) nbad += __shfl_xor_sync(0xffffffffu, nbad, o);
        __shared__ int sb;
        if (threadIdx.x == 0) sb = 0;
        __syncthreads();
        if ((threadIdx.x & 31) == 0 && nbad) atomicAdd(&sb, nbad);
        __syncthreads();
        if (threadIdx.x == 0) {
            acc->sum_q = df_to_double(a);
            acc->sum_absq = df_to_double(b);
            acc->nonfinite = (unsigned)sb;
        }
    }
    const float fxs = s_fxs;
    const int n = s_n;
    if (ovf < 0) {
        spread_tile<P>(bucket + (size_t)tile * cap, n, g64, kp, fxs, slab, tile, sacc, sE3, true,
                       &first);
        return;
    }
    constexpr int D = pick_d(P);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gi = lane / G, k = lane - gi * G;
    const int ngroups = kOverflowBlocks * (blockDim.x >> 5) * GPW;
    (void)D;
    if (gi < GPW) {
        for (int o = (ovf * (blockDim.x >> 5) + warp) * GPW + gi; o < n;
             o += ngroups)
            spread_particle_fx<P>(wrapped[over_idx[o]], g64, kp, fxs, sE3, k);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned t = atomicAdd(ticket, 1u);
        if (t == kOverflowBlocks - 1) {   // every overflow CTA has read the count
            *n_over = 0;
            *ticket = 0u;
        }
    }
}

// Gather (Eq. 3.9, Sec. 3.1) by tiles, for tiles that hold many particles:
// CTA t copies the real grid over tile t's region (the P-point supports of
// every particle of the tile) into shared memory once, then gathers the
// tile's bucket from it, with the arithmetic of k_gather in the same order;
// the last kOverflowBlocks CTAs gather the overflow list from the global
// grid.  The particles' factors are computed before the dependent-launch
// wait.  Outputs go to the particles' input positions; the energy
// 1/2 sum q phi is reduced as in k_gather.
template <int P, int DD = pick_d(P)>
struct TilePrep {
    static constexpr int D = DD;
    float gy[P], dgy[P], gz[D], dgz[D];
    float ux, uy, px0, Bx, q;
    int base;   // region offset of support point (0, 0, this lane's first z)
};

template <int P, int DD = pick_d(P)>
__device__ __forceinline__ void tile_prep(const f4& v, const KParams<float>& kp, int k, int t0x,
                                          int t0y, int t0z, int Ry, int Rz, TilePrep<P, DD>& g) {
    constexpr int D = DD, G = P / D;
    float t;
    const int cx = cell_of(v.x, kp.invh, kp.M, &t);
    g.ux = centre_offset(t, cx);
    const int cy = cell_of(v.y, kp.invh, kp.M, &t);
    const float uy = centre_offset(t, cy);
    const int cz = cell_of(v.z, kp.invh, kp.M, &t);
    const float uz = centre_offset(t, cz);
    fgg<float, P>(uy, kp.beta, kp.E3, g.gy);
    g.uy = uy;
#pragma unroll
    for (int b = 0; b < P; ++b) g.dgy[b] = (float(b) - 0.5f * float(P - 1) - uy) * g.gy[b];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const float dz = float(k + j * G) - 0.5f * float(P - 1) - uz;
        g.gz[j] = expf(-kp.beta * dz * dz);
        g.dgz[j] = dz * g.gz[j];
    }
    g.Bx = expf(2.0f * kp.beta * g.ux);
    g.px0 = expf(-kp.beta * g.ux * (g.ux + float(P - 1)));
    g.q = v.w;
    g.base = ((cx - t0x) * Ry + (cy - t0y)) * region_stride<P>(Rz) + (cz - t0z) + k;
}

template <int P, int DD = pick_d(P)>
__device__ __forceinline__ void tile_accum(const TilePrep<P, DD>& g, const float* reg, int Ry,
                                           int Rz, const float* sE3, float& vphi, float& vfx,
                                           float& vfy, float& vfz) {
    constexpr int D = DD, G = P / D;
    float acc0[D], accx[D], accy[D];
#pragma unroll
    for (int j = 0; j < D; ++j) acc0[j] = accx[j] = accy[j] = 0.0f;
    float px = g.px0;
    const int RS = region_stride<P>(Rz);
    const int plane = Ry * RS;
#pragma unroll(P <= 8 ? P : 1)
    for (int a = 0; a < P; ++a) {
        const float gxa = px * sE3[a];
        const float dgxa = (float(a) - 0.5f * float(P - 1) - g.ux) * gxa;
        px *= g.Bx;
        const float* rb = reg + g.base + a * plane;   // running row pointer: one add per row
        float tb0[D], tby[D];
#pragma unroll
        for (int j = 0; j < D; ++j) tb0[j] = tby[j] = 0.0f;
#pragma unroll
        for (int b = 0; b < P; ++b) {
#pragma unroll
            for (int j = 0; j < D; ++j) {
                const float hv = rb[j * G];
                tb0[j] += g.gy[b] * hv;
                tby[j] += g.dgy[b] * hv;
            }
            rb += RS;
        }
#pragma unroll
        for (int j = 0; j < D; ++j) {
            acc0[j] += gxa * tb0[j];
            accx[j] += dgxa * tb0[j];
            accy[j] += gxa * tby[j];
        }
    }
#pragma unroll
    for (int j = 0; j < D; ++j) {
        vphi += g.gz[j] * acc0[j];
        vfx += g.gz[j] * accx[j];
        vfy += g.gz[j] * accy[j];
        vfz += g.dgz[j] * acc0[j];
    }
}

// Copy the grid over a tile region (origin o = tile origin - P/2 + 1, extent
// Rx x Ry x Rz, wrapped periodically) into shared memory, rows RS values
// apart (RS >= Rz); the whole block.
__device__ __forceinline__ void load_region(const float* __restrict__ grid, int M, int ox, int oy,
                                            int oz, int Rx, int Ry, int Rz, int RS, float* reg) {
    const int nel = Rx * Ry * Rz;
    const FDiv fRz = fdiv_of(Rz), fRy = fdiv_of(Ry);
    for (int e0 = threadIdx.x; e0 < nel; e0 += blockDim.x * kLoadBatch) {
        float v[kLoadBatch];
#pragma unroll
        for (int u = 0; u < kLoadBatch; ++u) {
            const int e = e0 + u * (int)blockDim.x;
            if (e < nel) {
                const int r = fdiv(e, fRz), rz = e - r * Rz;
                const int rx = fdiv(r, fRy), ry = r - rx * Ry;
                v[u] = __ldg(grid + ((size_t)wrap_index(ox + rx, M) * M + wrap_index(oy + ry, M)) * M +
                             wrap_index(oz + rz, M));
            }
        }
#pragma unroll
        for (int u = 0; u < kLoadBatch; ++u) {
            const int e = e0 + u * (int)blockDim.x;
            if (e < nel) {
                const int r = fdiv(e, fRz);
                reg[r * RS + (e - r * Rz)] = v[u];
            }
        }
    }
}

// Sum over the G lanes of a particle, then lane 0 of the group writes phi and
// F at the particle's input position and adds q phi to the energy.
template <int P, int G = P / pick_d(P)>
__device__ __forceinline__ void gather_emit(int k, bool valid, int orig, float qq, float vphi,
                                            float vfx, float vfy, float vfz,
                                            const KParams<float>& kp, float* __restrict__ phi,
                                            float* __restrict__ F, float phi_mul, float F_mul,
                                            df2& e_df) {
#pragma unroll
    for (int o = 1; o < G; o <<= 1) {
        const float a0 = __shfl_down_sync(0xffffffffu, vphi, o);
        const float a1 = __shfl_down_sync(0xffffffffu, vfx, o);
        const float a2 = __shfl_down_sync(0xffffffffu, vfy, o);
        const float a3 = __shfl_down_sync(0xffffffffu, vfz, o);
        if (k + o < G) {
            vphi += a0;
            vfx += a1;
            vfy += a2;
            vfz += a3;
        }
    }
    if (valid && k == 0) {
        const float ph = vphi * kp.phi_scale;
        const float fs = qq * kp.F_scale;
        if (phi) phi[orig] = ph * phi_mul;
        if (F) {
            const float fm = fs * F_mul;
            F[3 * orig] = fm * vfx;
            F[3 * orig + 1] = fm * vfy;
            F[3 * orig + 2] = fm * vfz;
        }
        e_df = df_add(e_df, df_from(qq * ph));
    }
}

template <int P>
__global__ void __launch_bounds__(256, P <= 8 ? 4 : 1)
k_fgather(const f4* __restrict__ bucket, const int* __restrict__ bucket_idx, int cap,
          const int* __restrict__ tile_n, const int* __restrict__ over_idx,
          const f4* __restrict__ wrapped, const float* __restrict__ grid, float* __restrict__ phi,
          float* __restrict__ F, const KParams<float> kp, double* __restrict__ partials,
          unsigned* ticket, Acc* acc, double e_scale, double* E_out,
          const double* __restrict__ adj) {
    constexpr int D = pick_d(P), G = P / D, GPW = 32 / G;
    SE_STAMP(6, 0);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* reg = reinterpret_cast<float*>(smem_raw);
    __shared__ float sE3[P];
    __shared__ df2 sbuf[32];
    if (threadIdx.x < P) sE3[threadIdx.x] = kp.E3[threadIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gi = lane / G, k = lane - gi * G;
    const int group = warp * GPW + gi, ngroups = (blockDim.x >> 5) * GPW;
    const int ovf = (int)blockIdx.x < kOverflowBlocks ? (int)blockIdx.x : -1;   // as k_fspread
    const int tile = ovf < 0 ? (int)blockIdx.x - kOverflowBlocks : kp.ntiles;
    const int M = kp.M;
    // the buckets, their counts and the overflow list were written before the
    // transforms began: the first particle's factors are computed while the
    // grid is still being produced (before the dependent-launch wait)
    const int n = tile_n[tile];
    df2 e_df = df_from(0.0f);
    const float gsc = adj ? (float)__ldg(adj) : 1.0f;
    const float phi_mul = gsc, F_mul = adj ? -gsc : 1.0f;
    if (ovf < 0) {
        const int nT = kp.nT, TT = kp.tile;
        const int t0x = (tile / (nT * nT)) * TT, t0y = ((tile / nT) % nT) * TT, t0z = (tile % nT) * TT;
        const int Rx = min(TT, M - t0x) + P - 1, Ry = min(TT, M - t0y) + P - 1,
                  Rz = min(TT, M - t0z) + P - 1;
        TilePrep<P> tp;
        int orig = -1;
        if (gi < GPW && group < n) {
            tile_prep<P>(bucket[(size_t)tile * cap + group], kp, k, t0x, t0y, t0z, Ry, Rz, tp);
            orig = bucket_idx[(size_t)tile * cap + group];
        }
        pdl_wait();
        SE_STAMP(6, 1);
        load_region(grid, M, t0x - P / 2 + 1, t0y - P / 2 + 1, t0z - P / 2 + 1, Rx, Ry, Rz,
                    region_stride<P>(Rz), reg);
        __syncthreads();
        SE_STAMP(6, 2);
        for (int p0 = 0; p0 < n; p0 += ngroups) {
            const int p = p0 + group;
            const bool valid = gi < GPW && p < n;
            float vphi = 0.0f, vfx = 0.0f, vfy = 0.0f, vfz = 0.0f;
            if (valid) {
                if (p0 != 0) {
                    tile_prep<P>(bucket[(size_t)tile * cap + p], kp, k, t0x, t0y, t0z, Ry, Rz, tp);
                    orig = bucket_idx[(size_t)tile * cap + p];
                }
                tile_accum<P>(tp, reg, Ry, Rz, sE3, vphi, vfx, vfy, vfz);
            }
            gather_emit<P>(k, valid, orig, tp.q, vphi, vfx, vfy, vfz, kp, phi, F, phi_mul, F_mul, e_df);
        }
    } else {
        const int first = ovf * ngroups;   // this CTA's share of the list
        const int stride = kOverflowBlocks * ngroups;
        GatherPrep<float, P> gp;
        float qq = 0.0f;
        int orig = -1;
        if (gi < GPW && first + group < n) {
            orig = over_idx[first + group];
            const f4 v = wrapped[orig];
            qq = v.w;
            gather_prep<float, P>(v, kp, k, gp);
        }
        pdl_wait();
        SE_STAMP(6, 1);
        for (int o0 = first; o0 < n; o0 += stride) {
            const int o = o0 + group;
            const bool valid = gi < GPW && o < n;
            float vphi = 0.0f, vfx = 0.0f, vfy = 0.0f, vfz = 0.0f;
            if (valid) {
                if (o0 != first) {
                    orig = over_idx[o];
                    const f4 v = wrapped[orig];
                    qq = v.w;
                    gather_prep<float, P>(v, kp, k, gp);
                }
                gather_accum<float, P>(gp, grid, kp, sE3, vphi, vfx, vfy, vfz);
            }
            gather_emit<P>(k, valid, orig, qq, vphi, vfx, vfy, vfz, kp, phi, F, phi_mul, F_mul, e_df);
        }
    }
    SE_STAMP(6, 3);
    float* pf = reinterpret_cast<float*>(partials);
    const df2 r = block_sum_df(e_df, sbuf);
    SE_STAMP(6, 4);
    if (threadIdx.x == 0) {
        pf[2 * blockIdx.x] = r.hi;
        pf[2 * blockIdx.x + 1] = r.lo;
    }
    const bool lastb = last_block(ticket);
    SE_STAMP(6, 5);
    if (!lastb || threadIdx.x >= 32) return;
    const df2 t = warp_sum_partials_df(pf, gridDim.x, 1, 0);
    SE_STAMP(6, 6);
    if (threadIdx.x == 0) {
        const double sum = df_to_double(t);
        acc->e_gather = sum;
        if (E_out) *E_out = e_scale * sum;
        *ticket = 0u;
    }
}

// Unsorted spread (Eq. 3.5) in one kernel: a group of G lanes takes one
// particle (in input order) and adds its P^3 weights q c_g e^{-alpha r^2}
// into the float grid with global reductions, so that the last bits of the
// grid depend on the order in which the additions land.  The grid must be
// zero on entry.  Also writes every particle's wrapped (x, y, z, q) for the
// gather, and the input checks (q sums, non-finite count) through a
// last-block reduction.
template <int P>
__global__ void __launch_bounds__(256)
k_fdirect(const float* __restrict__ xyz, const float* __restrict__ q, const KParams<float> kp,
          float* __restrict__ grid, f4* __restrict__ wrapped, double* __restrict__ partials,
          unsigned* ticket, Acc* acc) {
    constexpr int D = pick_d(P), G = P / D, GPW = 32 / G;
    SE_STAMP(2, 0);
    pdl_wait();
    pdl_launch_next();
    SE_STAMP(2, 1);
    __shared__ float sE3[P];
    __shared__ df2 sbuf[32];
    __shared__ int sbad;
    if (threadIdx.x < P) sE3[threadIdx.x] = kp.E3[threadIdx.x];
    if (threadIdx.x == 0) sbad = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gi = lane / G, k = lane - gi * G;
    const int gpb = (blockDim.x >> 5) * GPW;
    const int M = kp.M;
    df2 sq = df_from(0.0f), sa = df_from(0.0f);
    int bad = 0;
    // group g of CTA b takes particles b + gridDim.x g + (all groups) i: the
    // particles of one CTA (and of one warp) lie far apart in the input order,
    // so that neighbouring particles, whose weights land on the same grid
    // points, do not queue on the same addresses at the same time
    const int ngroups = gridDim.x * gpb;
    for (int p = (warp * GPW + gi) * gridDim.x + blockIdx.x; gi < GPW && p < kp.N; p += ngroups) {
        const float x = xyz[3 * p], y = xyz[3 * p + 1], z = xyz[3 * p + 2], qq = q[p];
        f4 v;
        v.x = wrap_coord(x, kp.L, kp.invL);
        v.y = wrap_coord(y, kp.L, kp.invL);
        v.z = wrap_coord(z, kp.L, kp.invL);
        v.w = qq;
        if (k == 0) {
            wrapped[p] = v;
            if (!(isfinite(x) && isfinite(y) && isfinite(z) && isfinite(qq))) bad += 1;
            sq = df_add(sq, df_from(qq));
            sa = df_add(sa, df_from(fabsf(qq)));
        }
        float t;
        const int cx = cell_of(v.x, kp.invh, M, &t);
        const float ux = centre_offset(t, cx);
        const int cy = cell_of(v.y, kp.invh, M, &t);
        const float uy = centre_offset(t, cy);
        const int cz = cell_of(v.z, kp.invh, M, &t);
        const float uz = centre_offset(t, cz);
        float gy[P];
        int jy[P];
        fgg<float, P>(uy, kp.beta, kp.E3, gy);
#pragma unroll
        for (int b = 0; b < P; ++b) jy[b] = wrap_index(cy - P / 2 + 1 + b, M) * M;
        float gz[D];
        int jz[D];
        const float qw = qq * kp.qcg;
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const int c = k + j * G;
            const float dz = float(c) - 0.5f * float(P - 1) - uz;
            gz[j] = qw * expf(-kp.beta * dz * dz);
            jz[j] = wrap_index(cz - P / 2 + 1 + c, M);
        }
        const float Bx = expf(2.0f * kp.beta * ux);
        float px = expf(-kp.beta * ux * (ux + float(P - 1)));
#pragma unroll(P <= 8 ? P : 1)
        for (int a = 0; a < P; ++a) {
            const float gxa = px * sE3[a];
            px *= Bx;
            float* plane = grid + (size_t)wrap_index(cx - P / 2 + 1 + a, M) * M * M;
#pragma unroll
            for (int b = 0; b < P; ++b) {
                const float wab = gxa * gy[b];
                float* row = plane + jy[b];
#pragma unroll
                for (int j = 0; j < D; ++j) atomicAdd(row + jz[j], wab * gz[j]);
            }
        }
    }
    SE_STAMP(2, 2);
    if (bad) atomicAdd(&sbad, bad);
    const df2 r0 = block_sum_df(sq, sbuf);
    const df2 r1 = block_sum_df(sa, sbuf);
    float* pf = reinterpret_cast<float*>(partials);
    if (threadIdx.x == 0) {
        pf[6 * blockIdx.x] = r0.hi;
        pf[6 * blockIdx.x + 1] = r0.lo;
        pf[6 * blockIdx.x + 2] = r1.hi;
        pf[6 * blockIdx.x + 3] = r1.lo;
        pf[6 * blockIdx.x + 4] = __int_as_float(sbad);
    }
    if (!last_block(ticket)) return;
    const df2 a = sum_partials_df(pf, gridDim.x, 3, 0, sbuf);
    const df2 b = sum_partials_df(pf, gridDim.x, 3, 1, sbuf);
    __syncthreads();
    if (threadIdx.x == 0) sbad = 0;
    __syncthreads();
    int nbad = 0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) nbad += __float_as_int(__ldcg(pf + 6 * i + 4));
    if (nbad) atomicAdd(&sbad, nbad);
    __syncthreads();
    if (threadIdx.x == 0) {
        acc->sum_q = df_to_double(a);
        acc->sum_absq = df_to_double(b);
        acc->nonfinite = (unsigned)sbad;
        *ticket = 0u;
    }
    SE_STAMP(2, 3);
}

// ---------------------------------------------------------------------------
// The 3-D transform in three kernels.  tw[r] = (cos, sin)(2 pi r / M); the
// forward transform uses e^{-i}, the inverse e^{+i}; both unnormalised.
//   k_slab_fwd  per x-slab: z real-to-complex, then y      (C[x][ky][kz])
//   k_xpass     per (ky, kz-chunk): x forward, G(k)/M^3 and the grid energy,
//               x inverse
//   k_slab_inv  per x-slab: y inverse, then z complex-to-real (R[x][y][z])

constexpr int kSlabThreads = 512;
// threads of the single-system slab CTAs that take a whole x-slab each
// (grids too large for one 2-CTA cluster per slab on every SM)
#ifndef SE_SLAB_NC_THREADS
#define SE_SLAB_NC_THREADS 1024
#endif
constexpr int kSlabNCThreads = SE_SLAB_NC_THREADS;

__device__ __forceinline__ void load_twiddles(float2* tw, const float2* __restrict__ tw_g, int M) {
    for (int i = threadIdx.x; i < M; i += blockDim.x) tw[i] = tw_g[i];
}

// shared memory of the slab kernels: tw[M] | A: M x (M+1) floats, or the
// M x Mh complex slab | T: Mh x (M+1) complex | Z: M x Mh complex (scratch
// of the factored DFTs)
__host__ __device__ inline size_t slab_a_bytes(int M) {
    const size_t Mh = M / 2 + 1, SP = M + 1;
    const size_t a = (size_t)M * SP * sizeof(float), c = (size_t)M * Mh * sizeof(float2);
    return ((a > c ? a : c) + 15) / 16 * 16;
}
__host__ __device__ inline size_t slab_t_bytes(int M) {
    const size_t Mh = M / 2 + 1, SP = M + 1;
    return Mh * SP * sizeof(float2);
}
__host__ __device__ inline size_t slab_smem_bytes(int M) {
    const size_t Mh = M / 2 + 1;
    return (size_t)M * sizeof(float2) + slab_a_bytes(M) + slab_t_bytes(M) +
           (size_t)M * Mh * sizeof(float2);
}

// Forward 2-D transform (z real-to-complex, then y) of x-slab x.  The input
// is the fixed-point grid (long long, scaled by inv), or the float grid of
// the unsorted spread (float), which is cleared after it is read.
// HM: the z transform's form, 0 direct, 1 half-length, 2 chosen at run time
// (dft_half_ok with the threshold half_r4: the ensemble's many grid sizes).
template <typename G, bool kClear = (sizeof(G) == sizeof(float)), int HM = 2>
__device__ __forceinline__ void slab_fwd_body(G* __restrict__ grid, float2* __restrict__ C,
                                              const float2* __restrict__ tw_g, int M, float inv,
                                              int x, unsigned char* sm, int half_r4 = kDftHalfR4) {
    const int Mh = M / 2 + 1, SP = M + 1;
    float2* tw = reinterpret_cast<float2*>(sm);
    float* S = reinterpret_cast<float*>(sm + (size_t)M * sizeof(float2));
    float2* T = reinterpret_cast<float2*>(sm + (size_t)M * sizeof(float2) + slab_a_bytes(M));
    float2* Z = reinterpret_cast<float2*>(sm + (size_t)M * sizeof(float2) + slab_a_bytes(M) +
                                          slab_t_bytes(M));
    load_twiddles(tw, tw_g, M);
    G* src = grid + (size_t)x * M * M;
    const FDiv fM = fdiv_of(M);
    // kLoadBatch loads per thread in flight before any is used
    for (int e0 = threadIdx.x; e0 < M * M; e0 += blockDim.x * kLoadBatch) {
        std::remove_const_t<G> v[kLoadBatch];
#pragma unroll
        for (int u = 0; u < kLoadBatch; ++u) {
            const int e = e0 + u * (int)blockDim.x;
            v[u] = e < M * M ? src[e] : 0;
        }
#pragma unroll
        for (int u = 0; u < kLoadBatch; ++u) {
            const int e = e0 + u * (int)blockDim.x;
            if (e >= M * M) break;
            const int y = fdiv(e, fM), z = e - y * M;
            if constexpr (sizeof(G) == sizeof(float)) {
                S[y * SP + z] = v[u];
                src[e] = 0.0f;
            } else {
                // int64 -> float through its two 32-bit words (no 64-bit conversion)
                const unsigned long long w = (unsigned long long)v[u];
                const float hi = (float)(int)(w >> 32), lo = (float)(unsigned)(w & 0xffffffffull);
                S[y * SP + z] = fmaf(hi, 4294967296.0f, lo) * inv;
                if constexpr (kClear) src[e] = 0;
            }
        }
    }
    __syncthreads();
    SE_STAMP(3, 2);
    // z, real to complex: X(j = z, c = y) = S[y][z]  ->  T[kz][y] (through Z
    // and the dead S when M/2 factors)
    if (HM == 1 || (HM == 2 && dft_half_ok(M, half_r4)))
        dft_r2c_half<2, 2>(S, 1, SP, T, SP, 1, M, Z, reinterpret_cast<float2*>(S), tw, M);
    else
        dft_r2c<2, 2>(S, 1, SP, T, SP, 1, M, Mh, M, tw, M);
    __syncthreads();
    SE_STAMP(3, 3);
    // y forward: X(j = y, c = kz) = T[kz][y]  ->  C[x][ky][kz]
    dft_c2c_fact(T, 1, SP, C + (size_t)x * M * Mh, Mh, 1, Mh, Z, tw, M, -1.0f);
    SE_STAMP(3, 4);
}

#ifndef SE_BATCH_TU
template <bool kHalf>
__global__ void __launch_bounds__(kSlabNCThreads)
k_slab_fwd(long long* __restrict__ g64, float2* __restrict__ C,
           const float2* __restrict__ tw_g, int M, const Acc* __restrict__ acc) {
    SE_STAMP(3, 0);
    pdl_wait();
    pdl_launch_next();
    SE_STAMP(3, 1);
    extern __shared__ __align__(16) unsigned char sm[];
    slab_fwd_body<long long, true, kHalf ? 1 : 0>(g64, C, tw_g, M, acc->fx_inv, blockIdx.x, sm);   // clears the grid
}

// the same on the float grid of the unsorted spread (cleared after reading)
template <bool kHalf>
__global__ void __launch_bounds__(kSlabNCThreads)
k_slab_fwd_f(float* __restrict__ grid, float2* __restrict__ C, const float2* __restrict__ tw_g,
             int M) {
    SE_STAMP(3, 0);
    pdl_wait();
    pdl_launch_next();
    SE_STAMP(3, 1);
    extern __shared__ __align__(16) unsigned char sm[];
    slab_fwd_body<float, true, kHalf ? 1 : 0>(grid, C, tw_g, M, 1.0f, blockIdx.x, sm);
}
#endif  // SE_BATCH_TU

// x pass of work item `item` = (ky, kz chunk): forward DFT along x, scaling
// by G/M^3 with the grid energy (returned, valid in thread 0), inverse DFT.
template <int KC = kFastKC>
__device__ __forceinline__ df2 xpass_body(float2* __restrict__ C, const float2* __restrict__ tw_g,
                                          const float* __restrict__ green, int M, float invM3,
                                          int item) {
    __shared__ float2 tw[kFastMaxM];
    __shared__ float2 s[kFastMaxM * KC];
    __shared__ float2 s2[kFastMaxM * KC];
    __shared__ float2 s3[kFastMaxM * KC];   // scratch of the factored DFTs
    __shared__ df2 sbuf[32];
    const int Mh = M / 2 + 1;
    const int nch = (Mh + KC - 1) / KC;
    const int y = item / nch, c0 = (item % nch) * KC;
    const int nc = min(KC, Mh - c0);
    const FDiv fnc = fdiv_of(nc);
    load_twiddles(tw, tw_g, M);
    for (int e0 = threadIdx.x; e0 < M * nc; e0 += blockDim.x * kLoadBatch) {
        float2 v[kLoadBatch];
#pragma unroll
        for (int u = 0; u < kLoadBatch; ++u) {
            const int e = e0 + u * (int)blockDim.x;
            if (e < M * nc) {
                const int x = fdiv(e, fnc), kk = e - x * nc;
                v[u] = C[((size_t)x * M + y) * Mh + c0 + kk];
            }
        }
#pragma unroll
        for (int u = 0; u < kLoadBatch; ++u) {
            const int e = e0 + u * (int)blockDim.x;
            if (e < M * nc) {
                const int x = fdiv(e, fnc), kk = e - x * nc;
                s[x * KC + kk] = v[u];
            }
        }
    }
    __syncthreads();
    SE_STAMP(4, 2);
    dft_c2c_fact<1, 2>(s, KC, 1, s2, KC, 1, nc, s3, tw, M, -1.0f);
    __syncthreads();
    SE_STAMP(4, 3);
    df2 en = df_from(0.0f);   // double-float energy sum
    for (int e = threadIdx.x; e < M * nc; e += blockDim.x) {
        const int kx = fdiv(e, fnc), kk = e - kx * nc;
        const int kz = c0 + kk;
        const float2 v = s2[kx * KC + kk];
        const float g = green[((size_t)kx * M + y) * Mh + kz];
        en = df_add(en, df_from(((kz == 0 || 2 * kz == M) ? 1.0f : 2.0f) * g *
                                fmaf(v.x, v.x, v.y * v.y)));
        const float f = g * invM3;
        s2[kx * KC + kk] = make_float2(v.x * f, v.y * f);
    }
    __syncthreads();
    dft_c2c_fact<1, 2>(s2, KC, 1, C + (size_t)y * Mh + c0, M * Mh, 1, nc, s3, tw, M, 1.0f);
    SE_STAMP(4, 4);
    return block_sum_df(en, sbuf);
}

#ifndef SE_BATCH_TU
// Each CTA leaves its grid-energy partial (a double-float pair); the sum is
// taken by an extra CTA of k_slab_inv, off the critical path.
__global__ void __launch_bounds__(256)
k_xpass(float2* __restrict__ C, const float2* __restrict__ tw_g, const float* __restrict__ green,
        int M, float invM3, double* __restrict__ partials) {
    SE_STAMP(4, 0);
    pdl_wait();
    pdl_launch_next();
    SE_STAMP(4, 1);
    const df2 tot = xpass_body<kXpassKC>(C, tw_g, green, M, invM3, blockIdx.x);
    float* pf = reinterpret_cast<float*>(partials);
    if (threadIdx.x == 0) {
        pf[2 * blockIdx.x] = tot.hi;
        pf[2 * blockIdx.x + 1] = tot.lo;
    }
    SE_STAMP(4, 5);
}
#endif  // SE_BATCH_TU

// Inverse 2-D transform (y, then z complex-to-real) of x-slab x into R (HM
// as for slab_fwd_body).
template <int HM = 2>
__device__ __forceinline__ void slab_inv_body(const float2* __restrict__ C, float* __restrict__ R,
                                              const float2* __restrict__ tw_g, int M, int x,
                                              unsigned char* sm, int half_r4 = kDftHalfR4) {
    const int Mh = M / 2 + 1, SP = M + 1;
    float2* tw = reinterpret_cast<float2*>(sm);
    float* S = reinterpret_cast<float*>(sm + (size_t)M * sizeof(float2));
    float2* A = reinterpret_cast<float2*>(S);   // the slab, before S is needed
    float2* T = reinterpret_cast<float2*>(sm + (size_t)M * sizeof(float2) + slab_a_bytes(M));
    float2* Z = reinterpret_cast<float2*>(sm + (size_t)M * sizeof(float2) + slab_a_bytes(M) +
                                          slab_t_bytes(M));
    load_twiddles(tw, tw_g, M);
    const float2* src = C + (size_t)x * M * Mh;
    for (int e0 = threadIdx.x; e0 < M * Mh; e0 += blockDim.x * kLoadBatch) {
        float2 v[kLoadBatch];
#pragma unroll
        for (int u = 0; u < kLoadBatch; ++u) {
            const int e = e0 + u * (int)blockDim.x;
            if (e < M * Mh) v[u] = src[e];
        }
#pragma unroll
        for (int u = 0; u < kLoadBatch; ++u) {
            const int e = e0 + u * (int)blockDim.x;
            if (e < M * Mh) A[e] = v[u];
        }
    }
    __syncthreads();
    // y inverse: X(j = ky, c = kz) = A[ky][kz]  ->  T[kz][y], with the
    // Hermitian weights of the z real transform (1 at kz = 0 and M/2, else 2)
    dft_c2c_fact(A, Mh, 1, T, 1, SP, Mh, Z, tw, M, 1.0f);
    __syncthreads();
    SE_STAMP(5, 2);
    const FDiv fM = fdiv_of(M);
    if (HM == 1 || (HM == 2 && dft_half_ok(M, half_r4))) {
        // z complex to real through Z and S (the Hermitian symmetry of the
        // half-length form takes the place of the weights)
        dft_c2r_half<2, 2>(T, SP, 1, S, 1, SP, M, Z, reinterpret_cast<float2*>(S), tw, M, 1.0f);
    } else {
        for (int e = threadIdx.x; e < Mh * M; e += blockDim.x) {
            const int kz = fdiv(e, fM), y = e - kz * M;
            if (kz != 0 && 2 * kz != M) {
                float2 v = T[kz * SP + y];
                T[kz * SP + y] = make_float2(2.f * v.x, 2.f * v.y);
            }
        }
        __syncthreads();
        // z complex to real: X(j = kz, c = y) = T[kz][y]  ->  S[y][z]
        dft_c2r<2, 2>(T, SP, 1, S, 1, SP, Mh, M, M, tw, M);
    }
    __syncthreads();
    SE_STAMP(5, 3);
    float* dst = R + (size_t)x * M * M;
    for (int e = threadIdx.x; e < M * M; e += blockDim.x) {
        const int y = fdiv(e, fM), z = e - y * M;
        dst[e] = S[y * SP + z];
    }
    SE_STAMP(5, 4);
}

#ifndef SE_BATCH_TU
// CTAs 0..M-1: the inverse slab transforms; CTA M: the grid energy from the
// x pass's nparts partials (acc->e_grid and, scaled, *E_out).
template <bool kHalf>
__global__ void __launch_bounds__(kSlabNCThreads)
k_slab_inv(const float2* __restrict__ C, float* __restrict__ R, const float2* __restrict__ tw_g,
           int M, const double* __restrict__ xparts, int nparts, Acc* acc, double e_scale,
           double* E_out) {
    SE_STAMP(5, 0);
    pdl_wait();
    pdl_launch_next();
    SE_STAMP(5, 1);
    if ((int)blockIdx.x == M) {
        __shared__ df2 sbuf[32];
        const df2 sum = sum_partials_df(reinterpret_cast<const float*>(xparts), nparts, 1, 0, sbuf);
        if (threadIdx.x == 0) {
            const double e = df_to_double(sum);
            acc->e_grid = e;
            if (E_out) *E_out = e_scale * e;
        }
        return;
    }
    extern __shared__ __align__(16) unsigned char sm[];
    slab_inv_body<kHalf ? 1 : 0>(C, R, tw_g, M, blockIdx.x, sm);
}
#endif  // SE_BATCH_TU

// ---------------------------------------------------------------------------
// Slab transforms on 2-CTA thread-block clusters (single system): the two
// CTAs of a cluster share one x-slab, so that the transforms run on twice the
// SMs.  Forward: each CTA transforms half of the y rows along z and writes
// each result column straight into the shared memory of the CTA that owns
// that kz column (distributed shared memory stores), then, after one cluster
// barrier, transforms its kz columns along y.  Inverse: the same in the
// opposite order, with the Hermitian weights of the z real transform applied
// when the spectrum is loaded.

#ifndef SE_SLAB_CL
#define SE_SLAB_CL 2
#endif
constexpr int kSlabCL = SE_SLAB_CL;   // CTAs per x-slab cluster
// register tiles of the half-slab transforms (outputs x columns per thread):
// the forward one has too few outputs to give every thread a 2 x 2 tile;
// the inverse measured faster with 2 x 2
constexpr int kClTK = 1, kClTC = 2, kClInvTK = 2, kClInvTC = 2;

struct SlabClLayout {
    int ry, kc;                       // y rows and kz columns per CTA
    size_t tw, a, b, c, d, total;     // byte offsets of the regions
};

// forward: tw | S: ry x (M+1) floats | T: Mh x ry complex | X: kc x M complex
//          (written by both CTAs) | Z: kc x M complex (factored-DFT scratch)
// inverse: tw | A: M x kc complex | Z: M x kc complex | T: kc x (M+1) complex
//          | X: Mh x ry complex (written by both CTAs) | S: ry x (M+1) floats
__host__ __device__ inline SlabClLayout slabcl_layout(int M) {
    SlabClLayout l;
    const size_t Mh = M / 2 + 1, SP = M + 1;
    l.ry = (M + kSlabCL - 1) / kSlabCL;
    l.kc = (int)((Mh + kSlabCL - 1) / kSlabCL);
    auto up = [](size_t v) { return (v + 15) / 16 * 16; };
    const size_t f2 = sizeof(float2);
    const size_t r1 = up((size_t)l.ry * SP * sizeof(float));          // S
    const size_t r2 = up(Mh * l.ry * f2);                             // T (fwd) / X (inv)
    const size_t r3 = up((size_t)l.kc * M * f2);                      // X, Z (fwd) / A, Z (inv)
    const size_t r4 = up((size_t)l.kc * SP * f2);                     // T (inv)
    l.tw = 0;
    l.a = up((size_t)M * f2);
    l.b = l.a + (r1 > r3 ? r1 : r3);
    l.c = l.b + (r2 > r3 ? r2 : r3);
    l.d = l.c + (r3 > r4 ? r3 : r4);
    l.total = l.d + (r3 > r2 ? r3 : r2) + (r1 > r3 ? r1 : r3);
    return l;
}

#ifndef SE_BATCH_TU
template <bool kHalf>
__global__ void __launch_bounds__(kSlabThreads)
k_slab_fwd_cl(long long* __restrict__ g64, float2* __restrict__ Cg,
              const float2* __restrict__ tw_g, int M, const Acc* __restrict__ acc) {
    namespace cg = cooperative_groups;
    SE_STAMP(3, 0);
    pdl_wait();
    pdl_launch_next();
    SE_STAMP(3, 1);
    extern __shared__ __align__(16) unsigned char sm[];
    cg::cluster_group clu = cg::this_cluster();
    const int rank = (int)clu.block_rank(), x = blockIdx.x / kSlabCL;
    const SlabClLayout l = slabcl_layout(M);
    const int Mh = M / 2 + 1, SP = M + 1;
    float2* tw = reinterpret_cast<float2*>(sm + l.tw);
    float* S = reinterpret_cast<float*>(sm + l.a);
    float2* T = reinterpret_cast<float2*>(sm + l.b);
    float2* X = reinterpret_cast<float2*>(sm + l.c);
    float2* Z = reinterpret_cast<float2*>(sm + l.d);
    const int y0 = rank * l.ry, ny = max(0, min(l.ry, M - y0));
    const int k0 = rank * l.kc, nk = max(0, min(l.kc, Mh - k0));
    load_twiddles(tw, tw_g, M);
    const float inv = acc->fx_inv;
    const FDiv fM = fdiv_of(M);
    long long* src = g64 + ((size_t)x * M + y0) * M;   // read, then cleared for the next evaluation
    for (int e0 = threadIdx.x; e0 < ny * M; e0 += blockDim.x * kLoadBatch) {
        long long v[kLoadBatch];
#pragma unroll
        for (int u = 0; u < kLoadBatch; ++u) {
            const int e = e0 + u * (int)blockDim.x;
            v[u] = e < ny * M ? src[e] : 0;
        }
#pragma unroll
        for (int u = 0; u < kLoadBatch; ++u) {
            const int e = e0 + u * (int)blockDim.x;
            if (e >= ny * M) break;
            const int yl = fdiv(e, fM), z = e - yl * M;
            const unsigned long long w = (unsigned long long)v[u];
            const float hi = (float)(int)(w >> 32), lo = (float)(unsigned)(w & 0xffffffffull);
            S[yl * SP + z] = fmaf(hi, 4294967296.0f, lo) * inv;
            src[e] = 0;
        }
    }
    __syncthreads();
    SE_STAMP(3, 2);
    // z, real to complex, own rows: X(j = z, c = yl) = S[yl][z]  ->  T[kz][yl]
    // (through Z and the dead S when M/2 factors; X receives the partner's
    // pushes meanwhile and is not touched)
    if constexpr (kHalf)
        dft_r2c_half<kClTK, kClTC>(S, 1, SP, T, l.ry, 1, ny, Z, reinterpret_cast<float2*>(S), tw, M);
    else
        dft_r2c<kClTK, kClTC>(S, 1, SP, T, l.ry, 1, M, Mh, ny, tw, M);
    __syncthreads();
    // push: kz column k of these rows goes to the CTA owning k, X[k - k0'][y0 + yl]
    {
        float2* Xr[kSlabCL];
#pragma unroll
        for (int r = 0; r < kSlabCL; ++r) Xr[r] = clu.map_shared_rank(X, r);
        const FDiv fny = fdiv_of(max(ny, 1));
        for (int e = threadIdx.x; e < Mh * ny; e += blockDim.x) {
            const int kz = fdiv(e, fny), yl = e - kz * ny;
            const int owner = min(kz / l.kc, kSlabCL - 1);
            Xr[owner][(kz - owner * l.kc) * M + y0 + yl] = T[kz * l.ry + yl];
        }
    }
    clu.sync();   // every push has landed; no shared memory is read remotely afterwards
    SE_STAMP(3, 3);
    // y forward: X(j = y, c = kl)  ->  C[x][ky][k0 + kl]
    dft_c2c_fact<kClTK, kClTC>(X, 1, M, Cg + (size_t)x * M * Mh + k0, Mh, 1, nk, Z, tw, M, -1.0f);
    SE_STAMP(3, 4);
}

// Clusters 0..M-1: inverse slab transforms; cluster M: the grid energy from
// the x pass's nparts partials (acc->e_grid and, scaled, *E_out).
template <bool kHalf>
__global__ void __launch_bounds__(kSlabThreads)
k_slab_inv_cl(const float2* __restrict__ Cg, float* __restrict__ R, const float2* __restrict__ tw_g,
              int M, const double* __restrict__ xparts, int nparts, Acc* acc, double e_scale,
              double* E_out) {
    namespace cg = cooperative_groups;
    SE_STAMP(5, 0);
    pdl_wait();
    pdl_launch_next();
    SE_STAMP(5, 1);
    const int x = blockIdx.x / kSlabCL;
    if (x == M) {   // the whole cluster takes this branch
        if (blockIdx.x % kSlabCL != 0) return;
        __shared__ df2 sbuf[32];
        const df2 sum = sum_partials_df(reinterpret_cast<const float*>(xparts), nparts, 1, 0, sbuf);
        if (threadIdx.x == 0) {
            const double e = df_to_double(sum);
            acc->e_grid = e;
            if (E_out) *E_out = e_scale * e;
        }
        return;
    }
    extern __shared__ __align__(16) unsigned char sm[];
    cg::cluster_group clu = cg::this_cluster();
    const int rank = (int)clu.block_rank();
    const SlabClLayout l = slabcl_layout(M);
    const int Mh = M / 2 + 1, SP = M + 1;
    float2* tw = reinterpret_cast<float2*>(sm + l.tw);
    float2* A = reinterpret_cast<float2*>(sm + l.a);
    float2* Z = reinterpret_cast<float2*>(sm + l.b);
    float2* T = reinterpret_cast<float2*>(sm + l.c);
    float2* X = reinterpret_cast<float2*>(sm + l.d);
    float* S = reinterpret_cast<float*>(sm + l.a);   // A is dead by then
    const int y0 = rank * l.ry, ny = max(0, min(l.ry, M - y0));
    const int k0 = rank * l.kc, nk = max(0, min(l.kc, Mh - k0));
    load_twiddles(tw, tw_g, M);
    const FDiv fnk = fdiv_of(max(nk, 1)), fM = fdiv_of(M);
    // own kz columns of the slab, times the Hermitian weights (1 at kz = 0
    // and M/2, else 2): A[ky][kl]
    const float2* src = Cg + (size_t)x * M * Mh + k0;
    for (int e0 = threadIdx.x; e0 < M * nk; e0 += blockDim.x * kLoadBatch) {
        float2 v[kLoadBatch];
#pragma unroll
        for (int u = 0; u < kLoadBatch; ++u) {
            const int e = e0 + u * (int)blockDim.x;
            if (e < M * nk) {
                const int ky = fdiv(e, fnk), kl = e - ky * nk;
                v[u] = src[(size_t)ky * Mh + kl];
            }
        }
#pragma unroll
        for (int u = 0; u < kLoadBatch; ++u) {
            const int e = e0 + u * (int)blockDim.x;
            if (e < M * nk) {
                const int ky = fdiv(e, fnk), kl = e - ky * nk;
                const int kz = k0 + kl;
                const float wgt = (kz == 0 || 2 * kz == M) ? 1.0f : 2.0f;
                A[ky * l.kc + kl] = make_float2(wgt * v[u].x, wgt * v[u].y);
            }
        }
    }
    __syncthreads();
    SE_STAMP(5, 2);
    // y inverse: X(j = ky, c = kl) = A[ky][kl]  ->  T[kl][y]
    dft_c2c_fact<kClInvTK, kClInvTC>(A, l.kc, 1, T, 1, SP, nk, Z, tw, M, 1.0f);
    __syncthreads();
    // push: row y of these kz columns goes to the CTA owning y, X[k0 + kl][y - y0']
    {
        float2* Xr[kSlabCL];
#pragma unroll
        for (int r = 0; r < kSlabCL; ++r) Xr[r] = clu.map_shared_rank(X, r);
        for (int e = threadIdx.x; e < nk * M; e += blockDim.x) {
            const int kl = fdiv(e, fM), y = e - kl * M;
            const int owner = min(y / l.ry, kSlabCL - 1);
            Xr[owner][(k0 + kl) * l.ry + (y - owner * l.ry)] = T[kl * SP + y];
        }
    }
    clu.sync();   // every push has landed; no shared memory is read remotely afterwards
    // z complex to real, own rows: X(j = kz, c = yl) = X[kz][yl]  ->  S[yl][z]
    // (through Z and T when M/2 factors)
    if constexpr (kHalf)
        dft_c2r_half<kClInvTK, kClInvTC>(X, l.ry, 1, S, 1, SP, ny, Z, T, tw, M, 0.5f);
    else
        dft_c2r<kClInvTK, kClInvTC>(X, l.ry, 1, S, 1, SP, Mh, M, ny, tw, M);
    __syncthreads();
    SE_STAMP(5, 3);
    float* dst = R + ((size_t)x * M + y0) * M;
    for (int e = threadIdx.x; e < ny * M; e += blockDim.x) {
        const int yl = fdiv(e, fM), z = e - yl * M;
        dst[e] = S[yl * SP + z];
    }
    SE_STAMP(5, 4);
}
#endif  // SE_BATCH_TU

// ---------------------------------------------------------------------------
// Variant 5: the inverse slab transform fused with the gather (Eq. 3.9 and
// the analytic force of Sec. 3.1).  The 2-CTA cluster of x-slab x transforms
// the slab back to real space as k_slab_inv_cl does, but keeps the real
// plane Ht[x][y][z] in shared memory (each CTA sends the rows it produced to
// its partner, so both hold the whole plane) instead of writing the grid.
// Then every particle whose support contains plane x, i.e. x = i0x + a with
// 0 <= a < P, takes its sums over that plane,
//   S0 = sum_{b,c} gy_b gz_c Ht,  Sy = sum dgy_b gz_c Ht,  Sz = sum gy_b dgz_c Ht,
// and stores the plane's share of its potential and force sums as one
// float4 (gx_a S0, dgx_a S0, gx_a Sy, gx_a Sz) at part[a][particle].  Each
// (particle, a) pair is written by exactly one CTA: the particles come from
// the tile buckets of the columns of tiles holding the cells x - P/2 .. x +
// P/2 - 1, split between the two CTAs by tile, and from the overflow list,
// split over all warps of the cluster.  k_gfinish then adds the P shares of
// each particle in the order a = 0 .. P-1: the result does not depend on
// how the work was scheduled.  The grid is read from shared memory instead
// of L2, and the real grid is never written.

// shared memory: the inverse transform's regions (slabcl_layout) | the real
// plane, M rows sg_row_stride(M) floats apart
__host__ __device__ inline int sg_row_stride(int M) { return M + 1; }
__host__ __device__ inline size_t sg_plane_offset(int M) { return (slabcl_layout(M).total + 15) / 16 * 16; }
__host__ __device__ inline size_t sg_smem_bytes(int M) {
    return sg_plane_offset(M) + (size_t)M * sg_row_stride(M) * sizeof(float);
}

__device__ __forceinline__ f4 make_f4_zero() {
    f4 v;
    v.x = v.y = v.z = v.w = 0.0f;
    return v;
}

// One particle's share of plane x, by the G lanes of its group (lane k: z
// points k, k + G, ...); returns false (and zeros) when plane x is not in its
// support.  a: the support index of plane x.
template <int P, bool kForces>
__device__ __forceinline__ bool plane_sums(const f4& v, const KParams<float>& kp, int x,
                                           const float* __restrict__ PL, int SPL, int k, int* a_out,
                                           float4* out) {
    constexpr int D = pick_d(P), G = P / D;
    const int M = kp.M;
    float t;
    const int cx = cell_of(v.x, kp.invh, M, &t);
    int a = x - (cx - P / 2 + 1);
    a = a < 0 ? a + M : (a >= M ? a - M : a);
    *a_out = a;
    if (a >= P) {
        *out = make_float4(0.f, 0.f, 0.f, 0.f);
        return false;
    }
    const float ux = centre_offset(t, cx);
    const int cy = cell_of(v.y, kp.invh, M, &t);
    const float uy = centre_offset(t, cy);
    const int cz = cell_of(v.z, kp.invh, M, &t);
    const float uz = centre_offset(t, cz);
    float gy[P];
    fgg<float, P>(uy, kp.beta, kp.E3, gy);
    float gz[D], dgz[D];
    int jz[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const int c = k + j * G;
        const float dz = float(c) - 0.5f * float(P - 1) - uz;
        gz[j] = expf(-kp.beta * dz * dz);
        dgz[j] = dz * gz[j];
        jz[j] = wrap_index(cz - P / 2 + 1 + c, M);
    }
    float tb0[D], tby[D];
#pragma unroll
    for (int j = 0; j < D; ++j) tb0[j] = tby[j] = 0.0f;
    const int i0y = cy - P / 2 + 1;
#pragma unroll
    for (int b = 0; b < P; ++b) {
        const float* row = PL + wrap_index(i0y + b, M) * SPL;
        const float dgyb = (float(b) - 0.5f * float(P - 1) - uy) * gy[b];
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const float hv = row[jz[j]];
            tb0[j] += gy[b] * hv;
            if constexpr (kForces) tby[j] += dgyb * hv;
        }
    }
    float s0 = 0.0f, sy = 0.0f, sz = 0.0f;
#pragma unroll
    for (int j = 0; j < D; ++j) {
        s0 += gz[j] * tb0[j];
        if constexpr (kForces) {
            sy += gz[j] * tby[j];
            sz += dgz[j] * tb0[j];
        }
    }
    // x factor of support point a (the exponent written about the support
    // centre, as in fgg)
    const float gxa = expf(-kp.beta * ux * (ux + float(P - 1)) + 2.0f * kp.beta * ux * float(a)) *
                      kp.E3[a];
    const float dgxa = (float(a) - 0.5f * float(P - 1) - ux) * gxa;
    *out = make_float4(gxa * s0, dgxa * s0, gxa * sy, gxa * sz);
    return true;
}

// Sum of a float4 over the G lanes of a group (the whole warp takes part),
// valid in lane k = 0 of the group.
template <int G>
__device__ __forceinline__ float4 group_sum4(float4 v, int k) {
#pragma unroll
    for (int o = 1; o < G; o <<= 1) {
        const float a0 = __shfl_down_sync(0xffffffffu, v.x, o);
        const float a1 = __shfl_down_sync(0xffffffffu, v.y, o);
        const float a2 = __shfl_down_sync(0xffffffffu, v.z, o);
        const float a3 = __shfl_down_sync(0xffffffffu, v.w, o);
        if (k + o < G) {
            v.x += a0;
            v.y += a1;
            v.z += a2;
            v.w += a3;
        }
    }
    return v;
}

#ifndef SE_BATCH_TU
// Clusters 0..M-1: slab x = cluster index; cluster M: the grid energy from
// the x pass's nparts partials (acc->e_grid and, scaled, *E_grid).
// forces = 0: potential sums only (the force entries of part are zero).
template <int P, bool kForces>
__global__ void __launch_bounds__(kSlabThreads)
k_sinv_gather_cl(const float2* __restrict__ Cg, const float2* __restrict__ tw_g, const KParams<float> kp,
                 const double* __restrict__ xparts, int nparts, Acc* acc, double e_scale,
                 double* E_grid, const f4* __restrict__ bucket, const int* __restrict__ bucket_idx,
                 int cap, const int* __restrict__ tile_n, const int* __restrict__ over_idx,
                 const f4* __restrict__ wrapped, float4* __restrict__ part) {
    namespace cg = cooperative_groups;
    constexpr int D = pick_d(P), G = P / D, GPW = 32 / G;
    (void)D;
    pdl_wait();
    pdl_launch_next();
    const int M = kp.M;
    const int x = blockIdx.x / kSlabCL;
    if (x == M) {   // the whole cluster takes this branch
        if (blockIdx.x % kSlabCL != 0) return;
        __shared__ df2 sbuf[32];
        const df2 sum = sum_partials_df(reinterpret_cast<const float*>(xparts), nparts, 1, 0, sbuf);
        if (threadIdx.x == 0) {
            const double e = df_to_double(sum);
            acc->e_grid = e;
            if (E_grid) *E_grid = e_scale * e;
        }
        return;
    }
    extern __shared__ __align__(16) unsigned char sm[];
    cg::cluster_group clu = cg::this_cluster();
    const int rank = (int)clu.block_rank();
    const SlabClLayout l = slabcl_layout(M);
    const int Mh = M / 2 + 1, SP = M + 1, SPL = sg_row_stride(M);
    float2* tw = reinterpret_cast<float2*>(sm + l.tw);
    float2* A = reinterpret_cast<float2*>(sm + l.a);
    float2* Z = reinterpret_cast<float2*>(sm + l.b);
    float2* T = reinterpret_cast<float2*>(sm + l.c);
    float2* X = reinterpret_cast<float2*>(sm + l.d);
    float* PL = reinterpret_cast<float*>(sm + sg_plane_offset(M));
    const int y0 = rank * l.ry, ny = max(0, min(l.ry, M - y0));
    const int k0 = rank * l.kc, nk = max(0, min(l.kc, Mh - k0));
    load_twiddles(tw, tw_g, M);
    const FDiv fnk = fdiv_of(max(nk, 1)), fM = fdiv_of(M);
    // own kz columns of the slab times the Hermitian weights (1 at kz = 0 and
    // M/2, else 2): A[ky][kl]
    const float2* src = Cg + (size_t)x * M * Mh + k0;
    for (int e0 = threadIdx.x; e0 < M * nk; e0 += blockDim.x * kLoadBatch) {
        float2 v[kLoadBatch];
#pragma unroll
        for (int u = 0; u < kLoadBatch; ++u) {
            const int e = e0 + u * (int)blockDim.x;
            if (e < M * nk) {
                const int ky = fdiv(e, fnk), kl = e - ky * nk;
                v[u] = src[(size_t)ky * Mh + kl];
            }
        }
#pragma unroll
        for (int u = 0; u < kLoadBatch; ++u) {
            const int e = e0 + u * (int)blockDim.x;
            if (e < M * nk) {
                const int ky = fdiv(e, fnk), kl = e - ky * nk;
                const int kz = k0 + kl;
                const float wgt = (kz == 0 || 2 * kz == M) ? 1.0f : 2.0f;
                A[ky * l.kc + kl] = make_float2(wgt * v[u].x, wgt * v[u].y);
            }
        }
    }
    __syncthreads();
    // y inverse: X(j = ky, c = kl) = A[ky][kl]  ->  T[kl][y]
    dft_c2c_fact<kClInvTK, kClInvTC>(A, l.kc, 1, T, 1, SP, nk, Z, tw, M, 1.0f);
    __syncthreads();
    // push: row y of these kz columns goes to the CTA owning y
    {
        float2* Xr[kSlabCL];
#pragma unroll
        for (int r = 0; r < kSlabCL; ++r) Xr[r] = clu.map_shared_rank(X, r);
        for (int e = threadIdx.x; e < nk * M; e += blockDim.x) {
            const int kl = fdiv(e, fM), y = e - kl * M;
            const int owner = min(y / l.ry, kSlabCL - 1);
            Xr[owner][(k0 + kl) * l.ry + (y - owner * l.ry)] = T[kl * SP + y];
        }
    }
    clu.sync();   // every push has landed
    // z complex to real, own rows, straight into the plane: PL[y0 + yl][z]
    dft_c2r<kClInvTK, kClInvTC>(X, l.ry, 1, PL + (size_t)y0 * SPL, 1, SPL, Mh, M, ny, tw, M);
    __syncthreads();
    // own rows to the partner, so that both CTAs hold the whole plane
    for (int r = 0; r < kSlabCL; ++r) {
        if (r == rank) continue;
        float* PLr = clu.map_shared_rank(PL, r);
        for (int e = threadIdx.x; e < ny * M; e += blockDim.x) {
            const int yl = fdiv(e, fM), z = e - yl * M;
            const size_t o = (size_t)(y0 + yl) * SPL + z;
            PLr[o] = PL[o];
        }
    }
    clu.sync();   // the plane is complete in both CTAs; no remote access after this
    // the shares of plane x: tiles of the columns holding cells x - P/2 ..
    // x + P/2 - 1 (periodic), alternate tiles to the two CTAs, one tile per
    // warp at a time, GPW particles of it per round
    const int TT = kp.tile, nT = kp.nT, N = kp.N;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int gi = lane / G, k = lane - gi * G;
    const bool act = gi < GPW;
    const int c_first = wrap_index(x - P / 2, M);
    const int tx_first = c_first / TT;
    // tile columns tx_first, tx_first + 1, ... (mod nT) until the P cells are covered
    int ncol = 0;
    {
        int last = -1;
        for (int j = 0; j < P; ++j) {
            const int tx = wrap_index(c_first + j, M) / TT;
            if (tx != last) {
                ++ncol;
                last = tx;
            }
        }
    }
    const int nitems = ncol * nT * nT;
    for (int it = rank + kSlabCL * warp; it < nitems; it += kSlabCL * nw) {
        const int ci = it / (nT * nT), rem = it - ci * nT * nT;
        int tx = tx_first + ci;
        if (tx >= nT) tx -= nT;
        // a column reached twice through the wrap (ncol > nT) is taken once
        if (ci >= nT) continue;
        const int tile = tx * nT * nT + rem;
        const int n = min(tile_n[tile], cap);
        for (int s0 = 0; s0 < n; s0 += GPW) {
            const int s = s0 + gi;
            const bool valid = act && s < n;
            f4 v = make_f4_zero();
            int orig = 0;
            if (valid) {
                v = bucket[(size_t)tile * cap + s];
                orig = bucket_idx[(size_t)tile * cap + s];
            }
            int a = P;
            float4 sh = make_float4(0.f, 0.f, 0.f, 0.f);
            const bool in = valid && plane_sums<P, kForces>(v, kp, x, PL, SPL, k, &a, &sh);
            sh = group_sum4<G>(sh, k);
            if (in && k == 0) part[(size_t)a * N + orig] = sh;
        }
    }
    // the overflow list, over all warps of the cluster
    const int n_over = min(tile_n[kp.ntiles], N);
    const int gwarp = rank * nw + warp, ngw = kSlabCL * nw;
    for (int o0 = gwarp * GPW; o0 < n_over; o0 += ngw * GPW) {
        const int o = o0 + gi;
        const bool valid = act && o < n_over;
        f4 v = make_f4_zero();
        int orig = 0;
        if (valid) {
            orig = over_idx[o];
            v = wrapped[orig];
        }
        int a = P;
        float4 sh = make_float4(0.f, 0.f, 0.f, 0.f);
        const bool in = valid && plane_sums<P, kForces>(v, kp, x, PL, SPL, k, &a, &sh);
        sh = group_sum4<G>(sh, k);
        if (in && k == 0) part[(size_t)a * N + orig] = sh;
    }
}

// The P shares of each particle added in the order a = 0 .. P-1 (input
// order, one particle per thread): phi and F at the particle's input
// position, the energy 1/2 sum q phi by a double-float last-block reduction
// as in k_gather.  adj (device scalar, or null): the adjoint, phi and F
// scaled to dl/dq = g phi and dl/dx = -g F.
template <int P>
__global__ void __launch_bounds__(256)
k_gfinish(const float4* __restrict__ part, const f4* __restrict__ wrapped, float* __restrict__ phi,
          float* __restrict__ F, const KParams<float> kp, double* __restrict__ partials,
          unsigned* ticket, Acc* acc, double e_scale, double* E_out, const double* __restrict__ adj) {
    __shared__ df2 sbuf[32];
    pdl_wait();
    pdl_launch_next();
    const int N = kp.N;
    const float gsc = adj ? (float)__ldg(adj) : 1.0f;
    const float phi_mul = gsc, F_mul = adj ? -gsc : 1.0f;
    df2 e_df = df_from(0.0f);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        float4 sh[P];
#pragma unroll
        for (int a = 0; a < P; ++a) sh[a] = __ldcg(part + (size_t)a * N + i);
        float s0 = 0.f, sx = 0.f, sy = 0.f, sz = 0.f;
#pragma unroll
        for (int a = 0; a < P; ++a) {
            s0 += sh[a].x;
            sx += sh[a].y;
            sy += sh[a].z;
            sz += sh[a].w;
        }
        const float qq = wrapped[i].w;
        const float ph = s0 * kp.phi_scale;
        if (phi) phi[i] = ph * phi_mul;
        if (F) {
            const float fm = qq * kp.F_scale * F_mul;
            F[3 * i] = fm * sx;
            F[3 * i + 1] = fm * sy;
            F[3 * i + 2] = fm * sz;
        }
        e_df = df_add(e_df, df_from(qq * ph));
    }
    float* pf = reinterpret_cast<float*>(partials);
    const df2 r = block_sum_df(e_df, sbuf);
    if (threadIdx.x == 0) {
        pf[2 * blockIdx.x] = r.hi;
        pf[2 * blockIdx.x + 1] = r.lo;
    }
    const bool lastb = last_block(ticket);
    if (!lastb || threadIdx.x >= 32) return;
    const df2 t = warp_sum_partials_df(pf, gridDim.x, 1, 0);
    if (threadIdx.x == 0) {
        const double sum = df_to_double(t);
        acc->e_gather = sum;
        if (E_out) *E_out = e_scale * sum;
        *ticket = 0u;
    }
}

// The grid energy alone (acc->e_grid and, scaled, *E_out) from the x pass's
// nparts partials: one CTA, for an energy-only evaluation of variant 5 (its
// full evaluation sums it in the extra cluster of k_sinv_gather_cl).
__global__ void __launch_bounds__(256)
k_grid_energy(const double* __restrict__ xparts, int nparts, Acc* acc, double e_scale,
              double* E_out) {
    __shared__ df2 sbuf[32];
    pdl_wait();
    pdl_launch_next();
    const df2 sum = sum_partials_df(reinterpret_cast<const float*>(xparts), nparts, 1, 0, sbuf);
    if (threadIdx.x == 0) {
        const double e = df_to_double(sum);
        acc->e_grid = e;
        if (E_out) *E_out = e_scale * e;
    }
}
#endif  // SE_BATCH_TU

}  // namespace se

namespace se {

#ifndef SE_BATCH_TU
// fixed-point grid -> real grid (for inspection of the spread grid)
__global__ void __launch_bounds__(256)
k_fx_to_real(const long long* __restrict__ g64, float* __restrict__ dst, long long n,
             const Acc* __restrict__ acc) {
    pdl_wait();
    const float inv = acc->fx_inv;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
    {
        const unsigned long long u = (unsigned long long)g64[i];
        const float hi = (float)(int)(u >> 32), lo = (float)(unsigned)(u & 0xffffffffull);
        dst[i] = fmaf(hi, 4294967296.0f, lo) * inv;
    }
}
#endif  // SE_BATCH_TU

}  // namespace se
