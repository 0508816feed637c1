// se_kernels.cuh -- CUDA kernels of the SE k-space path (sm_103a).
//
// Algorithm 1 of arXiv:1712.04718 with the SE formulas of Table 2:
//   bin/sort -> spread (Eq. 3.5) -> [cuFFT R2C] -> scale (Eq. 3.6) ->
//   [cuFFT C2R] -> gather (Eq. 3.9, Sec. 3.1).
// Layout: real grids are M^3 with z fastest; the complex grid is the R2C
// half spectrum M x M x (M/2+1).  Particles are sorted by spreading tile and
// kept as (x, y, z, q) vectors with wrapped coordinates.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include "se_internal.h"

namespace se {

// ---------------------------------------------------------------------------
// Rounded arithmetic without contraction: the periodic wrap and the cell
// index are integer decisions and are taken by this exact sequence of
// rounded operations.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float expT(float a) { return expf(a); }
__device__ __forceinline__ double expT(double a) { return exp(a); }
// floor in the argument's own precision (a float must not go through the
// FP64 pipe; the result is the same integer-valued number either way)
__device__ __forceinline__ float floorT(float a) { return floorf(a); }
__device__ __forceinline__ double floorT(double a) { return floor(a); }

// Wrap one coordinate into [0, L): untouched when already inside, else
// x - L floor(x / L) with the reciprocal rounded once; anything left outside
// (or NaN) becomes 0.
template <typename T>
__device__ __forceinline__ T wrap_coord(T x, T L, T invL) {
    if (x >= T(0) && x < L) return x;
    T s = mul_rn(x, invL);
    T f = floorT(s);
    T p = mul_rn(f, L);
    T w = sub_rn(x, p);
    if (w >= L) w = sub_rn(w, L);
    if (w < T(0)) w = add_rn(w, L);
    if (!(w >= T(0) && w < L)) w = T(0);
    return w;
}

// Cell index floor(x M / L), clamped to [0, M-1]; also returns x M / L.
template <typename T>
__device__ __forceinline__ int cell_of(T xw, T invh, int M, T* t) {
    T s = mul_rn(xw, invh);
    *t = s;
    int c = (int)floorT(s);
    return c >= M ? M - 1 : (c < 0 ? 0 : c);
}

// Offset of the particle from the centre of its support, in grid units:
// u = (x/h - c) - 1/2, |u| <= 1/2.  The support point a (0..P-1) sits at
// (a - (P-1)/2 - u) h from the particle.
template <typename T>
__device__ __forceinline__ T centre_offset(T t, int c) {
    return (t - T(c)) - T(0.5);
}

// Fast Gaussian gridding (Eq. 3.10-3.11), written about the support centre so
// that no factor over- or underflows: with beta = alpha h^2 and
// a_c = a - (P-1)/2,
//   exp(-beta (a_c - u)^2) = exp(-beta u^2 - (P-1) beta u) * exp(2 beta u)^a
//                            * exp(-beta a_c^2),
// two exponentials per particle and dimension plus P multiplies; the last
// factor is the per-plan table E3.
template <typename T, int P>
__device__ __forceinline__ void fgg(T u, T beta, const T (&E3)[kMaxP], T (&g)[P]) {
    T A = expT(-beta * u * (u + T(P - 1)));
    T B = expT(T(2) * beta * u);
    T p = A;
#pragma unroll
    for (int a = 0; a < P; ++a) {
        g[a] = p * E3[a];
        p *= B;
    }
}

// Programmatic dependent launch: wait for the preceding kernel's results
// (a no-op when the kernel was launched without the attribute), and let the
// next kernel be scheduled early.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_next() { asm volatile("griddepcontrol.launch_dependents;"); }

// Optional phase tracing (build with -DSE_TRACE): thread 0 of each block
// records %globaltimer at phase boundaries of the single-precision kernels
// into se_trace_buf[kernel][block][phase]; compiled out otherwise.
#if defined(SE_TRACE) && !defined(SE_BATCH_TU)
constexpr int kTraceKernels = 8, kTraceBlocks = 2048, kTracePhases = 8;
__device__ unsigned long long se_trace_buf[kTraceKernels][kTraceBlocks][kTracePhases];
#define SE_STAMP(kid, ph)                                                                   \
    do {                                                                                    \
        if (threadIdx.x == 0 && blockIdx.x < kTraceBlocks) {                                \
            unsigned long long t_;                                                          \
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_));                          \
            se_trace_buf[kid][blockIdx.x][ph] = t_;                                         \
            if ((ph) == 0) {                                                                \
                unsigned sm_;                                                               \
                asm volatile("mov.u32 %0, %%smid;" : "=r"(sm_));                            \
                se_trace_buf[kid][blockIdx.x][kTracePhases - 1] = sm_;                      \
            }                                                                               \
        }                                                                                   \
    } while (0)
#else
#define SE_STAMP(kid, ph) \
    do {                  \
    } while (0)
#endif


constexpr int kScanSmem = 8192;   // tile counts staged in shared memory by the scan

// Periodic grid index for i in [-M, 2M): every caller passes a support index
// c - P/2 + 1 + a (0 <= c < M, 0 <= a < P) or a tile region offset of the
// same range, and every entry point enforces P <= M.
__device__ __forceinline__ int wrap_index(int i, int M) {
    if (i < 0) i += M;
    if (i >= M) i -= M;
    return i;
}

// Quotient n / d of integers 0 <= n < 2^22, d > 0, from a float reciprocal:
// (n + 1/2) / d lies at least 1/(2d) from an integer, and the two roundings
// (reciprocal and product) move it by less than (n + 1/2) 2^-23 / d < 1/(2d),
// so truncation gives the exact quotient.  A few instructions instead of the
// long integer division sequence, in index arithmetic of the hot loops.
struct FDiv {
    float inv;
    int d;
};
__device__ __forceinline__ FDiv fdiv_of(int d) { return FDiv{__frcp_rn((float)d), d}; }
__device__ __forceinline__ int fdiv(int n, FDiv f) { return (int)(((float)n + 0.5f) * f.inv); }

// Block-wide sum of one double (blockDim.x a multiple of 32, <= 1024).
__device__ __forceinline__ double block_sum(double v, double* sbuf) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sbuf[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sbuf[w];
    return r;  // valid in thread 0
}

// ---------------------------------------------------------------------------
// Double-float sums: a value hi + lo held in two floats (about 48 significant
// bits), added with two-sum.  The single-precision kernels reduce energies and
// charge sums this way: a chain of dependent FP64 additions costs microseconds
// on this GPU, FP32 two-sums do not.
struct df2 {
    float hi, lo;
};
__device__ __forceinline__ df2 df_add(df2 a, df2 b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bp = __fsub_rn(s, a.hi);
    const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bp)), __fsub_rn(b.hi, bp));
    const float lo = __fadd_rn(__fadd_rn(a.lo, b.lo), err);
    const float hi = __fadd_rn(s, lo);
    return df2{hi, __fsub_rn(lo, __fsub_rn(hi, s))};
}
__device__ __forceinline__ df2 df_from(float v) { return df2{v, 0.0f}; }
__device__ __forceinline__ double df_to_double(df2 a) { return (double)a.hi + (double)a.lo; }

// Block-wide double-float sum (blockDim.x a multiple of 32); valid in thread 0.
__device__ __forceinline__ df2 block_sum_df(df2 v, df2* sbuf) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        df2 u;
        u.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        u.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        v = df_add(v, u);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sbuf[warp] = v;
    __syncthreads();
    df2 r = df_from(0.0f);
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = df_add(r, sbuf[w]);
    return r;
}

// Sum of n double-float partials (pairs of floats, stride apart, from offset).
__device__ __forceinline__ df2 sum_partials_df(const float* partials, int n, int stride,
                                               int offset, df2* sbuf) {
    df2 v = df_from(0.0f);
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        df2 u;
        u.hi = __ldcg(partials + 2 * (k * stride + offset));
        u.lo = __ldcg(partials + 2 * (k * stride + offset) + 1);
        v = df_add(v, u);
    }
    return block_sum_df(v, sbuf);
}

// The same sum by one warp (valid in lane 0): eight loads per lane in flight
// at a time, then a shuffle reduction; no block barrier.
__device__ __forceinline__ df2 warp_sum_partials_df(const float* partials, int n, int stride,
                                                    int offset) {
    const int lane = threadIdx.x & 31;
    df2 v = df_from(0.0f);
    for (int k0 = lane; k0 < n; k0 += 32 * 8) {
        float hi[8], lo[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int k = k0 + 32 * u;
            hi[u] = k < n ? __ldcg(partials + 2 * (k * stride + offset)) : 0.0f;
            lo[u] = k < n ? __ldcg(partials + 2 * (k * stride + offset) + 1) : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) v = df_add(v, df2{hi[u], lo[u]});
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        df2 u;
        u.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        u.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        v = df_add(v, u);
    }
    return v;
}

// Last-block detection: every block stores its partial, fences, and takes a
// ticket; the block with the last ticket sees all partials.
__device__ __forceinline__ bool last_block(unsigned* ticket) {
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = atomicAdd(ticket, 1u);
        is_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (is_last) __threadfence();
    return is_last;
}

// Sum of n partials (stride apart, from offset), by the whole block; valid in
// thread 0.  The loads go through L2 (other blocks wrote them).
__device__ __forceinline__ double sum_partials(const double* partials, int n, int stride,
                                               int offset, double* sbuf) {
    double v = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) v += __ldcg(partials + k * stride + offset);
    return block_sum(v, sbuf);
}

// ---------------------------------------------------------------------------
// a1: bin.  Tile of every particle, its slot inside the tile, per-block sums
// of q and |q| and a NaN/Inf count.  The last block scans the tile counts into
// tile offsets, clears the counts for the next call and writes the checks.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
k_bin(const T* __restrict__ xyz, const T* __restrict__ q, const KParams<T> kp,
      int* __restrict__ tile_count, int* __restrict__ slot, int* __restrict__ tile_of,
      int* __restrict__ tile_start, double* __restrict__ partials, unsigned* ticket,
      Acc* acc) {
    __shared__ double sbuf[32];
    double sq = 0.0, sa = 0.0, bad = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kp.N; i += gridDim.x * blockDim.x) {
        T x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2], qq = q[i];
        if (!(isfinite(x) && isfinite(y) && isfinite(z) && isfinite(qq))) bad += 1.0;
        T t;
        int cx = cell_of(wrap_coord(x, kp.L, kp.invL), kp.invh, kp.M, &t);
        int cy = cell_of(wrap_coord(y, kp.L, kp.invL), kp.invh, kp.M, &t);
        int cz = cell_of(wrap_coord(z, kp.L, kp.invL), kp.invh, kp.M, &t);
        int tile = ((cx / kp.tile) * kp.nT + cy / kp.tile) * kp.nT + cz / kp.tile;
        slot[i] = atomicAdd(tile_count + tile, 1);
        tile_of[i] = tile;
        sq += (double)qq;
        sa += fabs((double)qq);
    }
    double r0 = block_sum(sq, sbuf);
    double r1 = block_sum(sa, sbuf);
    double r2 = block_sum(bad, sbuf);
    if (threadIdx.x == 0) {
        partials[3 * blockIdx.x] = r0;
        partials[3 * blockIdx.x + 1] = r1;
        partials[3 * blockIdx.x + 2] = r2;
    }
    if (!last_block(ticket)) return;

    // --- last block: checks, exclusive scan of the tile counts ---
    {
        const double a = sum_partials(partials, gridDim.x, 3, 0, sbuf);
        const double b = sum_partials(partials, gridDim.x, 3, 1, sbuf);
        const double c = sum_partials(partials, gridDim.x, 3, 2, sbuf);
        if (threadIdx.x == 0) {
            acc->sum_q = a;
            acc->sum_absq = b;
            acc->nonfinite = (unsigned)c;
            *ticket = 0u;
        }
    }
    __shared__ int warp_tot[32];
    __shared__ int scount[kScanSmem];
    const int n = kp.ntiles;
    const bool staged = n <= kScanSmem;
    if (staged) {
        // one coalesced pass over the counts (written by atomics in L2)
        for (int k = threadIdx.x; k < n; k += blockDim.x) scount[k] = __ldcg(tile_count + k);
        __syncthreads();
    }
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int b0 = min(n, (int)threadIdx.x * per), b1 = min(n, b0 + per);
    int local = 0;
    for (int k = b0; k < b1; ++k) local += staged ? scount[k] : __ldcg(tile_count + k);
    // block exclusive scan of `local`
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
        if (lane < nw) warp_tot[lane] = v;  // inclusive over warps
    }
    __syncthreads();
    int run = incl - local + (warp > 0 ? warp_tot[warp - 1] : 0);
    for (int k = b0; k < b1; ++k) {
        int cnt = staged ? scount[k] : __ldcg(tile_count + k);
        tile_start[k] = run;
        run += cnt;
    }
    for (int k = threadIdx.x; k < n; k += blockDim.x) tile_count[k] = 0;
    if (threadIdx.x == blockDim.x - 1) tile_start[n] = run;
}

// a1: scatter into tile order: sorted[tile_start[tile] + slot] = (x, y, z, q).
template <typename T>
__global__ void __launch_bounds__(256)
k_scatter(const T* __restrict__ xyz, const T* __restrict__ q, const KParams<T> kp,
          const int* __restrict__ slot, const int* __restrict__ tile_of,
          const int* __restrict__ tile_start, v4_t<T>* __restrict__ sorted,
          int* __restrict__ perm) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kp.N; i += gridDim.x * blockDim.x) {
        int dst = tile_start[tile_of[i]] + slot[i];
        v4_t<T> v;
        v.x = wrap_coord(xyz[3 * i], kp.L, kp.invL);
        v.y = wrap_coord(xyz[3 * i + 1], kp.L, kp.invL);
        v.z = wrap_coord(xyz[3 * i + 2], kp.L, kp.invL);
        v.w = q[i];
        sorted[dst] = v;
        perm[dst] = i;
    }
}

// Exact rounding error of the sum old + val as rounded by the atomic add
// (two-sum; the atomic rounds to nearest even).
template <typename T>
__device__ __forceinline__ T two_sum_err(T old, T val) {
    T s = add_rn(old, val);
    T bp = sub_rn(s, old);
    return add_rn(sub_rn(old, sub_rn(s, bp)), sub_rn(val, bp));
}

// ---------------------------------------------------------------------------
// a3: spread, shared-memory tiles.  One CTA per tile of `tile`^3 cells.  The
// particles of the tile add their P^3 weights q c_g gx gy gz into the tile's
// region ((tile + P - 1)^3 points) in shared memory; the region is then added
// to the global grid, each nonzero point once per tile.  With COMP the
// shared-memory sums are compensated: every add's rounding error (two-sum
// against the value the atomic returned) goes to a second array, and the
// region value flushed is hi + lo.  Regions larger than the shared-memory
// budget are processed in slabs of `slab` x-planes.
// ---------------------------------------------------------------------------
template <typename T, int P, bool COMP>
__global__ void __launch_bounds__(256)
k_spread_tiled(const v4_t<T>* __restrict__ sorted, const int* __restrict__ tile_start,
               T* __restrict__ grid, const KParams<T> kp, int slab) {
    constexpr int D = pick_d(P), G = P / D, GPW = 32 / G;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* hi = reinterpret_cast<T*>(smem_raw);
    __shared__ T sE3[P];

    const int tile = blockIdx.x;
    const int pbeg = tile_start[tile], pend = tile_start[tile + 1];
    if (pbeg == pend) return;
    if (threadIdx.x < P) sE3[threadIdx.x] = kp.E3[threadIdx.x];
    const int nT = kp.nT, M = kp.M, TT = kp.tile;
    const int tz = tile % nT, ty = (tile / nT) % nT, tx = tile / (nT * nT);
    const int t0x = tx * TT, t0y = ty * TT, t0z = tz * TT;
    const int Ry = min(TT, M - t0y) + P - 1, Rz = min(TT, M - t0z) + P - 1;
    const int Rx = min(TT, M - t0x) + P - 1;
    const int plane = Ry * Rz;
    T* lo = hi + (size_t)slab * plane;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gi = lane / G, k = lane - gi * G;
    const bool act = gi < GPW;
    const int ngroups = (blockDim.x >> 5) * GPW;
    const int group = warp * GPW + gi;

    for (int s0 = 0; s0 < Rx; s0 += slab) {
        const int ns = min(slab, Rx - s0);
        const int nel = ns * plane;
        for (int e = threadIdx.x; e < nel; e += blockDim.x) {
            hi[e] = T(0);
            if (COMP) lo[e] = T(0);
        }
        __syncthreads();
        if (act) {
            for (int p = pbeg + group; p < pend; p += ngroups) {
                const v4_t<T> v = sorted[p];
                T t;
                const int cx = cell_of(v.x, kp.invh, M, &t);
                const T ux = centre_offset(t, cx);
                const int cy = cell_of(v.y, kp.invh, M, &t);
                const T uy = centre_offset(t, cy);
                const int cz = cell_of(v.z, kp.invh, M, &t);
                const T uz = centre_offset(t, cz);
                const int lx = cx - t0x, ly = cy - t0y, lz = cz - t0z;
                const int alo = max(0, s0 - lx), ahi = min(P, s0 + ns - lx);
                if (alo >= ahi) continue;
                T gy[P];
                fgg<T, P>(uy, kp.beta, kp.E3, gy);
                T gz[D];
                const T qw = v.w * kp.qcg;
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    const T dz = T(k + j * G) - T(0.5) * T(P - 1) - uz;
                    gz[j] = qw * expT(-kp.beta * dz * dz);
                }
                // x factors by the FGG recurrence, starting at a = alo
                const T Bx = expT(T(2) * kp.beta * ux);
                T px = expT(-kp.beta * ux * (ux + T(P - 1)) + T(2) * kp.beta * ux * T(alo));
#pragma unroll 1
                for (int a = alo; a < ahi; ++a) {
                    const T gxa = px * sE3[a];
                    px *= Bx;
                    const int rowx = lx + a - s0;
                    T* rowp = hi + (rowx * Ry + ly) * Rz + lz + k;
#pragma unroll
                    for (int b = 0; b < P; ++b) {
                        const T wab = gxa * gy[b];
                        T* base = rowp + b * Rz;
#pragma unroll
                        for (int j = 0; j < D; ++j) {
                            const T val = wab * gz[j];
                            T* dst = base + j * G;
                            if (COMP) {
                                const T old = atomicAdd(dst, val);
                                atomicAdd(lo + (dst - hi), two_sum_err(old, val));
                            } else {
                                atomicAdd(dst, val);
                            }
                        }
                    }
                }
            }
        }
        __syncthreads();
        const int ox = t0x - P / 2 + 1 + s0, oy = t0y - P / 2 + 1, oz = t0z - P / 2 + 1;
        const FDiv fRz = fdiv_of(Rz), fRy = fdiv_of(Ry);
        for (int e = threadIdx.x; e < nel; e += blockDim.x) {
            T val = hi[e];
            if (COMP) val = add_rn(val, lo[e]);
            if (val != T(0)) {
                const int r = fdiv(e, fRz), rz = e - r * Rz;
                const int rx = fdiv(r, fRy), ry = r - rx * Ry;
                const int gx_ = wrap_index(ox + rx, M), gy_ = wrap_index(oy + ry, M),
                          gz_ = wrap_index(oz + rz, M);
                atomicAdd(grid + ((size_t)gx_ * M + gy_) * M + gz_, val);
            }
        }
        __syncthreads();
    }
}

// a3: spread straight into the global grid (each weight one global atomic
// add).  For large supports, where a tile's region would hold far more points
// than its particles touch.  Uncompensated.
template <typename T, int P>
__global__ void __launch_bounds__(256)
k_spread_direct(const v4_t<T>* __restrict__ sorted, T* __restrict__ grid, const KParams<T> kp) {
    constexpr int D = pick_d(P), G = P / D, GPW = 32 / G;
    __shared__ T sE3[P];
    if (threadIdx.x < P) sE3[threadIdx.x] = kp.E3[threadIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gi = lane / G, k = lane - gi * G;
    if (gi >= GPW) return;
    const int gpb = (blockDim.x >> 5) * GPW;
    const int M = kp.M;
    for (int p = blockIdx.x * gpb + warp * GPW + gi; p < kp.N; p += gridDim.x * gpb) {
        const v4_t<T> v = sorted[p];
        T t;
        const int cx = cell_of(v.x, kp.invh, M, &t);
        const T ux = centre_offset(t, cx);
        const int cy = cell_of(v.y, kp.invh, M, &t);
        const T uy = centre_offset(t, cy);
        const int cz = cell_of(v.z, kp.invh, M, &t);
        const T uz = centre_offset(t, cz);
        T gy[P];
        fgg<T, P>(uy, kp.beta, kp.E3, gy);
        T gz[D];
        int jz[D];
        const T qw = v.w * kp.qcg;
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const int c = k + j * G;
            const T dz = T(c) - T(0.5) * T(P - 1) - uz;
            gz[j] = qw * expT(-kp.beta * dz * dz);
            jz[j] = wrap_index(cz - P / 2 + 1 + c, M);
        }
        const int i0x = cx - P / 2 + 1, i0y = cy - P / 2 + 1;
        int jy[P];
#pragma unroll
        for (int b = 0; b < P; ++b) jy[b] = wrap_index(i0y + b, M);
        const T Bx = expT(T(2) * kp.beta * ux);
        T px = expT(-kp.beta * ux * (ux + T(P - 1)));
#pragma unroll 1
        for (int a = 0; a < P; ++a) {
            const T gxa = px * sE3[a];
            px *= Bx;
            const int jx = wrap_index(i0x + a, M);
#pragma unroll
            for (int b = 0; b < P; ++b) {
                T* row = grid + ((size_t)jx * M + jy[b]) * M;
                const T wab = gxa * gy[b];
#pragma unroll
                for (int j = 0; j < D; ++j) atomicAdd(row + jz[j], wab * gz[j]);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// a5: scale.  Hhat <- G(k)/M^3 Hhat on the half spectrum, the grid energy
// sum_k w_k G |Hhat|^2 (w = 1 on the kz = 0 and Nyquist planes, 2 elsewhere),
// and zeroing of the spread grid for the next spread (the forward FFT has
// consumed it).  G is an FP64 table.
// ---------------------------------------------------------------------------
template <typename T, typename C>
__global__ void __launch_bounds__(256)
k_scale(C* __restrict__ cgrid, const double* __restrict__ green, int M, double invM3,
        T* __restrict__ zero_grid, double* __restrict__ partials, unsigned* ticket,
        Acc* acc, double e_scale, double* E_out) {
    __shared__ double sbuf[32];
    const int Mh = M / 2 + 1;
    const long long total = (long long)M * M * Mh;
    const long long stride = (long long)gridDim.x * blockDim.x;
    double e = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        const int kz = (int)(i % Mh);
        const double g = green[i];
        C c = cgrid[i];
        const double m2 = (double)c.x * (double)c.x + (double)c.y * (double)c.y;
        e += ((kz == 0 || 2 * kz == M) ? 1.0 : 2.0) * g * m2;
        const T f = (T)(g * invM3);
        c.x *= f;
        c.y *= f;
        cgrid[i] = c;
    }
    if (zero_grid) {
        const long long n3 = (long long)M * M * M;
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += stride)
            zero_grid[i] = T(0);
    }
    double r = block_sum(e, sbuf);
    if (threadIdx.x == 0) partials[blockIdx.x] = r;
    if (!last_block(ticket)) return;
    const double s = sum_partials(partials, gridDim.x, 1, 0, sbuf);
    if (threadIdx.x == 0) {
        acc->e_grid = s;
        if (E_out) *E_out = e_scale * s;
        *ticket = 0u;
    }
}

// ---------------------------------------------------------------------------
// a7: gather.  Each particle's G lanes read its P^3 support from the grid
// (L2-resident) and reduce separably: z in the lane, y then x in registers:
//   phi ~ sum_a gx[a] sum_b gy[b] sum_c gz[c] Ht[a,b,c]
//   F   ~ sum (offset) * (same), the offset multiplying its own factor.
// Results are scattered to the caller's order; the energy sum q phi is
// reduced per block and finished by the last block.
// ---------------------------------------------------------------------------
// Potential and force sums of one particle on the grid (Eq. 3.9 and the
// analytic force of Sec. 3.1), in two parts: gather_prep computes the
// particle's separable Gaussian factors and grid indices (no grid access, so
// it may run before the grid is ready), gather_accum the sums over this
// lane's z points, vphi, vfx, vfy, vfz (to be reduced over the particle's G
// lanes).
template <typename T, int P>
struct GatherPrep {
    static constexpr int D = pick_d(P);
    T gy[P], dgy[P], gz[D], dgz[D];
    int jy[P], jz[D];
    T ux, uy, px0, Bx;
    int i0x, i0y;
};

template <typename T, int P>
__device__ __forceinline__ void gather_prep(const v4_t<T>& v, const KParams<T>& kp, int k,
                                            GatherPrep<T, P>& g) {
    constexpr int D = pick_d(P), G = P / D;
    const int M = kp.M;
    T t;
    const int cx = cell_of(v.x, kp.invh, M, &t);
    g.ux = centre_offset(t, cx);
    const int cy = cell_of(v.y, kp.invh, M, &t);
    const T uy = centre_offset(t, cy);
    const int cz = cell_of(v.z, kp.invh, M, &t);
    const T uz = centre_offset(t, cz);
    fgg<T, P>(uy, kp.beta, kp.E3, g.gy);
    g.uy = uy;
    g.i0x = cx - P / 2 + 1;
    const int i0y = cy - P / 2 + 1;
    g.i0y = i0y;
#pragma unroll
    for (int b = 0; b < P; ++b) {
        g.dgy[b] = (T(b) - T(0.5) * T(P - 1) - uy) * g.gy[b];
        g.jy[b] = wrap_index(i0y + b, M);
    }
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const int c = k + j * G;
        const T dz = T(c) - T(0.5) * T(P - 1) - uz;
        g.gz[j] = expT(-kp.beta * dz * dz);
        g.dgz[j] = dz * g.gz[j];
        g.jz[j] = wrap_index(cz - P / 2 + 1 + c, M);
    }
    g.Bx = expT(T(2) * kp.beta * g.ux);
    g.px0 = expT(-kp.beta * g.ux * (g.ux + T(P - 1)));
}

#ifndef SE_GATHER_UNROLL
#define SE_GATHER_UNROLL 2
#endif
constexpr int kGatherUnroll = SE_GATHER_UNROLL;   // x planes in flight (single precision, P <= 8)
template <typename T, int P>
__device__ __forceinline__ void gather_accum(const GatherPrep<T, P>& g, const T* __restrict__ grid,
                                             const KParams<T>& kp, const T* sE3, T& vphi, T& vfx,
                                             T& vfy, T& vfz) {
    constexpr int D = pick_d(P);
    const int M = kp.M;
    T acc0[D], accx[D], accy[D];
#pragma unroll
    for (int j = 0; j < D; ++j) acc0[j] = accx[j] = accy[j] = T(0);
    T px = g.px0;
    if constexpr (sizeof(T) == sizeof(float) && P <= 8) {
        // single precision, small supports: kGatherUnroll x planes at a
        // time, the rows' grid offsets formed in the loop instead of kept in
        // P registers.  Within the 64 registers of four CTAs per SM this
        // spills less than keeping them with all planes in flight (P = 8:
        // 76 against 140 bytes a thread); measured: the gather of the
        // 21 642-atom box at P = 8 13.8 us against 15.2 us (CUDA-graph replay)
#pragma unroll(kGatherUnroll)
        for (int a = 0; a < P; ++a) {
            const T gxa = px * sE3[a];
            const T dgxa = (T(a) - T(0.5) * T(P - 1) - g.ux) * gxa;
            px *= g.Bx;
            const T* plane = grid + (size_t)wrap_index(g.i0x + a, M) * M * M;
            T tb0[D], tby[D];
#pragma unroll
            for (int j = 0; j < D; ++j) tb0[j] = tby[j] = T(0);
#pragma unroll
            for (int b = 0; b < P; ++b) {
                const T* row = plane + wrap_index(g.i0y + b, M) * M;
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    const T hv = __ldg(row + g.jz[j]);
                    tb0[j] += g.gy[b] * hv;
                    tby[j] += g.dgy[b] * hv;
                }
            }
#pragma unroll
            for (int j = 0; j < D; ++j) {
                acc0[j] += gxa * tb0[j];
                accx[j] += dgxa * tb0[j];
                accy[j] += gxa * tby[j];
            }
        }
    } else {
        // the whole x loop unrolled for small supports, so that every load of
        // the particle's P^3 grid values is in flight at once
#pragma unroll(P <= 8 ? P : 1)
        for (int a = 0; a < P; ++a) {
            const T gxa = px * sE3[a];
            const T dgxa = (T(a) - T(0.5) * T(P - 1) - g.ux) * gxa;
            px *= g.Bx;
            const int jx = wrap_index(g.i0x + a, M);
            T tb0[D], tby[D];
#pragma unroll
            for (int j = 0; j < D; ++j) tb0[j] = tby[j] = T(0);
#pragma unroll
            for (int b = 0; b < P; ++b) {
                const T* row = grid + ((size_t)jx * M + g.jy[b]) * M;
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    const T hv = __ldg(row + g.jz[j]);
                    tb0[j] += g.gy[b] * hv;
                    tby[j] += g.dgy[b] * hv;
                }
            }
#pragma unroll
            for (int j = 0; j < D; ++j) {
                acc0[j] += gxa * tb0[j];
                accx[j] += dgxa * tb0[j];
                accy[j] += gxa * tby[j];
            }
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

// Single precision and P <= 8: at most 64 registers, so that four CTAs fit on
// an SM (a bound of 48 for five makes the accumulation spill).
#ifndef SE_GATHER_MINB
#define SE_GATHER_MINB 4
#endif
#ifndef SE_GATHER_THREADS
#define SE_GATHER_THREADS 256
#endif
// threads of a k_gather CTA (every launch of the instantiation uses it)
template <typename T, int P>
__host__ __device__ constexpr int gather_threads() {
    return (sizeof(T) == 4 && P <= 8) ? SE_GATHER_THREADS : 256;
}
template <typename T, int P>
__global__ void __launch_bounds__(gather_threads<T, P>(), (sizeof(T) == 4 && P <= 8) ? SE_GATHER_MINB : 1)
k_gather(const v4_t<T>* __restrict__ sorted, const int* __restrict__ perm,
 const T* __restrict__ grid, T* __restrict__ phi, T* __restrict__ F,
 const KParams<T> kp, double* __restrict__ partials, unsigned* ticket, Acc* acc,
 double e_scale, double* E_out, const double* __restrict__ adj) {
    constexpr int D = pick_d(P), G = P / D, GPW = 32 / G;
    constexpr bool kSingle = sizeof(T) == sizeof(float);
    SE_STAMP(6, 0);
    __shared__ double sbuf[32];
    __shared__ df2 sbuf_df[32];
    __shared__ T sE3[P];
    if (threadIdx.x < P) sE3[threadIdx.x] = kp.E3[threadIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gi = lane / G, k = lane - gi * G;
    const int gpb = (blockDim.x >> 5) * GPW;
    // the particles were written before the grid's transforms began: the
    // first particle's factors are computed while the grid is still being
    // produced (before the dependent-launch wait)
    int pb = blockIdx.x * gpb + warp * GPW;
    GatherPrep<T, P> g;
    T qq = T(0);
    if (gi < GPW && pb + gi < kp.N) {
        const v4_t<T> v = sorted[pb + gi];
        qq = v.w;
        gather_prep<T, P>(v, kp, k, g);
    }
    pdl_wait();
    SE_STAMP(6, 1);
    __syncthreads();
    // adjoint (backward) mode: outputs are dl/dq = g phi and dl/dx = -g F for
    // the upstream gradient g = dl/dE read from device memory
    const T gsc = adj ? (T)__ldg(adj) : T(1);
    const T phi_mul = gsc, F_mul = adj ? -gsc : T(1);
    double e_loc = 0.0;
    df2 e_df = df_from(0.0f);
    for (; pb < kp.N; pb += gridDim.x * gpb) {
        const int p = pb + gi;
        const bool valid = (gi < GPW) && (p < kp.N);
        T vphi = T(0), vfx = T(0), vfy = T(0), vfz = T(0);
        if (valid) {
            if (pb != blockIdx.x * gpb + warp * GPW) {   // later particles: after the wait
                const v4_t<T> v = sorted[p];
                qq = v.w;
                gather_prep<T, P>(v, kp, k, g);
            }
            gather_accum<T, P>(g, grid, kp, sE3, vphi, vfx, vfy, vfz);
        }
        SE_STAMP(6, 2);
        // reduce over the G lanes of each particle (lane 0 of the group ends with the sum)
#pragma unroll
        for (int o = 1; o < G; o <<= 1) {
            const T a0 = __shfl_down_sync(0xffffffffu, vphi, o);
            const T a1 = __shfl_down_sync(0xffffffffu, vfx, o);
            const T a2 = __shfl_down_sync(0xffffffffu, vfy, o);
            const T a3 = __shfl_down_sync(0xffffffffu, vfz, o);
            if (k + o < G) {
                vphi += a0;
                vfx += a1;
                vfy += a2;
                vfz += a3;
            }
        }
        if (valid && k == 0) {
            const T ph = vphi * kp.phi_scale;
            const T fs = qq * kp.F_scale;
            const int orig = perm ? perm[p] : p;   // no perm: particles in input order
            if (phi) phi[orig] = ph * phi_mul;
            if (F) {
                const T fm = fs * F_mul;
                F[3 * orig] = fm * vfx;
                F[3 * orig + 1] = fm * vfy;
                F[3 * orig + 2] = fm * vfz;
            }
            if (kSingle)
                e_df = df_add(e_df, df_from((float)(qq * ph)));
            else
                e_loc += (double)qq * (double)ph;
        }
    }
    SE_STAMP(6, 3);
    if (kSingle) {
        // double-float partials: (hi, lo) floats per block
        float* pf = reinterpret_cast<float*>(partials);
        const df2 r = block_sum_df(e_df, sbuf_df);
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

}  // namespace se
