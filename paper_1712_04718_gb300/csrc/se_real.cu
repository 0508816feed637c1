// se_real.cu -- the real-space part of the Ewald sum on the GPU, with cell
// lists: the complement of the SE k-space path for full Ewald energies and
// forces (Sec. 1, Eq. 1.5-1.7, the erfc terms and the self term).
//
// For charges q_n at x_n in the periodic box [0, L)^3, splitting parameter
// xi and cut-off r_c:
//   phi_m = kc [ sum_{n, images; 0 < r < r_c} q_n erfc(xi r) / r  -  2 xi / sqrt(pi) q_m ]
//   F_m   = kc q_m sum_{n, images; r < r_c} q_n (2 xi / sqrt(pi) e^{-xi^2 r^2} + erfc(xi r) / r)
//           (x_m - x_n^image) / r^2
//   E     = 1/2 sum_m q_m phi_m            (real-space energy plus the self energy)
// so that these plus the k-space results of se_evaluate are the whole Ewald
// potential, force and energy.
//
// GPU design: particles are counted into cells of edge >= r_c / K (nc =
// floor(K L / r_c) per dimension, at most 40, nc >= 2K+1, so the (2K+1)^3
// cells around a cell are distinct periodic images and every pair within r_c
// is met exactly once), scanned and scattered into cell order.  One CTA per
// home cell stages its stencil in shared memory with the image shifts
// applied (the cells' ranges fetched in parallel, offsets by a warp scan,
// each staged particle located by binary search; in chunks when they do not
// fit).  In single precision each thread holds three home particles and
// tests every candidate it loads from shared memory against all three (one
// shared load per three distance tests); the candidate loop of a set of home
// particles is split over S adjacent lanes (S a power of two), reduced by
// shuffles.  In double precision (one home particle per thread) the hits of
// a particle's S lanes are queued in shared memory and shared out evenly
// before the erfc terms.  Every particle sums its own potential and force:
// no atomics on the outputs.  The energy is a deterministic two-level
// reduction (last block).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "../../include/se.h"
#include "se_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxCellsPerDim = 40;     // at most 64 000 cells (one energy partial each)
#ifndef SE_RS_NB_KB
#define SE_RS_NB_KB 32
#endif
constexpr size_t kNbSmem = SE_RS_NB_KB * 1024;   // shared memory for staged neighbours

template <typename T> struct R4 { using type = se::v4_t<T>; };

// Single precision: erfc(x) = erfcx(x) e^{-x^2} with erfcx(x) ~ t P(t),
// t = 1 / (1 + p x), P of degree 8 (the form of Hastings' approximations,
// Abramowitz and Stegun 7.1.26), coefficients fitted by gen_erfcx_fit.py for
// relative accuracy on 0 <= x <= 6 (3.5e-7 evaluated in float32; beyond 6,
// where erfc < 2e-17, within 2e-5).  The e^{-x^2} is the one the force term
// needs anyway, so each pair evaluates one exponential.
constexpr float kErfcxP = 4.50000000e-01f;
__constant__ float kErfcx[9] = {
    2.536794543e-01f,
    2.576121688e-01f,
    1.990700811e-01f,
    3.049189448e-01f,
    -2.398110330e-01f,
    6.246721148e-01f,
    -6.125214100e-01f,
    2.510224283e-01f,
    -3.864272311e-02f};

__device__ __forceinline__ float erfcx_fit(float x) {
    const float t = __fdividef(1.0f, fmaf(kErfcxP, x, 1.0f));   // 2 ulp
    float a = kErfcx[8];
#pragma unroll
    for (int k = 7; k >= 0; --k) a = fmaf(a, t, kErfcx[k]);
    return a * t;
}

// erfc(xi r)/r and the force factor (2 xi/sqrt(pi) e^{-xi^2 r^2} + erfc(xi r)/r)/r^2
// for one pair, given r^2 and 1/r.
__device__ __forceinline__ void pair_terms(float r2, float ir, float xi, float c2xi, float& ec,
                                           float& fr) {
    const float x = xi * (r2 * ir);
    const float e = expf(-x * x);
    ec = erfcx_fit(x) * e * ir;
    fr = (c2xi * e + ec) * ir * ir;
}
__device__ __forceinline__ void pair_terms(double r2, double ir, double xi, double c2xi,
                                           double& ec, double& fr) {
    const double r = r2 * ir;
    ec = erfc(xi * r) * ir;
    fr = (c2xi * exp(-xi * xi * r2) + ec) * ir * ir;
}
__device__ __forceinline__ float rsqrtR(float a) { return rsqrtf(a); }
__device__ __forceinline__ double rsqrtR(double a) { return rsqrt(a); }
__device__ __forceinline__ float floorR(float a) { return floorf(a); }
__device__ __forceinline__ double floorR(double a) { return floor(a); }

// Wrap into [0, L): x - L floor(x / L), then one correction; NaN or anything
// still outside becomes 0.
template <typename T>
__device__ __forceinline__ T wrapR(T x, T L, T invL) {
    if (x >= T(0) && x < L) return x;
    T y = x - L * floorR(x * invL);
    if (y >= L) y -= L;
    if (!(y >= T(0) && y < L)) y = T(0);
    return y;
}

template <typename T>
__device__ __forceinline__ int cellR(T x, T cscale, int nc) {
    int c = (int)(x * cscale);
    return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_rs_count(const T* __restrict__ xyz, int N, T L, T invL, T cscale, int nc, int* count,
           int* __restrict__ cell_of, int* __restrict__ slot) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int cx = cellR(wrapR(xyz[3 * i], L, invL), cscale, nc);
    const int cy = cellR(wrapR(xyz[3 * i + 1], L, invL), cscale, nc);
    const int cz = cellR(wrapR(xyz[3 * i + 2], L, invL), cscale, nc);
    const int c = (cx * nc + cy) * nc + cz;
    cell_of[i] = c;
    slot[i] = atomicAdd(&count[c], 1);
}

// Exclusive scan of the cell counts into start[0..ncells] by one CTA of 1024
// threads, chunk by chunk with a running carry; the counts are cleared for
// the next evaluation.
__global__ void __launch_bounds__(1024) k_rs_scan(int* count, int* start, int ncells) {
    __shared__ int wsum[32];
    __shared__ int carry_s;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < ncells; base += 1024) {
        const int i = base + threadIdx.x;
        const int v = i < ncells ? count[i] : 0;
        if (i < ncells) count[i] = 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int w = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            wsum[lane] = w;
        }
        __syncthreads();
        const int carry = carry_s;
        const int incl = x + (warp > 0 ? wsum[warp - 1] : 0);
        if (i < ncells) start[i] = carry + incl - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry_s = carry + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) start[ncells] = carry_s;
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_rs_scatter(const T* __restrict__ xyz, const T* __restrict__ q, int N, T L, T invL,
             const int* __restrict__ cell_of, const int* __restrict__ slot,
             const int* __restrict__ start, typename R4<T>::type* __restrict__ sorted,
             int* __restrict__ perm) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int p = start[cell_of[i]] + slot[i];
    typename R4<T>::type v;
    v.x = wrapR(xyz[3 * i], L, invL);
    v.y = wrapR(xyz[3 * i + 1], L, invL);
    v.z = wrapR(xyz[3 * i + 2], L, invL);
    v.w = q[i];
    sorted[p] = v;
    perm[p] = i;
}

__device__ __forceinline__ double block_sum_d(double v, double* sbuf) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sbuf[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (warp == 0) {
        r = lane < (int)(blockDim.x >> 5) ? sbuf[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    return r;
}

// Stencil of a home cell: the (2K+1)^3 cells within K cells per direction
// (cells of edge >= rc / K, so that every pair within rc has both ends in
// such a pair of cells), each a distinct periodic image since nc >= 2K+1.
constexpr int kMaxStencil = 343;   // K <= 3
#ifndef SE_RS_THREADS
#define SE_RS_THREADS 192
#endif
constexpr int kPairThreads = SE_RS_THREADS;
#ifndef SE_RS_R32
#define SE_RS_R32 3   // home particles per thread, single precision
#endif

template <typename T>
__global__ void __launch_bounds__(kPairThreads)
k_rs_pairs(const typename R4<T>::type* __restrict__ sorted, const int* __restrict__ start,
           const int* __restrict__ perm, int nc, int K, T L, T rc2, T xi, T c2xi, T kc, int cap,
           T* __restrict__ phi, T* __restrict__ F, int accumulate, double* __restrict__ partials,
           unsigned* ticket, double* E_out) {
    using V = typename R4<T>::type;
    extern __shared__ __align__(32) unsigned char smem_raw[];
    V* nb = reinterpret_cast<V*>(smem_raw);
    __shared__ int s_b0[kMaxStencil], s_off[kMaxStencil + 1];
    __shared__ unsigned char s_sh[kMaxStencil];   // image shift per axis: 0, 1 (-L), 2 (+L)
    // hit queues of the double-precision sum: 32 S entries per set of lanes
    __shared__ unsigned short s_q[sizeof(T) == 8 ? 32 * kPairThreads : 1];
    __shared__ double sbuf[32];
    __shared__ bool last;
    const int cid = blockIdx.x;
    const int cx = cid / (nc * nc), cy = (cid / nc) % nc, cz = cid % nc;
    const int h0 = start[cid], nh = start[cid + 1] - h0;
    const int W = 2 * K + 1, W3 = W * W * W;
    // the stencil's cells: range and image shift, then offsets by a one-warp scan
    for (int k = threadIdx.x; k < W3; k += blockDim.x) {
        int nx = cx + k / (W * W) - K, ny = cy + (k / W) % W - K, nz = cz + k % W - K;
        unsigned char sh = 0;
        if (nx < 0) { nx += nc; sh |= 1; } else if (nx >= nc) { nx -= nc; sh |= 2; }
        if (ny < 0) { ny += nc; sh |= 4; } else if (ny >= nc) { ny -= nc; sh |= 8; }
        if (nz < 0) { nz += nc; sh |= 16; } else if (nz >= nc) { nz -= nc; sh |= 32; }
        const int nid = (nx * nc + ny) * nc + nz;
        const int b0 = start[nid];
        s_b0[k] = b0;
        s_off[k + 1] = start[nid + 1] - b0;   // count, scanned below
        s_sh[k] = sh;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        int carry = 0;
        if (lane == 0) s_off[0] = 0;
        for (int base = 0; base < W3; base += 32) {
            const int k = base + lane;
            int v = k < W3 ? s_off[k + 1] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += y;
            }
            if (k < W3) s_off[k + 1] = carry + v;
            carry += __shfl_sync(0xffffffffu, v, 31);
        }
    }
    __syncthreads();
    const int total = s_off[W3];
    // kR home particles per thread (single precision: 3, so that every
    // candidate loaded from shared memory is tested against three of them); S
    // lanes per set of kR particles, S the largest power of two up to 32 with
    // 2 S ceil(nh / kR) <= the block's threads
    constexpr int kR = sizeof(T) == 4 ? SE_RS_R32 : 1;
    const int nset = (nh + kR - 1) / kR;
    int S = 1;
    while (S < 32 && 2 * S * nset <= (int)blockDim.x) S <<= 1;
    const int sets = blockDim.x / S;
    const int per_pass = sets * kR;
    const int s = threadIdx.x % S, set = threadIdx.x / S;
    // the S lanes of a set: aligned, adjacent lanes of one warp
    const unsigned gmask = S == 32 ? 0xffffffffu
                                   : ((1u << S) - 1u) << ((threadIdx.x & 31) & ~(S - 1));
    double e_loc = 0.0;
    for (int pass0 = 0; pass0 < nh; pass0 += per_pass) {
        int li[kR];
        bool act[kR];
        V me[kR];
        T ph[kR], fx[kR], fy[kR], fz[kR];
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            li[r] = pass0 + set + r * sets;
            act[r] = li[r] < nh;
            if (act[r]) {
                me[r] = sorted[h0 + li[r]];
            } else {   // far from every candidate: no hits
                me[r].x = me[r].y = me[r].z = T(1e18);
                me[r].w = T(0);
            }
            ph[r] = fx[r] = fy[r] = fz[r] = T(0);
        }
        for (int c0 = 0; c0 < total; c0 += cap) {
            const int filled = min(cap, total - c0);
            __syncthreads();
            for (int t = threadIdx.x; t < filled; t += blockDim.x) {
                const int g = c0 + t;
                int lo = 0, hi = W3 - 1;   // the cell k with s_off[k] <= g < s_off[k + 1]
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (s_off[mid] <= g) lo = mid; else hi = mid - 1;
                }
                V v = sorted[s_b0[lo] + g - s_off[lo]];
                const unsigned sh = s_sh[lo];
                v.x += (sh & 1) ? -L : ((sh & 2) ? L : T(0));
                v.y += (sh & 4) ? -L : ((sh & 8) ? L : T(0));
                v.z += (sh & 16) ? -L : ((sh & 32) ? L : T(0));
                nb[t] = v;
            }
            __syncthreads();
            if (!act[0]) continue;   // act[r] implies act[0]
            // 32 candidates per lane at a time: distance tests into bit masks,
            // then the erfc terms of the hits only
            for (int jb = 0; jb < filled; jb += 32 * S) {   // uniform over the set
                const int j0 = jb + s;
                unsigned mask[kR];
#pragma unroll
                for (int r = 0; r < kR; ++r) mask[r] = 0u;
#pragma unroll 8
                for (int b = 0; b < 32; ++b) {
                    const int j = j0 + b * S;
                    if (j < filled) {
                        const V n = nb[j];
#pragma unroll
                        for (int r = 0; r < kR; ++r) {
                            const T dx = me[r].x - n.x, dy = me[r].y - n.y, dz = me[r].z - n.z;
                            const T r2 = dx * dx + dy * dy + dz * dz;
                            if (r2 < rc2 && r2 > T(0)) mask[r] |= 1u << b;
                        }
                    }
                }
                if constexpr (kR == 1) {
                    // double: the hit terms dominate, so the set's hits are
                    // queued in shared memory and shared out evenly (the set
                    // pays for its mean hit count per lane, not its largest)
                    unsigned short* qg = s_q + set * (32 * S);
                    const int cnt = __popc(mask[0]);
                    int pre = cnt;   // inclusive scan over the set's lanes
                    for (int o = 1; o < S; o <<= 1) {
                        const int y = __shfl_up_sync(gmask, pre, o, S);
                        if (s >= o) pre += y;
                    }
                    const int tot = __shfl_sync(gmask, pre, S - 1, S);
                    int w = pre - cnt;
                    unsigned m = mask[0];
                    while (m) {
                        const int b = __ffs(m) - 1;
                        m &= m - 1u;
                        qg[w++] = (unsigned short)(j0 + b * S);
                    }
                    __syncwarp(gmask);
                    for (int t = s; t < tot; t += S) {
                        const V n = nb[qg[t]];
                        const T dx = me[0].x - n.x, dy = me[0].y - n.y, dz = me[0].z - n.z;
                        const T r2 = dx * dx + dy * dy + dz * dz;
                        T ec, fr;
                        pair_terms(r2, rsqrtR(r2), xi, c2xi, ec, fr);
                        ph[0] += n.w * ec;
                        const T f = n.w * fr;
                        fx[0] += f * dx;
                        fy[0] += f * dy;
                        fz[0] += f * dz;
                    }
                    __syncwarp(gmask);   // the queue is rewritten by the next batch
                } else {
#pragma unroll
                    for (int r = 0; r < kR; ++r) {
                        unsigned m = mask[r];
                        while (m) {
                            const int b = __ffs(m) - 1;
                            m &= m - 1u;
                            const V n = nb[j0 + b * S];
                            const T dx = me[r].x - n.x, dy = me[r].y - n.y, dz = me[r].z - n.z;
                            const T r2 = dx * dx + dy * dy + dz * dz;
                            T ec, fr;
                            pair_terms(r2, rsqrtR(r2), xi, c2xi, ec, fr);
                            ph[r] += n.w * ec;
                            const T f = n.w * fr;
                            fx[r] += f * dx;
                            fy[r] += f * dy;
                            fz[r] += f * dz;
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            // sum over the S lanes of the set (adjacent lanes, aligned groups)
            for (int o = S >> 1; o > 0; o >>= 1) {
                ph[r] += __shfl_xor_sync(0xffffffffu, ph[r], o);
                fx[r] += __shfl_xor_sync(0xffffffffu, fx[r], o);
                fy[r] += __shfl_xor_sync(0xffffffffu, fy[r], o);
                fz[r] += __shfl_xor_sync(0xffffffffu, fz[r], o);
            }
            if (act[r] && s == 0) {
                const T pm = kc * (ph[r] - c2xi * me[r].w);
                const T fq = kc * me[r].w;
                const int o = perm[h0 + li[r]];
                if (phi) phi[o] = accumulate ? phi[o] + pm : pm;
                if (F) {
                    if (accumulate) {
                        F[3 * o] += fq * fx[r];
                        F[3 * o + 1] += fq * fy[r];
                        F[3 * o + 2] += fq * fz[r];
                    } else {
                        F[3 * o] = fq * fx[r];
                        F[3 * o + 1] = fq * fy[r];
                        F[3 * o + 2] = fq * fz[r];
                    }
                }
                e_loc += (double)me[r].w * (double)pm;
            }
        }
    }
    const double r = block_sum_d(e_loc, sbuf);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = r;
        __threadfence();
        const unsigned t = atomicAdd(ticket, 1u);
        last = t == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double e = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) e += partials[b];
    e = block_sum_d(e, sbuf);
    if (threadIdx.x == 0) {
        if (E_out) *E_out = accumulate ? *E_out + 0.5 * e : 0.5 * e;
        *ticket = 0u;
    }
}

}  // namespace

struct se_real {
    int64_t N = 0;
    double L = 0, xi = 0, rc = 0, kc = 1.0;
    int prec = SE_FP64;
    cudaStream_t stream = nullptr;
    int nc = 0, ncells = 0, K = 1;   // cells per dimension, stencil reach
    bool ready = false;
    int ready_prec = -1;
    int* count = nullptr;
    int* start = nullptr;
    int* cell_of = nullptr;
    int* slot = nullptr;
    int* perm = nullptr;
    void* sorted = nullptr;
    double* partials = nullptr;
    unsigned* ticket = nullptr;
};

namespace {

void rs_release(se_real* r) {
    void* b[] = {r->count, r->start, r->cell_of, r->slot, r->perm, r->sorted, r->partials, r->ticket};
    for (void* p : b)
        if (p) cudaFree(p);
    r->count = r->start = r->cell_of = r->slot = r->perm = nullptr;
    r->sorted = nullptr;
    r->partials = nullptr;
    r->ticket = nullptr;
    r->ready = false;
}

int rs_alloc(void** p, size_t bytes) {
    return cudaMalloc(p, bytes ? bytes : 16) == cudaSuccess ? SE_OK : SE_ERR_NOMEM;
}

int rs_prepare(se_real* r) {
    if (r->ready && r->ready_prec == r->prec) return SE_OK;
    rs_release(r);
    const size_t N = (size_t)r->N, ts = r->prec == SE_FP64 ? 8 : 4;
    int rc = SE_OK;
    if (rc == SE_OK) rc = rs_alloc((void**)&r->count, (size_t)r->ncells * sizeof(int));
    if (rc == SE_OK) rc = rs_alloc((void**)&r->start, ((size_t)r->ncells + 1) * sizeof(int));
    if (rc == SE_OK) rc = rs_alloc((void**)&r->cell_of, N * sizeof(int));
    if (rc == SE_OK) rc = rs_alloc((void**)&r->slot, N * sizeof(int));
    if (rc == SE_OK) rc = rs_alloc((void**)&r->perm, N * sizeof(int));
    if (rc == SE_OK) rc = rs_alloc(&r->sorted, N * 4 * ts);
    if (rc == SE_OK) rc = rs_alloc((void**)&r->partials, (size_t)r->ncells * sizeof(double));
    if (rc == SE_OK) rc = rs_alloc((void**)&r->ticket, sizeof(unsigned));
    if (rc == SE_OK && (cudaMemset(r->count, 0, (size_t)r->ncells * sizeof(int)) != cudaSuccess ||
                        cudaMemset(r->ticket, 0, sizeof(unsigned)) != cudaSuccess))
        rc = SE_ERR_CUDA;
    if (rc != SE_OK) {
        rs_release(r);
        return rc;
    }
    r->ready = true;
    r->ready_prec = r->prec;
    return SE_OK;
}

template <typename T>
int rs_run(se_real* r, const void* xyz, const void* q, void* F, void* phi, double* E, int acc) {
    using V = typename R4<T>::type;
    const int N = (int)r->N, nc = r->nc;
    const T L = (T)r->L, invL = (T)(1.0 / r->L), cscale = (T)(nc / r->L);
    const int nb = (N + kThreads - 1) / kThreads;
    cudaStream_t s = r->stream;
    k_rs_count<T><<<nb, kThreads, 0, s>>>((const T*)xyz, N, L, invL, cscale, nc, r->count,
                                          r->cell_of, r->slot);
    k_rs_scan<<<1, 1024, 0, s>>>(r->count, r->start, r->ncells);
    k_rs_scatter<T><<<nb, kThreads, 0, s>>>((const T*)xyz, (const T*)q, N, L, invL, r->cell_of,
                                            r->slot, r->start, (V*)r->sorted, r->perm);
    const int cap = (int)(kNbSmem / sizeof(V));
    if (cudaFuncSetAttribute(k_rs_pairs<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kNbSmem) != cudaSuccess)
        return SE_ERR_CUDA;
    const double c2xi = 2.0 * r->xi / sqrt(3.14159265358979323846);
    k_rs_pairs<T><<<r->ncells, kPairThreads, kNbSmem, s>>>(
        (const V*)r->sorted, r->start, r->perm, nc, r->K, L, (T)(r->rc * r->rc), (T)r->xi, (T)c2xi,
        (T)r->kc, cap, (T*)phi, (T*)F, acc, r->partials, r->ticket, E);
    return cudaGetLastError() == cudaSuccess ? SE_OK : SE_ERR_CUDA;
}

}  // namespace

// Cells per dimension and stencil reach for (L, rc); reach_user 1-3 forces
// K (SE_ERR_UNSUPPORTED if its 2K+1 cells do not fit), 0 chooses.
static int rs_layout(double L, double rc, int reach_user, int* K_out, int* nc_out) {
    if (floor(L / rc) < 3.0) return SE_ERR_UNSUPPORTED;   // r_c > L/3
    // stencil reach K: cells of edge >= rc/K, nc >= 2K+1 distinct images
    // (rc <= L/3 gives floor(2 L / rc) >= 6); K = 2 by default (a 5^3 stencil:
    // fewer candidates per particle than 3^3 cells of edge rc, and 8 times
    // the CTAs; measured 2-5 times faster than K = 1 and 1.2-1.5 times faster
    // than K = 3 on water boxes of 21.6k and 100k atoms), K = 3 when K = 2
    // leaves fewer than 512 cells (CTAs) for the GPU (1000 charges in a 3 nm
    // box: 1.3 times faster than K = 2)
    auto cells_for = [&](int K) {
        return (int)std::min<double>(floor(K * L / rc), kMaxCellsPerDim);
    };
    int K = 2;
    if (reach_user >= 1) K = reach_user;
    else if (cells_for(3) >= 7 && cells_for(2) * cells_for(2) * cells_for(2) < 512)
        K = 3;
    if (cells_for(K) < 2 * K + 1) return SE_ERR_UNSUPPORTED;
    *K_out = K;
    *nc_out = cells_for(K);
    return SE_OK;
}

extern "C" int se_real_create(se_real** out, int64_t N, double L, double xi, double rc) {
    if (!out) return SE_ERR_ARG;
    *out = nullptr;
    if (N < 0 || N >= ((int64_t)1 << 31) || !(L > 0.0) || !isfinite(L) || !(xi > 0.0) ||
        !isfinite(xi) || !(rc > 0.0) || !isfinite(rc))
        return SE_ERR_ARG;
    int K = 0, nc = 0;
    const int st = rs_layout(L, rc, 0, &K, &nc);
    if (st != SE_OK) return st;
    se_real* r = new (std::nothrow) se_real;
    if (!r) return SE_ERR_NOMEM;
    r->N = N;
    r->L = L;
    r->xi = xi;
    r->rc = rc;
    r->K = K;
    r->nc = nc;
    r->ncells = nc * nc * nc;
    *out = r;
    return SE_OK;
}

extern "C" int se_real_set_reach(se_real* r, int K) {
    if (!r || K < 0 || K > 3) return SE_ERR_ARG;
    int Kn = 0, nc = 0;
    const int st = rs_layout(r->L, r->rc, K, &Kn, &nc);
    if (st != SE_OK) return st;
    if (nc * nc * nc != r->ncells) rs_release(r);   // buffers sized by the cell count
    r->K = Kn;
    r->nc = nc;
    r->ncells = nc * nc * nc;
    return SE_OK;
}

extern "C" int se_real_destroy(se_real* r) {
    if (!r) return SE_OK;
    rs_release(r);
    delete r;
    return SE_OK;
}

extern "C" int se_real_set_precision(se_real* r, int prec) {
    if (!r || (prec != SE_FP64 && prec != SE_FP32)) return SE_ERR_ARG;
    r->prec = prec;
    return SE_OK;
}

extern "C" int se_real_set_prefactor(se_real* r, double kc) {
    if (!r || !(kc > 0.0) || !isfinite(kc)) return SE_ERR_ARG;
    r->kc = kc;
    return SE_OK;
}

extern "C" int se_real_set_stream(se_real* r, void* stream) {
    if (!r) return SE_ERR_ARG;
    r->stream = (cudaStream_t)stream;
    return SE_OK;
}

extern "C" int se_real_get_cells(const se_real* r, int* cells_per_dim) {
    if (!r || !cells_per_dim) return SE_ERR_ARG;
    *cells_per_dim = r->nc;
    return SE_OK;
}

extern "C" int se_real_evaluate(se_real* r, const void* xyz, const void* q, void* F, void* phi,
                                double* E, int accumulate) {
    if (!r || (r->N > 0 && (!xyz || !q))) return SE_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SE_ERR_CUDA;
    int rc = rs_prepare(r);
    if (rc != SE_OK) return rc;
    if (r->N == 0) {
        if (E && !accumulate && cudaMemsetAsync(E, 0, sizeof(double), r->stream) != cudaSuccess)
            return SE_ERR_CUDA;
        return SE_OK;
    }
    return r->prec == SE_FP64 ? rs_run<double>(r, xyz, q, F, phi, E, accumulate)
                              : rs_run<float>(r, xyz, q, F, phi, E, accumulate);
}
