// se_batch.cu -- many independent systems (each its own box L_s, grid M_s
// and N_s particles) through the single-precision SE pipeline with ONE launch
// per stage for all of them:
//
//   k_bbin       all particles: system, tile, slot; clears all fixed-point grids
//   k_bscatter   one block per system: tile offsets, particles in tile order,
//                charge checks and the system's fixed-point scale
//   k_bspread    one block per tile of every system (Eq. 3.5)
//   k_bslab_fwd  one block per x-slab of every system (z and y transforms)
//   k_bxpass     one block per (ky, kz chunk) of every system (x transforms,
//                Green's function, grid energy)
//   k_bslab_inv  one block per x-slab of every system (y and z inverse)
//   k_bgather    all particles (Eq. 3.9, Sec. 3.1)
//   k_bfinish    one block per system: energies
//
// The kernels run the device bodies of the single-system pipeline with the
// system's parameters; which system a block works on comes from tables built
// once on the host.  Kernels after the first are chained by programmatic
// dependent launch, and the whole sequence is replayed as one CUDA graph.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "../../include/se.h"
#define SE_BATCH_TU  // the single-system kernels live in se_kernels_fast.cu
#include "se_fast.cuh"
#include "se_launch.cuh"

namespace se {

struct SysParams {
    KParams<float> kp;   // the system's kernel parameters (N, M, P, tile, box, Gaussian)
    long long p0;        // first particle of the system in the concatenated arrays
    long long g0;        // offset of its M^3 grids
    long long c0;        // offset of its M x M x (M/2+1) complex grid and G table
    int t0;              // first global tile
    int tw0;             // offset of its twiddles
    int slab0;           // first global x-slab block
    int x0;              // first global x-pass block
    int nx;              // x-pass blocks of the system
    float invM3;         // 1 / M^3
    double e_scale;      // kc h^3 / (2 M^3) for the grid energy
};

struct BAcc {
    double sum_q, sum_absq;
    unsigned nonfinite;
    float fx_scale, fx_inv;
    float pad;
};

// Largest p0s[s] <= i (p0s ascending, p0s[0] = 0, S entries).
__device__ __forceinline__ int system_of(const long long* p0s, int S, long long i) {
    int lo = 0, hi = S - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p0s[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

constexpr int kBatchMaxSys = 1024;

__global__ void __launch_bounds__(256)
k_bbin(const float* __restrict__ xyz, const float* __restrict__ q, long long Ntot, int S,
       const SysParams* __restrict__ sys, int* __restrict__ tile_count, int* __restrict__ slot,
       int* __restrict__ tile_of, long long* __restrict__ g64, long long Gtot) {
    pdl_wait();
    pdl_launch_next();
    __shared__ long long p0s[kBatchMaxSys];
    for (int s = threadIdx.x; s < S; s += blockDim.x) p0s[s] = sys[s].p0;
    __syncthreads();
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < Gtot; i += stride)
        g64[i] = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < Ntot; i += stride) {
        const int s = system_of(p0s, S, i);
        const KParams<float>& kp = sys[s].kp;
        float t;
        const int cx = cell_of(wrap_coord(xyz[3 * i], kp.L, kp.invL), kp.invh, kp.M, &t);
        const int cy = cell_of(wrap_coord(xyz[3 * i + 1], kp.L, kp.invL), kp.invh, kp.M, &t);
        const int cz = cell_of(wrap_coord(xyz[3 * i + 2], kp.L, kp.invL), kp.invh, kp.M, &t);
        const int tile = sys[s].t0 + ((cx / kp.tile) * kp.nT + cy / kp.tile) * kp.nT + cz / kp.tile;
        slot[i] = atomicAdd(tile_count + tile, 1);
        tile_of[i] = tile;
    }
}

__global__ void __launch_bounds__(1024)
k_bscatter(const float* __restrict__ xyz, const float* __restrict__ q,
           const SysParams* __restrict__ sys, int* __restrict__ tile_count,
           const int* __restrict__ slot, const int* __restrict__ tile_of,
           int* __restrict__ tile_start, f4* __restrict__ sorted, int* __restrict__ perm,
           BAcc* __restrict__ bacc, int S, long long Ntot) {
    pdl_wait();
    pdl_launch_next();
    __shared__ int s_start[kScanSmem + 1];
    __shared__ df2 sbuf[32];
    __shared__ unsigned smax;
    __shared__ int sbad;
    const int s = blockIdx.x;
    const KParams<float>& kp = sys[s].kp;
    const int n = kp.ntiles, t0 = sys[s].t0;
    const long long p0 = sys[s].p0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        s_start[k] = tile_count[t0 + k];
        tile_count[t0 + k] = 0;   // consumed: ready for the next evaluation
    }
    if (threadIdx.x == 0) {
        smax = 0u;
        sbad = 0;
    }
    __syncthreads();
    block_scan_smem(s_start, n);
    for (int k = threadIdx.x; k < n; k += blockDim.x) tile_start[t0 + k] = (int)(p0 + s_start[k]);
    if (s == S - 1 && threadIdx.x == 0) tile_start[t0 + n] = (int)Ntot;
    df2 sq = df_from(0.0f), sa = df_from(0.0f);
    float qm = 0.0f;
    int bad = 0;
    for (int li = threadIdx.x; li < kp.N; li += blockDim.x) {
        const long long i = p0 + li;
        const float x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2], qq = q[i];
        if (!(isfinite(x) && isfinite(y) && isfinite(z) && isfinite(qq))) ++bad;
        const int dst = (int)p0 + s_start[tile_of[i] - t0] + slot[i];
        f4 v;
        v.x = wrap_coord(x, kp.L, kp.invL);
        v.y = wrap_coord(y, kp.L, kp.invL);
        v.z = wrap_coord(z, kp.L, kp.invL);
        v.w = qq;
        sorted[dst] = v;
        perm[dst] = (int)i;
        sq = df_add(sq, df_from(qq));
        sa = df_add(sa, df_from(fabsf(qq)));
        qm = fmaxf(qm, fabsf(qq));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) qm = fmaxf(qm, __shfl_xor_sync(0xffffffffu, qm, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&smax, __float_as_uint(qm));
    if (bad) atomicAdd(&sbad, bad);
    const df2 a = block_sum_df(sq, sbuf);
    const df2 b = block_sum_df(sa, sbuf);
    if (threadIdx.x == 0) {
        BAcc r;
        r.sum_q = df_to_double(a);
        r.sum_absq = df_to_double(b);
        r.nonfinite = (unsigned)sbad;
        const int k = fx_shift_for((double)kp.qcg * (double)__uint_as_float(smax));
        r.fx_scale = ldexpf(1.0f, k);
        r.fx_inv = ldexpf(1.0f, -k);
        r.pad = 0.0f;
        bacc[s] = r;
    }
}

template <int P>
__global__ void __launch_bounds__(256)
k_bspread(const f4* __restrict__ sorted, const int* __restrict__ tile_start,
          unsigned long long* __restrict__ g64, const SysParams* __restrict__ sys,
          const BAcc* __restrict__ bacc, const int* __restrict__ tile_sys, int slab) {
    pdl_wait();
    pdl_launch_next();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ float sE3[P];
    const int s = tile_sys[blockIdx.x];
    const SysParams& sp = sys[s];
    const int tile = blockIdx.x - sp.t0;
    const int pb = tile_start[sp.t0 + tile];
    spread_tile<P>(sorted + pb, tile_start[sp.t0 + tile + 1] - pb, g64 + sp.g0, sp.kp,
                   bacc[s].fx_scale, slab, tile, reinterpret_cast<unsigned*>(smem_raw), sE3);
}

// kz columns per block of the ensemble's x pass: 12 measured fastest for
// the 64-box water ensemble (its x pass 123 us against 137 at 8 and 193 at
// 4; the shared-memory arrays of xpass_body bound it below 16)
#ifndef SE_BX_KC
#define SE_BX_KC 12
#endif
constexpr int kBxKC = SE_BX_KC;

// threads of the ensemble's slab CTAs (one x-slab of one system each):
// 256 measured fastest for the 64-box water ensemble (0.821 ms per
// evaluation against 0.851 at 512 and 0.954 at 1024; 128 as 256), the
// slabs of many systems filling every SM at any size
#ifndef SE_BSLAB_THREADS
#define SE_BSLAB_THREADS 256
#endif
constexpr int kBSlabThreads = SE_BSLAB_THREADS;

__global__ void __launch_bounds__(kBSlabThreads)
k_bslab_fwd(const long long* __restrict__ g64, float2* __restrict__ C, const float2* __restrict__ tw,
            const SysParams* __restrict__ sys, const BAcc* __restrict__ bacc,
            const int* __restrict__ slab_sys) {
    pdl_wait();
    pdl_launch_next();
    extern __shared__ __align__(16) unsigned char sm[];
    const int s = slab_sys[blockIdx.x];
    const SysParams& sp = sys[s];
    slab_fwd_body(g64 + sp.g0, C + sp.c0, tw + sp.tw0, sp.kp.M, bacc[s].fx_inv,
                  blockIdx.x - sp.slab0, sm, SE_DFT_HALF_BATCH_R4);
}

__global__ void __launch_bounds__(256)
k_bxpass(float2* __restrict__ C, const float2* __restrict__ tw, const float* __restrict__ green,
         const SysParams* __restrict__ sys, const int* __restrict__ x_sys,
         float* __restrict__ x_part) {
    pdl_wait();
    pdl_launch_next();
    const int s = x_sys[blockIdx.x];
    const SysParams& sp = sys[s];
    const df2 e = xpass_body<kBxKC>(C + sp.c0, tw + sp.tw0, green + sp.c0, sp.kp.M, sp.invM3,
                             blockIdx.x - sp.x0);
    if (threadIdx.x == 0) {
        x_part[2 * blockIdx.x] = e.hi;
        x_part[2 * blockIdx.x + 1] = e.lo;
    }
}

__global__ void __launch_bounds__(kBSlabThreads)
k_bslab_inv(const float2* __restrict__ C, float* __restrict__ R, const float2* __restrict__ tw,
            const SysParams* __restrict__ sys, const int* __restrict__ slab_sys) {
    pdl_wait();
    pdl_launch_next();
    extern __shared__ __align__(16) unsigned char sm[];
    const int s = slab_sys[blockIdx.x];
    const SysParams& sp = sys[s];
    slab_inv_body(C + sp.c0, R + sp.g0, tw + sp.tw0, sp.kp.M, blockIdx.x - sp.slab0, sm,
                  SE_DFT_HALF_BATCH_R4);
}

template <int P>
__global__ void __launch_bounds__(256)
k_bgather(const f4* __restrict__ sorted, const int* __restrict__ perm, const float* __restrict__ R,
          const SysParams* __restrict__ sys, int S, long long Ntot, float* __restrict__ phi,
          float* __restrict__ F, float* __restrict__ e_part) {
    constexpr int D = pick_d(P), G = P / D, GPW = 32 / G;
    pdl_wait();
    pdl_launch_next();
    __shared__ long long p0s[kBatchMaxSys];
    for (int s = threadIdx.x; s < S; s += blockDim.x) p0s[s] = sys[s].p0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gi = lane / G, k = lane - gi * G;
    const long long gpb = (blockDim.x >> 5) * GPW;
    for (long long pb = blockIdx.x * gpb + warp * GPW; pb < Ntot; pb += gridDim.x * gpb) {
        const long long p = pb + gi;
        const bool valid = (gi < GPW) && (p < Ntot);
        float vphi = 0.f, vfx = 0.f, vfy = 0.f, vfz = 0.f, qq = 0.f;
        int s = 0;
        if (valid) {
            s = system_of(p0s, S, p);
            const f4 v = sorted[p];
            qq = v.w;
            GatherPrep<float, P> g;
            gather_prep<float, P>(v, sys[s].kp, k, g);
            gather_accum<float, P>(g, R + sys[s].g0, sys[s].kp, sys[s].kp.E3, vphi, vfx, vfy, vfz);
        }
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
            const KParams<float>& kp = sys[s].kp;
            const float ph = vphi * kp.phi_scale;
            const float fs = qq * kp.F_scale;
            const int orig = perm[p];
            if (phi) phi[orig] = ph;
            if (F) {
                F[3 * (long long)orig] = fs * vfx;
                F[3 * (long long)orig + 1] = fs * vfy;
                F[3 * (long long)orig + 2] = fs * vfz;
            }
            e_part[p] = 0.5f * qq * ph;
        }
    }
}

// Gather by tiles of every system, for dense tiles: CTA t stages the real
// grid over global tile t's region of its system in shared memory, gathers
// the tile's particles (tile order) from it and leaves the tile's energy
// partial 1/2 sum q phi (a double-float pair) in e_tile[t].
template <int P>
__global__ void __launch_bounds__(256, P <= 8 ? 4 : 1)
k_bgather_tile(const f4* __restrict__ sorted, const int* __restrict__ perm,
               const int* __restrict__ tile_start, const float* __restrict__ R,
               const SysParams* __restrict__ sys, const int* __restrict__ tile_sys,
               float* __restrict__ phi, float* __restrict__ F, float* __restrict__ e_tile) {
    // two z points per lane for small supports (half the lanes of k_gather per
    // particle): the per-particle set-up and the lane reduction are shared by
    // fewer lanes, each with twice the grid points
    constexpr int D = P <= 8 ? 2 * pick_d(P) : pick_d(P), G = P / D, GPW = 32 / G;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* reg = reinterpret_cast<float*>(smem_raw);
    __shared__ df2 sbuf[32];
    __shared__ float sE3[P];
    const int s = tile_sys[blockIdx.x];
    const SysParams& sp = sys[s];
    const KParams<float>& kp = sp.kp;
    const int tile = blockIdx.x - sp.t0;
    if (threadIdx.x < P) sE3[threadIdx.x] = kp.E3[threadIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gi = lane / G, k = lane - gi * G;
    const int group = warp * GPW + gi, ngroups = (blockDim.x >> 5) * GPW;
    const int M = kp.M, nT = kp.nT, TT = kp.tile;
    const int t0x = (tile / (nT * nT)) * TT, t0y = ((tile / nT) % nT) * TT, t0z = (tile % nT) * TT;
    const int Rx = min(TT, M - t0x) + P - 1, Ry = min(TT, M - t0y) + P - 1,
              Rz = min(TT, M - t0z) + P - 1;
    pdl_wait();
    pdl_launch_next();
    const int pb = tile_start[blockIdx.x], n = tile_start[blockIdx.x + 1] - pb;
    TilePrep<P, D> tp;
    int orig = -1;
    if (gi < GPW && group < n) {
        tile_prep<P, D>(sorted[pb + group], kp, k, t0x, t0y, t0z, Ry, Rz, tp);
        orig = perm[pb + group];
    }
    load_region(R + sp.g0, M, t0x - P / 2 + 1, t0y - P / 2 + 1, t0z - P / 2 + 1, Rx, Ry, Rz,
                region_stride<P>(Rz), reg);
    __syncthreads();
    df2 e_df = df_from(0.0f);
    for (int p0 = 0; p0 < n; p0 += ngroups) {
        const int p = p0 + group;
        const bool valid = gi < GPW && p < n;
        float vphi = 0.0f, vfx = 0.0f, vfy = 0.0f, vfz = 0.0f;
        if (valid) {
            if (p0 != 0) {
                tile_prep<P, D>(sorted[pb + p], kp, k, t0x, t0y, t0z, Ry, Rz, tp);
                orig = perm[pb + p];
            }
            tile_accum<P, D>(tp, reg, Ry, Rz, sE3, vphi, vfx, vfy, vfz);
        }
        gather_emit<P, G>(k, valid, orig, tp.q, vphi, vfx, vfy, vfz, kp, phi, F, 1.0f, 1.0f, e_df);
    }
    const df2 r = block_sum_df(e_df, sbuf);
    if (threadIdx.x == 0) {
        e_tile[2 * blockIdx.x] = 0.5f * r.hi;    // exact: a power-of-two scale
        e_tile[2 * blockIdx.x + 1] = 0.5f * r.lo;
    }
}

__global__ void __launch_bounds__(256)
k_bfinish(const float* __restrict__ e_part, const float* __restrict__ e_tile, int tiled,
          const float* __restrict__ x_part, const SysParams* __restrict__ sys,
          double* __restrict__ E, double* __restrict__ Eg) {
    pdl_wait();
    __shared__ df2 sbuf[32];
    const int s = blockIdx.x;
    const SysParams& sp = sys[s];
    df2 a = df_from(0.0f), b = df_from(0.0f);
    if (tiled) {   // one double-float partial per tile of the system
        for (int i = threadIdx.x; i < sp.kp.ntiles; i += blockDim.x) {
            df2 u;
            u.hi = e_tile[2 * (sp.t0 + i)];
            u.lo = e_tile[2 * (sp.t0 + i) + 1];
            a = df_add(a, u);
        }
    } else {
        for (int i = threadIdx.x; i < sp.kp.N; i += blockDim.x) a = df_add(a, df_from(e_part[sp.p0 + i]));
    }
    for (int i = threadIdx.x; i < sp.nx; i += blockDim.x) {
        df2 u;
        u.hi = x_part[2 * (sp.x0 + i)];
        u.lo = x_part[2 * (sp.x0 + i) + 1];
        b = df_add(b, u);
    }
    a = block_sum_df(a, sbuf);
    b = block_sum_df(b, sbuf);
    if (threadIdx.x == 0) {
        if (E) E[s] = df_to_double(a);
        if (Eg) Eg[s] = sp.e_scale * df_to_double(b);
    }
}

}  // namespace se

using se::BAcc;
using se::SysParams;

struct se_batch {
    int S = 0;
    int P = 0;
    double xi = 0, c_shape = 0.95, kc = 1.0;
    std::vector<long long> N;
    std::vector<double> L;
    std::vector<int> M;
    int tile = 8;
    cudaStream_t stream = nullptr;
    int device = -1;
    // derived
    long long Ntot = 0, Gtot = 0, Ctot = 0;
    int Ttot = 0, Stot = 0, Xtot = 0, TWtot = 0, maxM = 0;
    // device
    SysParams* d_sys = nullptr;
    BAcc* d_bacc = nullptr;
    int *tile_count = nullptr, *tile_start = nullptr, *slot = nullptr, *tile_of = nullptr;
    int *perm = nullptr, *tile_sys = nullptr, *slab_sys = nullptr, *x_sys = nullptr;
    se::f4* sorted = nullptr;
    long long* g64 = nullptr;
    float2* cgrid = nullptr;
    float* rgrid = nullptr;
    float* green = nullptr;
    float2* tw = nullptr;
    float* e_part = nullptr;
    float* e_tile = nullptr;   // per-tile energy partials of the tile gather
    float* x_part = nullptr;
    double* Eg = nullptr;
    int alloc_tiles = 0;   // capacity of the tile arrays
    // graph
    bool use_graph = true;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t gexec = nullptr;
    const void* gkey[5] = {};
    // stage timing (se_batch_set_timing): an event after each of the 8 stages
    static constexpr int kStages = 8;
    bool timing = false;
    bool ev_created = false;
    cudaEvent_t ev[kStages + 1] = {};
    double stage_ms[kStages] = {};
    int64_t stage_count = 0;
};

namespace {

const double kPiB = 3.14159265358979323846;

void free_all(se_batch* b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    void* p[] = {b->d_sys, b->d_bacc, b->tile_count, b->tile_start, b->slot, b->tile_of, b->perm,
                 b->tile_sys, b->slab_sys, b->x_sys, b->sorted, b->g64, b->cgrid, b->rgrid,
                 b->green, b->tw, b->e_part, b->x_part, b->Eg, b->e_tile};
    for (void* x : p)
        if (x) cudaFree(x);
    b->d_sys = nullptr;
    b->d_bacc = nullptr;
    b->tile_count = b->tile_start = b->slot = b->tile_of = b->perm = nullptr;
    b->tile_sys = b->slab_sys = b->x_sys = nullptr;
    b->sorted = nullptr;
    b->g64 = nullptr;
    b->cgrid = nullptr;
    b->rgrid = b->green = b->e_part = b->x_part = b->e_tile = nullptr;
    b->tw = nullptr;
    b->Eg = nullptr;
    b->alloc_tiles = 0;
}

template <typename T>
int balloc(T** p, size_t n) {
    if (n == 0) n = 1;
    return cudaMalloc((void**)p, n * sizeof(T)) == cudaSuccess ? SE_OK : SE_ERR_NOMEM;
}

// Per-system parameters and the block -> system tables for the current tile edge.
int build_tables(se_batch* b) {
    const int S = b->S;
    std::vector<SysParams> sp(S);
    std::vector<int> tile_sys, slab_sys, x_sys;
    long long p0 = 0, g0 = 0, c0 = 0;
    int t0 = 0, tw0 = 0, slab0 = 0, x0 = 0;
    for (int s = 0; s < S; ++s) {
        se::KParams<float> kp;
        se::KParams<double> kd;
        if (se::make_kparams_f64(b->N[s], b->L[s], b->xi, b->M[s], b->P, b->tile, &kd) != SE_OK)
            return SE_ERR_ARG;
        memset(&kp, 0, sizeof(kp));
        kp.N = kd.N;
        kp.M = kd.M;
        kp.P = kd.P;
        kp.tile = kd.tile;
        kp.nT = kd.nT;
        kp.ntiles = kd.ntiles;
        kp.L = (float)kd.L;
        kp.invL = (float)kd.invL;
        kp.h = (float)kd.h;
        kp.invh = (float)kd.invh;
        kp.beta = (float)kd.beta;
        kp.qcg = (float)kd.qcg;
        kp.phi_scale = (float)(b->kc * kd.phi_scale);
        kp.F_scale = (float)(b->kc * kd.F_scale);
        for (int a = 0; a < se::kMaxP; ++a) kp.E3[a] = (float)kd.E3[a];
        if (kp.ntiles > se::kScanLimit) return SE_ERR_UNSUPPORTED;
        const int M = b->M[s], Mh = M / 2 + 1;
        const int nch = (Mh + se::kBxKC - 1) / se::kBxKC;
        SysParams& q = sp[s];
        q.kp = kp;
        q.p0 = p0;
        q.g0 = g0;
        q.c0 = c0;
        q.t0 = t0;
        q.tw0 = tw0;
        q.slab0 = slab0;
        q.x0 = x0;
        q.nx = M * nch;
        q.invM3 = (float)(1.0 / ((double)M * M * M));
        const double h = b->L[s] / M;
        q.e_scale = b->kc * h * h * h / (2.0 * (double)M * M * M);
        for (int k = 0; k < kp.ntiles; ++k) tile_sys.push_back(s);
        for (int k = 0; k < M; ++k) slab_sys.push_back(s);
        for (int k = 0; k < M * nch; ++k) x_sys.push_back(s);
        p0 += b->N[s];
        g0 += (long long)M * M * M;
        c0 += (long long)M * M * Mh;
        t0 += kp.ntiles;
        tw0 += M;
        slab0 += M;
        x0 += M * nch;
    }
    b->Ttot = t0;
    b->Stot = slab0;
    b->Xtot = x0;
    if (b->Ttot > b->alloc_tiles) {
        if (b->tile_count) cudaFree(b->tile_count);
        if (b->tile_start) cudaFree(b->tile_start);
        if (b->tile_sys) cudaFree(b->tile_sys);
        if (b->e_tile) cudaFree(b->e_tile);
        b->tile_count = b->tile_start = b->tile_sys = nullptr;
        b->e_tile = nullptr;
        int rc = SE_OK;
        if (rc == SE_OK) rc = balloc(&b->tile_count, b->Ttot);
        if (rc == SE_OK) rc = balloc(&b->tile_start, b->Ttot + 1);
        if (rc == SE_OK) rc = balloc(&b->tile_sys, b->Ttot);
        if (rc == SE_OK) rc = balloc(&b->e_tile, 2 * (size_t)b->Ttot);
        if (rc != SE_OK) return rc;
        b->alloc_tiles = b->Ttot;
    }
    if (cudaMemcpy(b->d_sys, sp.data(), S * sizeof(SysParams), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->tile_sys, tile_sys.data(), tile_sys.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->slab_sys, slab_sys.data(), slab_sys.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->x_sys, x_sys.data(), x_sys.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(b->tile_count, 0, (size_t)b->Ttot * sizeof(int)) != cudaSuccess)
        return SE_ERR_CUDA;
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    return SE_OK;
}

int prepare_batch(se_batch* b) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SE_ERR_CUDA;
    if (b->d_sys && b->device == dev) return SE_OK;
    free_all(b);
    b->device = dev;
    const int S = b->S;
    long long Ntot = 0, Gtot = 0, Ctot = 0;
    int TW = 0, slabs = 0, xs = 0, maxM = 0;
    for (int s = 0; s < S; ++s) {
        const long long M = b->M[s], Mh = M / 2 + 1;
        Ntot += b->N[s];
        Gtot += M * M * M;
        Ctot += M * M * Mh;
        TW += (int)M;
        slabs += (int)M;
        xs += (int)(M * ((Mh + se::kBxKC - 1) / se::kBxKC));
        maxM = std::max(maxM, (int)M);
    }
    b->Ntot = Ntot;
    b->Gtot = Gtot;
    b->Ctot = Ctot;
    b->TWtot = TW;
    b->maxM = maxM;
    int rc = SE_OK;
    if (rc == SE_OK) rc = balloc(&b->d_sys, S);
    if (rc == SE_OK) rc = balloc(&b->d_bacc, S);
    if (rc == SE_OK) rc = balloc(&b->slot, Ntot);
    if (rc == SE_OK) rc = balloc(&b->tile_of, Ntot);
    if (rc == SE_OK) rc = balloc(&b->perm, Ntot);
    if (rc == SE_OK) rc = balloc(&b->sorted, Ntot);
    if (rc == SE_OK) rc = balloc(&b->e_part, Ntot);
    if (rc == SE_OK) rc = balloc(&b->g64, Gtot);
    if (rc == SE_OK) rc = balloc(&b->rgrid, Gtot);
    if (rc == SE_OK) rc = balloc(&b->cgrid, Ctot);
    if (rc == SE_OK) rc = balloc(&b->green, Ctot);
    if (rc == SE_OK) rc = balloc(&b->tw, TW);
    if (rc == SE_OK) rc = balloc(&b->slab_sys, slabs);
    if (rc == SE_OK) rc = balloc(&b->x_sys, xs);
    if (rc == SE_OK) rc = balloc(&b->x_part, 2 * (size_t)xs);
    if (rc == SE_OK) rc = balloc(&b->Eg, S);
    if (rc != SE_OK) {
        free_all(b);
        return rc;
    }
    // Green's function tables (float) and twiddles, per system
    std::vector<float> green((size_t)Ctot), tw(2 * (size_t)TW);
    size_t gc = 0, tc = 0;
    for (int s = 0; s < S; ++s) {
        const int M = b->M[s], Mh = M / 2 + 1;
        const double h = b->L[s] / M;
        const double w = b->P * h / 2.0, m = b->c_shape * sqrt(kPiB * b->P);
        const double eta = (2.0 * w * b->xi / m) * (2.0 * w * b->xi / m);
        const double t = 2.0 * kPiB / b->L[s];
        for (int kx = 0; kx < M; ++kx) {
            const int sx = (2 * kx <= M) ? kx : kx - M;
            for (int ky = 0; ky < M; ++ky) {
                const int sy = (2 * ky <= M) ? ky : ky - M;
                for (int kz = 0; kz < Mh; ++kz) {
                    const double n2 = (double)sx * sx + (double)sy * sy + (double)kz * kz;
                    double v = 0.0;
                    if (n2 > 0) {
                        const double k2 = t * t * n2;
                        v = 4.0 * kPiB * exp(-(1.0 - eta) * k2 / (4.0 * b->xi * b->xi)) / k2;
                    }
                    green[gc++] = (float)v;
                }
            }
        }
        for (int r = 0; r < M; ++r) {
            double c = cos(2.0 * kPiB * r / M), sn = sin(2.0 * kPiB * r / M);
            if ((4 * r) % M == 0) {
                const int q4 = (4 * r) / M;
                c = q4 == 0 ? 1.0 : (q4 == 2 ? -1.0 : 0.0);
                sn = q4 == 1 ? 1.0 : (q4 == 3 ? -1.0 : 0.0);
            }
            tw[tc++] = (float)c;
            tw[tc++] = (float)sn;
        }
    }
    if (cudaMemcpy(b->green, green.data(), green.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->tw, tw.data(), tw.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
        free_all(b);
        return SE_ERR_CUDA;
    }
    rc = build_tables(b);
    if (rc != SE_OK) free_all(b);
    return rc;
}

template <int P>
cudaError_t launch_bspread(se_batch* b, cudaStream_t s) {
    const size_t R = (size_t)b->tile + P - 1;
    // one 32-bit accumulator per point, rows padded to the region stride
    const size_t plane = R * (size_t)se::region_stride<P>((int)R) * sizeof(unsigned);
    const int slab = (int)std::min(R, se::kSmemBudget / plane);
    if (slab < 1) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(se::k_bspread<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)se::kSmemBudget);
    if (e != cudaSuccess) return e;
    return se::launch_ex(se::k_bspread<P>, b->Ttot, se::kThreads, (size_t)slab * plane, s, true,
                         (const se::f4*)b->sorted, (const int*)b->tile_start,
                         (unsigned long long*)b->g64, (const SysParams*)b->d_sys,
                         (const BAcc*)b->d_bacc, (const int*)b->tile_sys, slab);
}

template <int P>
cudaError_t launch_bgather(se_batch* b, float* phi, float* F, cudaStream_t s) {
    constexpr int GPW = 32 / (P / se::pick_d(P));
    const long long gpb = (se::kThreads / 32) * GPW;
    const int blocks = (int)std::max(1LL, std::min((b->Ntot + gpb - 1) / gpb, 8192LL));
    return se::launch_ex(se::k_bgather<P>, blocks, se::kThreads, 0, s, true, (const se::f4*)b->sorted,
                         (const int*)b->perm, (const float*)b->rgrid, (const SysParams*)b->d_sys, b->S,
                         b->Ntot, phi, F, b->e_part);
}

template <int P>
cudaError_t launch_bgather_tile(se_batch* b, float* phi, float* F, cudaStream_t s) {
    const size_t R = (size_t)b->tile + P - 1;
    const size_t bytes = R * R * (size_t)se::region_stride<P>((int)R) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(se::k_bgather_tile<P>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    return se::launch_ex(se::k_bgather_tile<P>, b->Ttot, se::kThreads, bytes, s, true,
                         (const se::f4*)b->sorted, (const int*)b->perm, (const int*)b->tile_start,
                         (const float*)b->rgrid, (const SysParams*)b->d_sys,
                         (const int*)b->tile_sys, phi, F, b->e_tile);
}

// The tile gather for dense tiles (mean particles per tile x P^3 at least 8
// times the region) whose region fits the shared-memory budget.
bool batch_gather_tiled(const se_batch* b) {
    const double R = (double)b->tile + b->P - 1;
    const double RS = b->P <= 16 ? b->P + 15 : R;   // region_stride
    const double per_tile = (double)b->Ntot / std::max(1, b->Ttot);
    return R * R * RS * sizeof(float) <= (double)se::kTileGatherSmem &&
           per_tile * b->P * b->P * b->P >= 8.0 * R * R * R;
}

int batch_launch(se_batch* b, const float* xyz, const float* q, float* F, float* phi, double* E,
                 cudaStream_t s) {
    cudaError_t e;
    // stage timing: events between the launches (which then do not overlap)
    auto mark = [&](int k) {
        if (b->timing) cudaEventRecord(b->ev[k], s);
    };
    mark(0);
    const int nbin = (int)std::max(1LL, std::min((std::max(b->Ntot, b->Gtot) + 255) / 256, 4096LL));
    e = se::launch_ex(se::k_bbin, nbin, se::kThreads, 0, s, false, xyz, q, b->Ntot, b->S,
                      (const SysParams*)b->d_sys, b->tile_count, b->slot, b->tile_of, b->g64, b->Gtot);
    if (e != cudaSuccess) return SE_ERR_CUDA;
    mark(1);
    e = se::launch_ex(se::k_bscatter, b->S, 1024, 0, s, true, xyz, q, (const SysParams*)b->d_sys,
                      b->tile_count, (const int*)b->slot, (const int*)b->tile_of, b->tile_start,
                      b->sorted, b->perm, b->d_bacc, b->S, b->Ntot);
    if (e != cudaSuccess) return SE_ERR_CUDA;
    mark(2);
    switch (b->P) {
#define SE_CASE(PP) case PP: e = launch_bspread<PP>(b, s); break;
        SE_FOR_EACH_P(SE_CASE)
#undef SE_CASE
        default: return SE_ERR_UNSUPPORTED;
    }
    if (e != cudaSuccess) return SE_ERR_CUDA;
    mark(3);
    const size_t slab = se::slab_smem_bytes(b->maxM);
    if (cudaFuncSetAttribute(se::k_bslab_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)slab) != cudaSuccess ||
        cudaFuncSetAttribute(se::k_bslab_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)slab) != cudaSuccess)
        return SE_ERR_CUDA;
    e = se::launch_ex(se::k_bslab_fwd, b->Stot, se::kBSlabThreads, slab, s, true, (const long long*)b->g64,
                      b->cgrid, (const float2*)b->tw, (const SysParams*)b->d_sys,
                      (const BAcc*)b->d_bacc, (const int*)b->slab_sys);
    if (e != cudaSuccess) return SE_ERR_CUDA;
    mark(4);
    e = se::launch_ex(se::k_bxpass, b->Xtot, se::kThreads, 0, s, true, b->cgrid, (const float2*)b->tw,
                      (const float*)b->green, (const SysParams*)b->d_sys, (const int*)b->x_sys,
                      b->x_part);
    if (e != cudaSuccess) return SE_ERR_CUDA;
    mark(5);
    e = se::launch_ex(se::k_bslab_inv, b->Stot, se::kBSlabThreads, slab, s, true, (const float2*)b->cgrid,
                      b->rgrid, (const float2*)b->tw, (const SysParams*)b->d_sys,
                      (const int*)b->slab_sys);
    if (e != cudaSuccess) return SE_ERR_CUDA;
    mark(6);
    const bool tiled = batch_gather_tiled(b);
    switch (b->P) {
#define SE_CASE(PP) \
    case PP: e = tiled ? launch_bgather_tile<PP>(b, phi, F, s) : launch_bgather<PP>(b, phi, F, s); break;
        SE_FOR_EACH_P(SE_CASE)
#undef SE_CASE
        default: return SE_ERR_UNSUPPORTED;
    }
    if (e != cudaSuccess) return SE_ERR_CUDA;
    mark(7);
    e = se::launch_ex(se::k_bfinish, b->S, se::kThreads, 0, s, true, (const float*)b->e_part,
                      (const float*)b->e_tile, (int)tiled, (const float*)b->x_part,
                      (const SysParams*)b->d_sys, E, b->Eg);
    if (e != cudaSuccess) return SE_ERR_CUDA;
    mark(8);
    return SE_OK;
}

int batch_eval(se_batch* b, const void* xyz, const void* q, void* F, void* phi, double* E) {
    if (b->timing) {   // direct launches with events between them; waits for the stages
        const int rc = batch_launch(b, (const float*)xyz, (const float*)q, (float*)F, (float*)phi,
                                    E, b->stream);
        if (rc != SE_OK) return rc;
        if (cudaEventSynchronize(b->ev[se_batch::kStages]) != cudaSuccess) return SE_ERR_CUDA;
        for (int k = 0; k < se_batch::kStages; ++k) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, b->ev[k], b->ev[k + 1]) != cudaSuccess) return SE_ERR_CUDA;
            b->stage_ms[k] += ms;
        }
        ++b->stage_count;
        return SE_OK;
    }
    if (b->use_graph) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(b->stream, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
            const void* key[5] = {xyz, q, F, phi, E};
            bool match = b->gexec != nullptr;
            for (int i = 0; i < 5 && match; ++i) match = key[i] == b->gkey[i];
            if (!match) {
                if (b->gexec) cudaGraphExecDestroy(b->gexec);
                b->gexec = nullptr;
                if (!b->cap && cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess)
                    return SE_ERR_CUDA;
                cudaGraph_t g = nullptr;
                int rc = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess
                             ? SE_OK : SE_ERR_CUDA;
                if (rc == SE_OK) {
                    rc = batch_launch(b, (const float*)xyz, (const float*)q, (float*)F, (float*)phi, E, b->cap);
                    if (cudaStreamEndCapture(b->cap, &g) != cudaSuccess && rc == SE_OK) rc = SE_ERR_CUDA;
                }
                if (rc == SE_OK && cudaGraphInstantiate(&b->gexec, g, 0) != cudaSuccess) {
                    b->gexec = nullptr;
                    rc = SE_ERR_CUDA;
                }
                if (g) cudaGraphDestroy(g);
                if (rc != SE_OK) {
                    cudaGetLastError();
                    b->use_graph = false;
                    return batch_launch(b, (const float*)xyz, (const float*)q, (float*)F, (float*)phi, E,
                                        b->stream);
                }
                for (int i = 0; i < 5; ++i) b->gkey[i] = key[i];
            }
            return cudaGraphLaunch(b->gexec, b->stream) == cudaSuccess ? SE_OK : SE_ERR_CUDA;
        }
    }
    return batch_launch(b, (const float*)xyz, (const float*)q, (float*)F, (float*)phi, E, b->stream);
}

}  // namespace

extern "C" {

int se_batch_create(se_batch** out, int S, const int64_t* N, const double* L, const int* M,
                    double xi, int P) {
    if (!out) return SE_ERR_ARG;
    *out = nullptr;
    if (S < 1 || S > se::kBatchMaxSys || !N || !L || !M || !(xi > 0) || !isfinite(xi)) return SE_ERR_ARG;
    if ((P & 1) || P < 2 || P > se::kMaxP) return SE_ERR_UNSUPPORTED;
    long long Ntot = 0;
    for (int s = 0; s < S; ++s) {
        if (N[s] < 0 || !(L[s] > 0) || !isfinite(L[s]) || M[s] < P || M[s] > se::kFastMaxM)
            return SE_ERR_ARG;
        Ntot += N[s];
        se::KParams<double> kd;
        if (se::make_kparams_f64(N[s], L[s], xi, M[s], P, 8, &kd) != SE_OK) return SE_ERR_ARG;
    }
    if (Ntot > 0x7fffffffLL) return SE_ERR_ARG;
    se_batch* b = new (std::nothrow) se_batch();
    if (!b) return SE_ERR_NOMEM;
    b->S = S;
    b->P = P;
    b->xi = xi;
    b->N.assign(N, N + S);
    b->L.assign(L, L + S);
    b->M.assign(M, M + S);
    *out = b;
    return SE_OK;
}

int se_batch_destroy(se_batch* b) {
    if (!b) return SE_OK;
    free_all(b);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->ev_created)
        for (cudaEvent_t& e : b->ev) cudaEventDestroy(e);
    delete b;
    return SE_OK;
}

int se_batch_set_timing(se_batch* b, int enable) {
    if (!b) return SE_ERR_ARG;
    if (enable && !b->ev_created) {
        for (cudaEvent_t& e : b->ev)
            if (cudaEventCreate(&e) != cudaSuccess) return SE_ERR_CUDA;
        b->ev_created = true;
    }
    b->timing = enable != 0;
    return SE_OK;
}

int se_batch_get_timing(se_batch* b, double* ms, int nstages, int64_t* count, int reset) {
    if (!b || !ms || nstages < se_batch::kStages) return SE_ERR_ARG;
    for (int k = 0; k < se_batch::kStages; ++k) ms[k] = b->stage_ms[k];
    if (count) *count = b->stage_count;
    if (reset) {
        for (double& v : b->stage_ms) v = 0.0;
        b->stage_count = 0;
    }
    return SE_OK;
}

int se_batch_set_stream(se_batch* b, void* stream) {
    if (!b) return SE_ERR_ARG;
    b->stream = (cudaStream_t)stream;
    return SE_OK;
}

int se_batch_set_prefactor(se_batch* b, double kc) {
    if (!b || !isfinite(kc)) return SE_ERR_ARG;
    b->kc = kc;
    if (b->d_sys) return build_tables(b);
    return SE_OK;
}

int se_batch_set_tile(se_batch* b, int tile) {
    if (!b || tile < 2 || tile > 32) return SE_ERR_ARG;
    if (b->P <= 16 && tile > 16) tile = 16;   // the staged regions' row stride allows 16
    b->tile = tile;
    if (b->d_sys) return build_tables(b);
    return SE_OK;
}

int se_batch_set_graph(se_batch* b, int enable) {
    if (!b) return SE_ERR_ARG;
    b->use_graph = enable != 0;
    if (!b->use_graph && b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    return SE_OK;
}

int se_batch_evaluate(se_batch* b, const void* xyz, const void* q, void* F, void* phi, double* E) {
    if (!b || !xyz || !q) return SE_ERR_ARG;
    int rc = prepare_batch(b);
    if (rc != SE_OK) return rc;
    return batch_eval(b, xyz, q, F, phi, E);
}

int se_batch_grid_energy(se_batch* b, double* Eg) {
    if (!b || !Eg || !b->d_sys) return SE_ERR_ARG;
    return cudaMemcpyAsync(Eg, b->Eg, b->S * sizeof(double), cudaMemcpyDeviceToDevice, b->stream) == cudaSuccess
               ? SE_OK : SE_ERR_CUDA;
}

int se_batch_get_status(se_batch* b, int* status) {
    if (!b || !status) return SE_ERR_ARG;
    *status = SE_OK;
    if (!b->d_sys) return SE_OK;
    std::vector<BAcc> a(b->S);
    if (cudaMemcpyAsync(a.data(), b->d_bacc, b->S * sizeof(BAcc), cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return SE_ERR_CUDA;
    for (const BAcc& x : a) {
        if (x.nonfinite) {
            *status = SE_ERR_NONFINITE;
            return SE_OK;
        }
        if (fabs(x.sum_q) > 1e-10 * x.sum_absq) *status = SE_WARN_NONNEUTRAL;
    }
    return SE_OK;
}

int se_batch_autotune(se_batch* b, const void* xyz, const void* q, void* F, void* phi, double* E,
                      const int* candidates, int ncand, int reps, int* best_tile, float* best_ms) {
    if (!b || !xyz || !q || !candidates || ncand < 1 || reps < 1) return SE_ERR_ARG;
    int rc = prepare_batch(b);
    if (rc != SE_OK) return rc;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return SE_ERR_CUDA;
    int best = b->tile;
    float bms = 1e30f;
    for (int c = 0; c < ncand; ++c) {
        const int t = candidates[c];
        if (t < 2 || t > 32 || (b->P <= 16 && t > 16)) continue;
        b->tile = t;
        rc = build_tables(b);
        if (rc != SE_OK) continue;
        for (int w = 0; w < 3; ++w) batch_eval(b, xyz, q, F, phi, E);
        cudaEventRecord(e0, b->stream);
        for (int r = 0; r < reps; ++r) batch_eval(b, xyz, q, F, phi, E);
        cudaEventRecord(e1, b->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = SE_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= reps;
        if (ms < bms) {
            bms = ms;
            best = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->tile = best;
    int rc2 = build_tables(b);
    if (best_tile) *best_tile = best;
    if (best_ms) *best_ms = bms;
    return rc == SE_OK ? rc2 : rc;
}

}  // extern "C"
