// se_plan.cu -- libse host side: plans, device buffers, cuFFT plans and the
// C ABI declared in include/se.h.
//
// One evaluation (se_energy_force) enqueues, on the plan's stream, either the
// cuFFT pipeline (spread variants 1 and 2: FP64, or grids above 128^3):
//   k_bin (tile of each particle, slots, checks, tile offsets)
//   k_scatter (particles in tile order)
//   k_spread_{tiled,direct} (Eq. 3.5)
//   cuFFT R2C
//   k_scale (Eq. 3.6, grid energy; clears the spread grid for the next call)
//   cuFFT C2R
//   k_gather (Eq. 3.9 and the analytic force; energy 1/2 sum q phi)
// or the single-precision pipeline of se_fast.cuh (variant 3: k_fbin,
// k_fspread, k_slab_fwd, k_xpass, k_slab_inv, k_gather; variant 4: k_fdirect
// in place of the first two; variant 5: k_fbin, k_fspread, k_slab_fwd,
// k_xpass, then k_sinv_gather_cl, the inverse transform fused with the
// gather, and k_gfinish), and nothing else: no allocation, no memset, no
// host synchronisation except the final copy of the energy when the caller
// asks for it on the host.
#include <cufft.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <type_traits>
#include <vector>

#include "../../include/se.h"
#include "se_internal.h"

using se::Acc;
using se::KParams;

struct se_plan {
    // user parameters
    int64_t N = 0;
    double L = 0, xi = 0;
    int M = 0, P = 0;
    int prec = SE_FP64;
    double c_shape = 0.95, eta_user = 0.0;
    int eta_fixed = 0;
    double kc = 1.0;
    cudaStream_t stream = nullptr;
    int tune_variant = 0, tune_tile = 0;
    int force_mode = SE_FORCE_ANALYTIC;

    // derived (set by derive())
    double h = 0, w = 0, eta = 0, alpha = 0, cg = 0, m = 0;
    int tile = 0, nT = 0, ntiles = 0, variant = 0;
    int cap = 0;                   // tile bucket capacity (single-precision pipeline)

    // device state (prepare())
    bool ready = false;
    int ready_prec = -1;
    int ready_force = -1;
    int device = -1;
    void* grid_spread = nullptr;   // M^3 real: spread output, FFT input
    void* grid_gather = nullptr;   // M^3 real: inverse FFT output, gather input; with ik
                                   // forces 4 grids ik_gstride apart: Ht, then its x, y, z
                                   // derivatives
    void* cgrid_ik = nullptr;      // ik forces: 3 spectra ik_cstride apart, i k_d G/M^3 Hhat
    void* cgrid = nullptr;         // M x M x (M/2+1) complex
    double* green = nullptr;       // G(k) on the half spectrum (FP64)
    int* tile_count = nullptr;
    int* tile_start = nullptr;
    int* slot = nullptr;
    int* tile_of = nullptr;
    int* perm = nullptr;
    void* sorted = nullptr;
    void* bucket = nullptr;        // tile buckets (single-precision pipeline)
    int* bucket_idx = nullptr;     // their input positions
    long long* g64 = nullptr;      // fixed-point spread grid (single-precision pipeline)
    void* part = nullptr;          // variant 5: float4 [P][N] shares of the x-planes
    float* green_f = nullptr;      // G(k) table in float (single-precision pipeline)
    void* tw = nullptr;            // twiddles of the single-precision pipeline
    double* partials = nullptr;    // 8 x kMaxPartials
    unsigned* tickets = nullptr;   // 8 counters (see FastBufs)
    Acc* acc = nullptr;
    double* dE = nullptr;          // device energy for se_energy_force
    cufftHandle fwd = 0, inv = 0;
    bool have_fft = false;
    // staging buffers of se_energy_force_host
    void* h_xyz = nullptr;
    void* h_q = nullptr;
    void* h_F = nullptr;
    void* h_phi = nullptr;

    bool spread_clean = false;     // the spread grid is known to be zero
    bool have_spread = false, have_scale = false;

    // stage timing: a ring of event sets, one set (8 events) per evaluation
    static constexpr int kStages = 7, kRing = 64;
    bool timing = false;
    cudaEvent_t ev[kRing][kStages + 1] = {};
    bool ev_pending[kRing] = {};
    bool ev_created = false;
    int ev_cur = -1;               // set used by the evaluation in flight
    int ev_next = 0;
    double stage_ms[kStages] = {};
    int64_t stage_count = 0;

    // CUDA graph of one whole evaluation, replayed while its arguments match
    bool use_graph = true;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    const void* gkey[5] = {};
    double gkey_kc = 0.0;
    // se_energy_force_host with page-locked, mapped host buffers: one CUDA
    // graph in which the kernels read and write the host buffers directly,
    // replayed while the host pointers match; the reduction record comes back
    // to acc_host (pinned)
    cudaGraphExec_t hexec = nullptr;
    const void* hkey[4] = {};
    double hkey_kc = 0.0;
    Acc* acc_host = nullptr;
};

namespace {

const double kPi = 3.14159265358979323846;

int check_cuda(cudaError_t e) { return e == cudaSuccess ? SE_OK : SE_ERR_CUDA; }

// ---- stage timing ----
void fold_set(se_plan* p, int i) {
    if (!p->ev_pending[i]) return;
    cudaEventSynchronize(p->ev[i][se_plan::kStages]);
    for (int s = 0; s < se_plan::kStages; ++s) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p->ev[i][s], p->ev[i][s + 1]) == cudaSuccess)
            p->stage_ms[s] += ms;
    }
    p->stage_count += 1;
    p->ev_pending[i] = false;
}

// Start an evaluation's event set (no-op unless timing is on).
void timing_begin(se_plan* p) {
    p->ev_cur = -1;
    if (!p->timing || !p->ev_created) return;
    int i = p->ev_next;
    p->ev_next = (i + 1) % se_plan::kRing;
    fold_set(p, i);
    p->ev_cur = i;
    cudaEventRecord(p->ev[i][0], p->stream);
}

// Mark the end of stage s (0-based) of the evaluation in flight.
void timing_mark(se_plan* p, int s) {
    if (p->ev_cur < 0) return;
    cudaEventRecord(p->ev[p->ev_cur][s + 1], p->stream);
    if (s + 1 == se_plan::kStages) {
        p->ev_pending[p->ev_cur] = true;
        p->ev_cur = -1;
    }
}

#define SE_TRY(expr)                      \
    do {                                  \
        int _rc = (expr);                 \
        if (_rc != SE_OK) return _rc;     \
    } while (0)
#define SE_CUDA(expr) SE_TRY(check_cuda(expr))
#define SE_CUFFT(expr)                                   \
    do {                                                 \
        if ((expr) != CUFFT_SUCCESS) return SE_ERR_CUFFT; \
    } while (0)

size_t tsize(int prec) { return prec == SE_FP64 ? sizeof(double) : sizeof(float); }

// Spacing of the four real grids (values) and of the three derivative spectra
// (complex values) of ik forces: M^3 and M^2 (M/2+1) rounded up so that every
// grid starts on a 256-byte boundary (an odd M^3 would not).
size_t ik_gstride(const se_plan* p) { return ((size_t)p->M * p->M * p->M + 63) & ~(size_t)63; }
size_t ik_cstride(const se_plan* p) { return ((size_t)p->M * p->M * (p->M / 2 + 1) + 31) & ~(size_t)31; }

// Sec. 3 and Eq. 4.2: h = L/M, w = P h / 2, m = c sqrt(pi P),
// eta = (2 w xi / m)^2, alpha = 2 xi^2 / eta, c_g = (2 xi^2 / (pi eta))^{3/2}.
void derive(se_plan* p) {
    p->h = p->L / p->M;
    p->w = p->P * p->h / 2.0;
    p->m = p->c_shape * sqrt(kPi * p->P);
    p->eta = p->eta_fixed ? p->eta_user : (2.0 * p->w * p->xi / p->m) * (2.0 * p->w * p->xi / p->m);
    p->alpha = 2.0 * p->xi * p->xi / p->eta;
    p->cg = pow(2.0 * p->xi * p->xi / (kPi * p->eta), 1.5);
    // spreading variant and tile edge
    int tile = p->tune_tile > 0 ? p->tune_tile : 8;
    if (p->P <= 16 && tile > 16) tile = 16;   // the staged regions' row stride allows 16
    if (tile > p->M) tile = p->M;
    p->tile = tile;
    p->nT = (p->M + tile - 1) / tile;
    p->ntiles = p->nT * p->nT * p->nT;
    const bool fast_ok = p->prec != SE_FP64 && p->M <= se::kFastMaxM;
    int variant = p->tune_variant;
    if ((variant == 3 || variant == 5) && !fast_ok) variant = 0;
    if (variant == 4 && (p->prec == SE_FP64 || p->M > se::kFastMaxM)) variant = 0;
    // ik forces need the three extra inverse transforms of the cuFFT pipeline
    if (p->force_mode == SE_FORCE_IK && variant >= 3) variant = 0;
    if (variant == 0) {
        if (p->prec == SE_FP64) variant = p->P > 12 ? 2 : 1;
        else variant = (fast_ok && p->force_mode != SE_FORCE_IK) ? 3 : 1;
    }
    if (p->prec == SE_FP32 && variant == 2) variant = 1;  // the compensated sum needs the tiles
    p->variant = variant;
    // bucket capacity: twice the mean tile occupancy plus a margin, fuller
    // tiles spilling to the overflow list; for sparse tiles (mean within 3/4
    // of the particles one spread CTA takes per round), exactly one round, so
    // that no tile CTA needs a second one (the rare excess goes to the
    // overflow CTAs, which run beside the tiles)
    const int64_t mean = (p->N + p->ntiles - 1) / std::max(1, p->ntiles);
    const int64_t round = (256 / 32) * (32 / (p->P / se::pick_d(p->P)));
    int64_t cap = std::max<int64_t>(32, 2 * mean + 32);
    if (4 * mean <= 3 * round) cap = round;
    p->cap = (int)std::min<int64_t>(cap, std::max<int64_t>(32, p->N));
}

void drop_graph(se_plan* p) {
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    p->gexec = nullptr;
    if (p->hexec) cudaGraphExecDestroy(p->hexec);
    p->hexec = nullptr;
}

void release_device(se_plan* p) {
    drop_graph(p);
    if (p->have_fft) {
        cufftDestroy(p->fwd);
        cufftDestroy(p->inv);
        p->have_fft = false;
    }
    void* bufs[] = {p->grid_spread, p->grid_gather, p->cgrid, p->green, p->tile_count,
                    p->tile_start, p->slot, p->tile_of, p->perm, p->sorted, p->partials,
                    p->tickets, p->acc, p->dE, p->h_xyz, p->h_q, p->h_F, p->h_phi, p->g64, p->tw, p->green_f,
                    p->bucket, p->bucket_idx, p->cgrid_ik, p->part};
    for (void* b : bufs)
        if (b) cudaFree(b);
    p->grid_spread = p->grid_gather = p->cgrid = p->sorted = p->tw = p->bucket = nullptr;
    p->bucket_idx = nullptr;
    p->cgrid_ik = nullptr;
    p->part = nullptr;
    p->g64 = nullptr;
    p->green_f = nullptr;
    p->green = p->partials = p->dE = nullptr;
    p->tile_count = p->tile_start = p->slot = p->tile_of = p->perm = nullptr;
    p->tickets = nullptr;
    p->acc = nullptr;
    p->h_xyz = p->h_q = p->h_F = p->h_phi = nullptr;
    if (p->acc_host) cudaFreeHost(p->acc_host);
    p->acc_host = nullptr;
    p->ready = false;
    p->ready_prec = -1;
    p->ready_force = -1;
}

int dalloc(void** ptr, size_t bytes) {
    if (bytes == 0) bytes = 16;
    return cudaMalloc(ptr, bytes) == cudaSuccess ? SE_OK : SE_ERR_NOMEM;
}

template <typename T>
KParams<T> make_kparams(const se_plan* p) {
    KParams<T> kp;
    memset(&kp, 0, sizeof(kp));
    kp.N = (int)p->N;
    kp.M = p->M;
    kp.P = p->P;
    kp.tile = p->tile;
    kp.nT = p->nT;
    kp.ntiles = p->ntiles;
    kp.L = (T)p->L;
    kp.invL = (T)(1.0 / p->L);
    kp.h = (T)p->h;
    kp.invh = (T)((double)p->M / p->L);
    const double beta = p->alpha * p->h * p->h;
    kp.beta = (T)beta;
    kp.qcg = (T)p->cg;
    kp.phi_scale = (T)(p->kc * p->h * p->h * p->h * p->cg);
    kp.F_scale = (T)(-p->kc * 2.0 * p->alpha * p->h * p->h * p->h * p->h * p->cg);
    for (int a = 0; a < p->P; ++a) {
        const double ac = a - 0.5 * (p->P - 1);
        kp.E3[a] = (T)exp(-beta * ac * ac);
    }
    return kp;
}

// G(k) = 4 pi exp(-(1-eta) k^2 / (4 xi^2)) / k^2 on the half spectrum, G(0) = 0.
std::vector<double> green_table(const se_plan* p) {
    const int M = p->M, Mh = M / 2 + 1;
    std::vector<double> g((size_t)M * M * Mh);
    const double t = 2.0 * kPi / p->L;
    for (int kx = 0; kx < M; ++kx) {
        const int sx = (2 * kx <= M) ? kx : kx - M;
        for (int ky = 0; ky < M; ++ky) {
            const int sy = (2 * ky <= M) ? ky : ky - M;
            for (int kz = 0; kz < Mh; ++kz) {
                const double n2 = (double)sx * sx + (double)sy * sy + (double)kz * kz;
                double v = 0.0;
                if (n2 > 0) {
                    const double k2 = t * t * n2;
                    v = 4.0 * kPi * exp(-(1.0 - p->eta) * k2 / (4.0 * p->xi * p->xi)) / k2;
                }
                g[((size_t)kx * M + ky) * Mh + kz] = v;
            }
        }
    }
    return g;
}

int prepare(se_plan* p) {
    int dev = 0;
    SE_CUDA(cudaGetDevice(&dev));
    if (p->ready && p->ready_prec == p->prec && p->ready_force == p->force_mode && p->device == dev)
        return SE_OK;
    release_device(p);
    derive(p);
    p->device = dev;
    const size_t ts = tsize(p->prec);
    const size_t M3 = (size_t)p->M * p->M * p->M;
    const size_t nc = (size_t)p->M * p->M * (p->M / 2 + 1);
    const size_t N = (size_t)p->N;
    const bool fast = p->variant >= 3;
    const bool ik = p->force_mode == SE_FORCE_IK;
    int rc = SE_OK;
    if (rc == SE_OK && !fast) rc = dalloc(&p->grid_spread, M3 * ts);
    if (rc == SE_OK && fast) rc = dalloc((void**)&p->g64, M3 * sizeof(long long));
    const bool buckets = p->variant == 3 || p->variant == 5;
    if (rc == SE_OK && buckets)
        rc = dalloc(&p->bucket, (size_t)p->ntiles * p->cap * 4 * sizeof(float));
    if (rc == SE_OK && buckets)
        rc = dalloc((void**)&p->bucket_idx, (size_t)p->ntiles * p->cap * sizeof(int));
    if (rc == SE_OK && p->variant == 5)
        rc = dalloc(&p->part, N * (size_t)p->P * 4 * sizeof(float));
    if (rc == SE_OK && fast) rc = dalloc(&p->tw, (size_t)p->M * 2 * sizeof(float));
    if (rc == SE_OK && fast) rc = dalloc((void**)&p->green_f, nc * sizeof(float));
    if (rc == SE_OK) rc = dalloc(&p->grid_gather, ik ? 4 * ik_gstride(p) * ts : M3 * ts);
    if (rc == SE_OK && ik) rc = dalloc(&p->cgrid_ik, 3 * ik_cstride(p) * 2 * ts);
    if (rc == SE_OK) rc = dalloc(&p->cgrid, nc * 2 * ts);
    if (rc == SE_OK) rc = dalloc((void**)&p->green, nc * sizeof(double));
    if (rc == SE_OK) rc = dalloc((void**)&p->tile_count, (size_t)p->ntiles * sizeof(int));
    if (rc == SE_OK) rc = dalloc((void**)&p->tile_start, ((size_t)p->ntiles + 1) * sizeof(int));
    if (rc == SE_OK) rc = dalloc((void**)&p->slot, N * sizeof(int));
    if (rc == SE_OK) rc = dalloc((void**)&p->tile_of, N * sizeof(int));
    if (rc == SE_OK) rc = dalloc((void**)&p->perm, N * sizeof(int));
    if (rc == SE_OK) rc = dalloc(&p->sorted, N * 4 * ts);
    if (rc == SE_OK) rc = dalloc((void**)&p->partials, 8 * se::kMaxPartials * sizeof(double));
    if (rc == SE_OK) rc = dalloc((void**)&p->tickets, 8 * sizeof(unsigned));
    if (rc == SE_OK) rc = dalloc((void**)&p->acc, sizeof(Acc));
    if (rc == SE_OK) rc = dalloc((void**)&p->dE, sizeof(double));
    if (rc != SE_OK) {
        release_device(p);
        return rc;
    }
    std::vector<double> g = green_table(p);
    if (cudaMemcpy(p->green, g.data(), nc * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(p->tile_count, 0, (size_t)p->ntiles * sizeof(int)) != cudaSuccess ||
        cudaMemset(p->tickets, 0, 8 * sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(p->acc, 0, sizeof(Acc)) != cudaSuccess ||
        (!fast && cudaMemset(p->grid_spread, 0, M3 * ts) != cudaSuccess) ||
        (p->variant >= 3 && cudaMemset(p->g64, 0, M3 * sizeof(long long)) != cudaSuccess)) {
        release_device(p);
        return SE_ERR_CUDA;
    }
    if (fast) {
        // twiddles (cos, sin)(2 pi r / M), exact at the quarter turns
        std::vector<float> tw(2 * (size_t)p->M);
        for (int r = 0; r < p->M; ++r) {
            double c = cos(2.0 * kPi * r / p->M), sn = sin(2.0 * kPi * r / p->M);
            if ((4 * r) % p->M == 0) {
                const int q4 = (4 * r) / p->M;
                c = q4 == 0 ? 1.0 : (q4 == 2 ? -1.0 : 0.0);
                sn = q4 == 1 ? 1.0 : (q4 == 3 ? -1.0 : 0.0);
            }
            tw[2 * r] = (float)c;
            tw[2 * r + 1] = (float)sn;
        }
        std::vector<float> gf(nc);
        for (size_t i = 0; i < nc; ++i) gf[i] = (float)g[i];
        if (cudaMemcpy(p->tw, tw.data(), tw.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(p->green_f, gf.data(), nc * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
            release_device(p);
            return SE_ERR_CUDA;
        }
    }
    if (fast) {
        p->spread_clean = true;
        p->have_spread = p->have_scale = false;
        p->ready = true;
        p->ready_prec = p->prec;
        p->ready_force = p->force_mode;
        return SE_OK;
    }
    const cufftType tf = p->prec == SE_FP64 ? CUFFT_D2Z : CUFFT_R2C;
    const cufftType ti = p->prec == SE_FP64 ? CUFFT_Z2D : CUFFT_C2R;
    if (cufftPlan3d(&p->fwd, p->M, p->M, p->M, tf) != CUFFT_SUCCESS) {
        release_device(p);
        return SE_ERR_CUFFT;
    }
    if (cufftPlan3d(&p->inv, p->M, p->M, p->M, ti) != CUFFT_SUCCESS) {
        cufftDestroy(p->fwd);
        release_device(p);
        return SE_ERR_CUFFT;
    }
    p->have_fft = true;
    p->spread_clean = true;
    p->have_spread = p->have_scale = false;
    p->ready = true;
    p->ready_prec = p->prec;
    p->ready_force = p->force_mode;
    return SE_OK;
}

void invalidate(se_plan* p) {
    // parameters changed: rebuild tables and buffers at the next call
    if (p->ready) release_device(p);
    derive(p);
}

se::FastBufs fast_bufs(se_plan* p) {
    se::FastBufs b;
    b.g64 = p->g64;
    b.cgrid = p->cgrid;
    b.rgrid = (float*)p->grid_gather;
    b.tw = p->tw;
    b.green = p->green;
    b.green_f = p->green_f;
    b.tile_count = p->tile_count;
    b.bucket = p->bucket;
    b.bucket_idx = p->bucket_idx;
    b.tile_n = p->tile_start;
    b.cap = p->cap;
    b.over_idx = p->slot;
    b.wrapped = p->sorted;
    b.partials = p->partials;
    b.tickets = p->tickets;
    b.acc = p->acc;
    b.unsorted = p->variant == 4;
    b.part = p->part;
    return b;
}

void mark_cb(void* ctx, int s) { timing_mark(static_cast<se_plan*>(ctx), s); }


int fast_spread(se_plan* p, const void* xyz, const void* q) {
    const KParams<float> kp = make_kparams<float>(p);
    // the spread adds into g64 (fixed point, or float with variant 4), which
    // the forward slab kernel clears as it reads it
    if (!p->spread_clean)
        SE_CUDA(cudaMemsetAsync(p->g64, 0, (size_t)p->M * p->M * p->M * sizeof(long long), p->stream));
    p->spread_clean = false;
    timing_begin(p);
    SE_CUDA(se::fast_spread((const float*)xyz, (const float*)q, kp, fast_bufs(p), p->stream,
                            p->ev_cur >= 0, mark_cb, p));
    timing_mark(p, 2);
    p->have_spread = true;
    p->have_scale = false;
    return SE_OK;
}

int fast_scale(se_plan* p, double* E_grid) {
    const KParams<float> kp = make_kparams<float>(p);
    const double M3 = (double)p->M * p->M * p->M;
    const double e_scale = p->kc * p->h * p->h * p->h / (2.0 * M3);
    // variant 5 runs the inverse transform inside its gather; the grid energy
    // is summed here only when it is asked for
    const bool v5 = p->variant == 5;
    SE_CUDA(se::fast_transform(kp, fast_bufs(p), e_scale, E_grid, p->stream, p->ev_cur >= 0,
                               mark_cb, p, !v5));
    if (v5 && E_grid) SE_CUDA(se::fast_grid_energy(kp, fast_bufs(p), e_scale, E_grid, p->stream));
    p->spread_clean = true;
    p->have_scale = true;
    return SE_OK;
}

int fast_gather(se_plan* p, void* phi, void* F, double* E, const double* adj = nullptr) {
    const KParams<float> kp = make_kparams<float>(p);
    if (p->variant == 5) {   // the inverse transform fused with the gather
        SE_CUDA(se::fast_gather_slab(kp, fast_bufs(p), (float*)phi, (float*)F,
                                     p->partials + 4 * se::kMaxPartials, p->tickets + 2, 0.5, E,
                                     adj, p->stream));
        timing_mark(p, 6);
        return SE_OK;
    }
    // dense tiles: the tile gather, with or without forces (it stages the
    // grid once per tile, which outweighs the force sums it then skips)
    if (p->variant == 3 && se::fast_gather_tiled(kp)) {
        SE_CUDA(se::fast_gather(kp, fast_bufs(p), (float*)phi, (float*)F,
                                p->partials + 4 * se::kMaxPartials, p->tickets + 2, 0.5, E, adj,
                                p->stream));
        timing_mark(p, 6);
        return SE_OK;
    }
    if (!F && !adj) {   // potential (and energy) only, L2 reads: the plain window
        SE_CUDA(se::launch_gather_plain<float>(1, (const se::f4*)p->sorted, nullptr,
                                               (const float*)p->grid_gather,
                                               (size_t)p->M * p->M * p->M, (float*)phi, nullptr, kp,
                                               p->partials + 4 * se::kMaxPartials, p->tickets + 2,
                                               p->acc, 0.5, E, true, p->stream));
        timing_mark(p, 6);
        return SE_OK;
    }
    SE_CUDA(se::launch_gather_pdl((const se::f4*)p->sorted, nullptr, (const float*)p->grid_gather,
                                  (float*)phi, (float*)F, kp, p->partials + 4 * se::kMaxPartials,
                                  p->tickets + 2, p->acc, 0.5, E, adj, p->stream));
    timing_mark(p, 6);
    return SE_OK;
}

template <typename T>
int do_spread(se_plan* p, const void* xyz, const void* q) {
    const KParams<T> kp = make_kparams<T>(p);
    using V = se::v4_t<T>;
    const size_t M3 = (size_t)p->M * p->M * p->M;
    if (!p->spread_clean) SE_CUDA(cudaMemsetAsync(p->grid_spread, 0, M3 * sizeof(T), p->stream));
    timing_begin(p);
    SE_CUDA(se::launch_bin<T>((const T*)xyz, (const T*)q, kp, p->tile_count, p->slot, p->tile_of,
                              p->tile_start, p->partials, p->tickets + 0, p->acc, p->stream));
    timing_mark(p, 0);
    SE_CUDA(se::launch_scatter<T>((const T*)xyz, (const T*)q, kp, p->slot, p->tile_of,
                                  p->tile_start, (V*)p->sorted, p->perm, p->stream));
    timing_mark(p, 1);
    if (p->N > 0) {
        if (p->variant == 2)
            SE_CUDA(se::launch_spread_direct<T>((const V*)p->sorted, (T*)p->grid_spread, kp, p->stream));
        else
            SE_CUDA(se::launch_spread_tiled<T>((const V*)p->sorted, p->tile_start, (T*)p->grid_spread,
                                               kp, p->prec == SE_FP32, p->stream));
    }
    timing_mark(p, 2);
    p->spread_clean = false;
    p->have_spread = true;
    p->have_scale = false;
    return SE_OK;
}

template <typename T>
int do_scale(se_plan* p, double* E_grid) {
    SE_CUFFT(cufftSetStream(p->fwd, p->stream));
    SE_CUFFT(cufftSetStream(p->inv, p->stream));
    if (p->prec == SE_FP64)
        SE_CUFFT(cufftExecD2Z(p->fwd, (cufftDoubleReal*)p->grid_spread, (cufftDoubleComplex*)p->cgrid));
    else
        SE_CUFFT(cufftExecR2C(p->fwd, (cufftReal*)p->grid_spread, (cufftComplex*)p->cgrid));
    timing_mark(p, 3);
    const double M3 = (double)p->M * p->M * p->M;
    const double e_scale = p->kc * p->h * p->h * p->h / (2.0 * M3);
    const bool ik = p->force_mode == SE_FORCE_IK;
    if (ik)
        SE_CUDA(se::launch_scale_ik<T>(p->cgrid, p->cgrid_ik, ik_cstride(p), p->green, p->M, p->L,
                                       (T*)p->grid_spread,
                                       p->partials + 3 * se::kMaxPartials, p->tickets + 1, p->acc,
                                       e_scale, E_grid, p->stream));
    else
        SE_CUDA(se::launch_scale<T>(p->cgrid, p->green, p->M, (T*)p->grid_spread, p->partials + 3 * se::kMaxPartials,
                                    p->tickets + 1, p->acc, e_scale, E_grid, p->stream));
    timing_mark(p, 4);
    p->spread_clean = true;
    // Ht, then (ik forces) the three derivative grids, each by the plan's
    // inverse transform from a 256-byte aligned spectrum to an aligned grid
    using C = typename std::conditional<std::is_same<T, float>::value, cufftComplex,
                                        cufftDoubleComplex>::type;
    for (int d = 0; d < (ik ? 4 : 1); ++d) {
        C* src = d == 0 ? (C*)p->cgrid : (C*)p->cgrid_ik + (size_t)(d - 1) * ik_cstride(p);
        T* dst = (T*)p->grid_gather + (size_t)d * ik_gstride(p);
        if (p->prec == SE_FP64)
            SE_CUFFT(cufftExecZ2D(p->inv, (cufftDoubleComplex*)src, (cufftDoubleReal*)dst));
        else
            SE_CUFFT(cufftExecC2R(p->inv, (cufftComplex*)src, (cufftReal*)dst));
    }
    timing_mark(p, 5);
    p->have_scale = true;
    return SE_OK;
}

template <typename T>
int do_gather(se_plan* p, void* phi, void* F, double* E, const double* adj = nullptr) {
    const KParams<T> kp = make_kparams<T>(p);
    using V = se::v4_t<T>;
    // ik forces: potential and force from the four grids with the plain window;
    // no forces asked for: the plain window on Ht alone; else (and for the
    // adjoint, which needs the analytic derivative) the analytic gather
    const int ng = adj ? 0 : (p->force_mode == SE_FORCE_IK && F ? 4 : (F ? 0 : 1));
    if (ng > 0)
        SE_CUDA(se::launch_gather_plain<T>(ng, (const V*)p->sorted, p->perm, (const T*)p->grid_gather,
                                           ik_gstride(p), (T*)phi, (T*)F, kp,
                                           p->partials + 4 * se::kMaxPartials, p->tickets + 2,
                                           p->acc, 0.5, E, false, p->stream));
    else
        SE_CUDA(se::launch_gather<T>((const V*)p->sorted, p->perm, (const T*)p->grid_gather, (T*)phi,
                                     (T*)F, kp, p->partials + 4 * se::kMaxPartials, p->tickets + 2,
                                     p->acc, 0.5, E, adj, p->stream));
    timing_mark(p, 6);
    return SE_OK;
}

// E^L read back from the device results: 1/2 sum q phi from the gather, or in
// the energy-only mode (no gather) the grid energy kc h^3/(2 M^3) sum_k w G |Hhat|^2.
double energy_from_acc(const se_plan* p, const Acc& a, bool energy_only) {
    if (!energy_only) return 0.5 * a.e_gather;
    const double M3 = (double)p->M * p->M * p->M;
    return p->kc * p->h * p->h * p->h / (2.0 * M3) * a.e_grid;
}

int status_from_acc(const Acc& a) {
    if (a.nonfinite) return SE_ERR_NONFINITE;
    if (fabs(a.sum_q) > 1e-10 * a.sum_absq) return SE_WARN_NONNEUTRAL;
    return SE_OK;
}

// Energy only (F and phi both NULL): no gather; E is the grid energy of the
// scaling step, equal to 1/2 sum q phi to rounding (Parseval).
int evaluate(se_plan* p, const void* xyz, const void* q, void* F, void* phi, double* dE) {
    const bool energy_only = !F && !phi;
    if (p->variant >= 3) {
        SE_TRY(fast_spread(p, xyz, q));
        SE_TRY(fast_scale(p, energy_only ? dE : nullptr));
        if (!energy_only) SE_TRY(fast_gather(p, phi, F, dE));
        return SE_OK;
    }
    if (p->prec == SE_FP64) {
        SE_TRY(do_spread<double>(p, xyz, q));
        SE_TRY(do_scale<double>(p, energy_only ? dE : nullptr));
        if (!energy_only) SE_TRY(do_gather<double>(p, phi, F, dE));
    } else {
        SE_TRY(do_spread<float>(p, xyz, q));
        SE_TRY(do_scale<float>(p, energy_only ? dE : nullptr));
        if (!energy_only) SE_TRY(do_gather<float>(p, phi, F, dE));
    }
    return SE_OK;
}

// One evaluation as a replayed CUDA graph: captured on a private stream the
// first time (and whenever an argument pointer or the prefactor changes),
// then launched on the plan's stream.  Returns SE_ERR_UNSUPPORTED when the
// graph cannot be used (the caller then launches directly).
int graph_evaluate(se_plan* p, const void* xyz, const void* q, void* F, void* phi, double* dE) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(p->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
        return SE_ERR_UNSUPPORTED;  // the caller is capturing: launch into its capture
    const void* key[5] = {xyz, q, F, phi, dE};
    bool match = p->gexec && p->gkey_kc == p->kc;
    for (int i = 0; i < 5 && match; ++i) match = key[i] == p->gkey[i];
    if (!match) {
        drop_graph(p);
        if (!p->cap_stream)
            SE_CUDA(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
        if (!p->spread_clean) {
            const size_t M3 = (size_t)p->M * p->M * p->M;
            if (p->variant >= 3)
                SE_CUDA(cudaMemsetAsync(p->g64, 0, M3 * sizeof(long long), p->stream));
            else
                SE_CUDA(cudaMemsetAsync(p->grid_spread, 0, M3 * tsize(p->prec), p->stream));
            p->spread_clean = true;
        }
        // the capture stream must see the state the user stream has reached
        SE_CUDA(cudaStreamSynchronize(p->stream));
        cudaStream_t user = p->stream;
        p->stream = p->cap_stream;
        const bool timing = p->timing;
        p->timing = false;
        cudaGraph_t g = nullptr;
        int rc = check_cuda(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
        if (rc == SE_OK) {
            rc = evaluate(p, xyz, q, F, phi, dE);
            cudaError_t e = cudaStreamEndCapture(p->cap_stream, &g);
            if (rc == SE_OK && e != cudaSuccess) rc = SE_ERR_CUDA;
        }
        p->stream = user;
        p->timing = timing;
        if (rc == SE_OK && cudaGraphInstantiate(&p->gexec, g, 0) != cudaSuccess) {
            p->gexec = nullptr;
            rc = SE_ERR_CUDA;
        }
        if (g) cudaGraphDestroy(g);
        if (rc != SE_OK) {
            cudaGetLastError();
            p->gexec = nullptr;
            return rc;
        }
        for (int i = 0; i < 5; ++i) p->gkey[i] = key[i];
        p->gkey_kc = p->kc;
    }
    SE_CUDA(cudaGraphLaunch(p->gexec, p->stream));
    p->spread_clean = true;
    p->have_spread = p->have_scale = true;
    return SE_OK;
}

// The device address of page-locked host memory that is mapped into the
// device's address space (cudaMallocHost / cudaHostAlloc, or cudaHostRegister
// with cudaHostRegisterMapped), else NULL.  *ok: NULL in, or mapped.
const void* mapped_host(const void* ptr, bool* ok) {
    if (!ptr) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        *ok = false;
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) {
        *ok = false;
        return nullptr;
    }
    return a.devicePointer;
}

// se_energy_force_host as one CUDA graph when every host array is page-locked
// and mapped: the kernels read xyz and q straight from host memory (the first
// kernel, over the host link) and the gather writes F and phi straight into
// it, so the only copy is the reduction record into the plan's pinned
// acc_host.  Captured the first time (and whenever a host pointer or the
// prefactor changes) and replayed; the caller synchronises.
// SE_ERR_UNSUPPORTED when the graph cannot be used (the caller then copies and
// launches directly).
int graph_evaluate_host(se_plan* p, const void* xyz, const void* q, void* F, void* phi) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(p->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
        return SE_ERR_UNSUPPORTED;
    const void* key[4] = {xyz, q, F, phi};
    bool match = p->hexec && p->hkey_kc == p->kc;
    for (int i = 0; i < 4 && match; ++i) match = key[i] == p->hkey[i];
    if (!match) {
        if (p->hexec) cudaGraphExecDestroy(p->hexec);
        p->hexec = nullptr;
        bool ok = true;
        const void* dx = mapped_host(xyz, &ok);
        const void* dq = mapped_host(q, &ok);
        void* dF = const_cast<void*>(mapped_host(F, &ok));
        void* dphi = const_cast<void*>(mapped_host(phi, &ok));
        if (!ok) return SE_ERR_UNSUPPORTED;
        if (!p->acc_host && cudaMallocHost((void**)&p->acc_host, sizeof(Acc)) != cudaSuccess) {
            cudaGetLastError();
            p->acc_host = nullptr;
            return SE_ERR_UNSUPPORTED;
        }
        if (!p->cap_stream)
            SE_CUDA(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
        if (!p->spread_clean) {
            const size_t M3 = (size_t)p->M * p->M * p->M;
            if (p->variant >= 3)
                SE_CUDA(cudaMemsetAsync(p->g64, 0, M3 * sizeof(long long), p->stream));
            else
                SE_CUDA(cudaMemsetAsync(p->grid_spread, 0, M3 * tsize(p->prec), p->stream));
            p->spread_clean = true;
        }
        SE_CUDA(cudaStreamSynchronize(p->stream));
        cudaStream_t user = p->stream;
        p->stream = p->cap_stream;
        const bool timing = p->timing;
        p->timing = false;
        cudaGraph_t g = nullptr;
        int rc = check_cuda(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
        if (rc == SE_OK) {
            rc = evaluate(p, dx, dq, dF, dphi, p->dE);
            if (rc == SE_OK)
                rc = check_cuda(cudaMemcpyAsync(p->acc_host, p->acc, sizeof(Acc), cudaMemcpyDeviceToHost,
                                                p->stream));
            cudaError_t e = cudaStreamEndCapture(p->cap_stream, &g);
            if (rc == SE_OK && e != cudaSuccess) rc = SE_ERR_CUDA;
        }
        p->stream = user;
        p->timing = timing;
        if (rc == SE_OK && cudaGraphInstantiate(&p->hexec, g, 0) != cudaSuccess) {
            p->hexec = nullptr;
            rc = SE_ERR_CUDA;
        }
        if (g) cudaGraphDestroy(g);
        if (rc != SE_OK) {
            cudaGetLastError();
            p->hexec = nullptr;
            return rc;
        }
        for (int i = 0; i < 4; ++i) p->hkey[i] = key[i];
        p->hkey_kc = p->kc;
    }
    SE_CUDA(cudaGraphLaunch(p->hexec, p->stream));
    p->spread_clean = true;
    p->have_spread = p->have_scale = true;
    return SE_OK;
}

// evaluate() through the graph when allowed, else by direct launches.
int run_eval(se_plan* p, const void* xyz, const void* q, void* F, void* phi, double* dE) {
    if (p->use_graph && !p->timing) {
        int rc = graph_evaluate(p, xyz, q, F, phi, dE);
        if (rc == SE_OK) return rc;
        if (rc != SE_ERR_UNSUPPORTED) p->use_graph = false;  // capture failed: stop trying
    }
    return evaluate(p, xyz, q, F, phi, dE);
}

}  // namespace

namespace se {

// FP64 kernel parameters from raw arguments, through a plan on the stack
// (no allocation of any kind).
int make_kparams_f64(int64_t N, double L, double xi, int M, int P, int tile, KParams<double>* out) {
    if (!out || N < 0 || !(L > 0) || !isfinite(L) || !(xi > 0) || !isfinite(xi)) return SE_ERR_ARG;
    se_plan tmp;
    tmp.N = N;
    tmp.L = L;
    tmp.xi = xi;
    tmp.M = M;
    tmp.P = P;
    tmp.prec = SE_FP64;
    tmp.tune_variant = 1;
    tmp.tune_tile = tile;
    derive(&tmp);
    if (!(tmp.eta > 0.0 && tmp.eta < 1.0)) return SE_ERR_ARG;
    *out = make_kparams<double>(&tmp);
    return SE_OK;
}

}  // namespace se

extern "C" {

int se_plan_create(se_plan** out, int64_t N, double L, double xi, int M, int P) {
    if (!out) return SE_ERR_ARG;
    *out = nullptr;
    if (N < 0 || N > 0x7fffffffLL) return SE_ERR_ARG;
    if (!(L > 0) || !isfinite(L) || !(xi > 0) || !isfinite(xi)) return SE_ERR_ARG;
    if (M < 2 || P < 2 || P > M) return SE_ERR_ARG;
    if ((P & 1) || P > se::kMaxP) return SE_ERR_UNSUPPORTED;
    if ((double)M * M * M > 2.0e9) return SE_ERR_ARG;
    se_plan* p = new (std::nothrow) se_plan();
    if (!p) return SE_ERR_NOMEM;
    p->N = N;
    p->L = L;
    p->xi = xi;
    p->M = M;
    p->P = P;
    derive(p);
    if (!(p->eta > 0.0 && p->eta < 1.0)) {
        delete p;
        return SE_ERR_ARG;
    }
    *out = p;
    return SE_OK;
}

int se_plan_destroy(se_plan* p) {
    if (!p) return SE_OK;
    if (p->ev_created) {
        for (int i = 0; i < se_plan::kRing; ++i)
            for (int s = 0; s <= se_plan::kStages; ++s) cudaEventDestroy(p->ev[i][s]);
        p->ev_created = false;
    }
    if (p->cap_stream) {
        drop_graph(p);
        cudaStreamDestroy(p->cap_stream);
        p->cap_stream = nullptr;
    }
    int cur = -1;
    if (p->ready && cudaGetDevice(&cur) == cudaSuccess && cur != p->device) {
        cudaSetDevice(p->device);
        release_device(p);
        cudaSetDevice(cur);
    } else {
        release_device(p);
    }
    delete p;
    return SE_OK;
}

int se_plan_set_precision(se_plan* p, int prec) {
    if (!p || (prec != SE_FP64 && prec != SE_FP32 && prec != SE_FP32_PLAIN)) return SE_ERR_ARG;
    if (prec != p->prec) {
        p->prec = prec;
        invalidate(p);
    }
    return SE_OK;
}

int se_plan_set_shape(se_plan* p, double value, int is_eta) {
    if (!p || !isfinite(value)) return SE_ERR_ARG;
    if (is_eta) {
        if (!(value > 0.0 && value < 1.0)) return SE_ERR_ARG;
        p->eta_fixed = 1;
        p->eta_user = value;
    } else {
        if (!(value > 0.0)) return SE_ERR_ARG;
        double m = value * sqrt(kPi * p->P);
        double eta = (2.0 * p->w * p->xi / m) * (2.0 * p->w * p->xi / m);
        if (!(eta > 0.0 && eta < 1.0)) return SE_ERR_ARG;
        p->eta_fixed = 0;
        p->c_shape = value;
    }
    invalidate(p);
    return SE_OK;
}

int se_plan_set_prefactor(se_plan* p, double kc) {
    if (!p || !isfinite(kc)) return SE_ERR_ARG;
    p->kc = kc;  // only the kernel parameters change
    return SE_OK;
}

int se_plan_set_stream(se_plan* p, void* stream) {
    if (!p) return SE_ERR_ARG;
    p->stream = (cudaStream_t)stream;
    return SE_OK;
}

int se_plan_set_tuning(se_plan* p, int spread_variant, int tile) {
    if (!p || spread_variant < 0 || spread_variant > 5 || (tile != 0 && (tile < 2 || tile > 32)))
        return SE_ERR_ARG;
    if (spread_variant >= 3 && (p->prec == SE_FP64 || p->M > se::kFastMaxM)) return SE_ERR_UNSUPPORTED;
    if (spread_variant == 2 && p->prec == SE_FP32) return SE_ERR_UNSUPPORTED;
    if (spread_variant == 5 && !se::fast_slab_gather_ok(p->M)) return SE_ERR_UNSUPPORTED;
    p->tune_variant = spread_variant;
    p->tune_tile = tile;
    invalidate(p);
    return SE_OK;
}

int se_plan_set_force_mode(se_plan* p, int mode) {
    if (!p || (mode != SE_FORCE_ANALYTIC && mode != SE_FORCE_IK)) return SE_ERR_ARG;
    if (mode == p->force_mode) return SE_OK;
    p->force_mode = mode;
    invalidate(p);
    return SE_OK;
}

int se_plan_get_params(const se_plan* p, double* out) {
    if (!p || !out) return SE_ERR_ARG;
    out[0] = p->h;
    out[1] = p->w;
    out[2] = p->eta;
    out[3] = p->alpha;
    out[4] = p->cg;
    out[5] = p->m;
    out[6] = p->tile;
    out[7] = p->variant;
    out[8] = p->prec;
    out[9] = p->kc;
    return SE_OK;
}

int se_spread(se_plan* p, const void* xyz, const void* q) {
    if (!p || (p->N > 0 && (!xyz || !q))) return SE_ERR_ARG;
    SE_TRY(prepare(p));
    if (p->variant >= 3) return fast_spread(p, xyz, q);
    return p->prec == SE_FP64 ? do_spread<double>(p, xyz, q) : do_spread<float>(p, xyz, q);
}

int se_scale(se_plan* p, double* E_grid) {
    if (!p) return SE_ERR_ARG;
    if (!p->ready || !p->have_spread) return SE_ERR_ARG;
    if (p->variant >= 3) return fast_scale(p, E_grid);
    return p->prec == SE_FP64 ? do_scale<double>(p, E_grid) : do_scale<float>(p, E_grid);
}

int se_gather(se_plan* p, const void* xyz, const void* q, void* phi, void* F, double* E) {
    if (!p || (p->N > 0 && (!xyz || !q))) return SE_ERR_ARG;
    if (!p->ready || !p->have_scale) return SE_ERR_ARG;
    if (p->variant >= 3) return fast_gather(p, phi, F, E);
    return p->prec == SE_FP64 ? do_gather<double>(p, phi, F, E) : do_gather<float>(p, phi, F, E);
}

int se_adjoint(se_plan* p, const void* xyz, const void* q, const double* gE, void* grad_x,
               void* grad_q) {
    if (!p || !gE || (p->N > 0 && (!xyz || !q))) return SE_ERR_ARG;
    if (!p->ready || !p->have_scale) return SE_ERR_ARG;
    if (p->variant >= 3) return fast_gather(p, grad_q, grad_x, nullptr, gE);
    return p->prec == SE_FP64 ? do_gather<double>(p, grad_q, grad_x, nullptr, gE)
                              : do_gather<float>(p, grad_q, grad_x, nullptr, gE);
}

int se_energy_force(se_plan* p, const void* xyz, const void* q, double* E, void* F, void* phi) {
    if (!p || (p->N > 0 && (!xyz || !q))) return SE_ERR_ARG;
    SE_TRY(prepare(p));
    SE_TRY(run_eval(p, xyz, q, F, phi, p->dE));
    if (E) {
        Acc a;
        SE_CUDA(cudaMemcpyAsync(&a, p->acc, sizeof(Acc), cudaMemcpyDeviceToHost, p->stream));
        SE_CUDA(cudaStreamSynchronize(p->stream));
        *E = energy_from_acc(p, a, !F && !phi);
        return status_from_acc(a);
    }
    return SE_OK;
}

int se_energy_force_host(se_plan* p, const void* xyz, const void* q, double* E, void* F, void* phi) {
    if (!p || (p->N > 0 && (!xyz || !q))) return SE_ERR_ARG;
    SE_TRY(prepare(p));
    const size_t ts = tsize(p->prec), N = (size_t)p->N;
    if (!p->h_xyz) {
        int rc = SE_OK;
        if (rc == SE_OK) rc = dalloc(&p->h_xyz, 3 * N * ts);
        if (rc == SE_OK) rc = dalloc(&p->h_q, N * ts);
        if (rc == SE_OK) rc = dalloc(&p->h_F, 3 * N * ts);
        if (rc == SE_OK) rc = dalloc(&p->h_phi, N * ts);
        if (rc != SE_OK) return rc;
    }
    // page-locked, mapped host buffers: the evaluation reads and writes them
    // directly, as one replayed graph
    if (N > 0 && p->use_graph && !p->timing) {
        const int rc = graph_evaluate_host(p, xyz, q, F, phi);
        if (rc == SE_OK) {
            SE_CUDA(cudaStreamSynchronize(p->stream));
            const Acc a = *p->acc_host;
            if (E) *E = energy_from_acc(p, a, !F && !phi);
            return status_from_acc(a);
        }
        if (rc != SE_ERR_UNSUPPORTED) p->use_graph = false;   // capture failed: stop trying
    }
    if (N > 0) {
        SE_CUDA(cudaMemcpyAsync(p->h_xyz, xyz, 3 * N * ts, cudaMemcpyHostToDevice, p->stream));
        SE_CUDA(cudaMemcpyAsync(p->h_q, q, N * ts, cudaMemcpyHostToDevice, p->stream));
    }
    SE_TRY(run_eval(p, p->h_xyz, p->h_q, F ? p->h_F : nullptr, phi ? p->h_phi : nullptr, p->dE));
    if (N > 0 && F) SE_CUDA(cudaMemcpyAsync(F, p->h_F, 3 * N * ts, cudaMemcpyDeviceToHost, p->stream));
    if (N > 0 && phi) SE_CUDA(cudaMemcpyAsync(phi, p->h_phi, N * ts, cudaMemcpyDeviceToHost, p->stream));
    Acc a;
    SE_CUDA(cudaMemcpyAsync(&a, p->acc, sizeof(Acc), cudaMemcpyDeviceToHost, p->stream));
    SE_CUDA(cudaStreamSynchronize(p->stream));
    if (E) *E = energy_from_acc(p, a, !F && !phi);
    return status_from_acc(a);
}

int se_evaluate(se_plan* p, const void* xyz, const void* q, void* F, void* phi, double* E) {
    if (!p || (p->N > 0 && (!xyz || !q))) return SE_ERR_ARG;
    SE_TRY(prepare(p));
    return run_eval(p, xyz, q, F, phi, E);
}

int se_plan_set_graph(se_plan* p, int enable) {
    if (!p) return SE_ERR_ARG;
    p->use_graph = enable != 0;
    if (!p->use_graph) drop_graph(p);
    return SE_OK;
}

int se_plan_get_status(se_plan* p, int* status) {
    if (!p || !status) return SE_ERR_ARG;
    if (!p->ready) {
        *status = SE_OK;
        return SE_OK;
    }
    Acc a;
    SE_CUDA(cudaMemcpyAsync(&a, p->acc, sizeof(Acc), cudaMemcpyDeviceToHost, p->stream));
    SE_CUDA(cudaStreamSynchronize(p->stream));
    *status = status_from_acc(a);
    return SE_OK;
}

int se_copy_grid(se_plan* p, int which, void* dst) {
    if (!p || !dst || (which != 0 && which != 1)) return SE_ERR_ARG;
    if (!p->ready) return SE_ERR_ARG;
    const size_t bytes = (size_t)p->M * p->M * p->M * tsize(p->prec);
    // the single-precision pipelines clear the spread grid in the transform:
    // it is there only between se_spread and se_scale
    if (which == 0 && p->variant >= 3 && p->spread_clean) return SE_ERR_ARG;
    if (which == 0 && (p->variant == 3 || p->variant == 5))
        return check_cuda(se::fast_to_real(fast_bufs(p), p->M, (float*)dst, p->stream));
    if (which == 1 && p->variant == 5) {
        // variant 5 keeps the real grid on chip: transform it back on request
        if (!p->have_scale) return SE_ERR_ARG;
        SE_CUDA(se::fast_inverse(make_kparams<float>(p), fast_bufs(p), 0.0, nullptr, p->stream));
    }
    if (which == 0 && p->variant == 4) {
        SE_CUDA(cudaMemcpyAsync(dst, p->g64, bytes, cudaMemcpyDeviceToDevice, p->stream));
        return SE_OK;
    }
    SE_CUDA(cudaMemcpyAsync(dst, which == 0 ? p->grid_spread : p->grid_gather, bytes,
                            cudaMemcpyDeviceToDevice, p->stream));
    return SE_OK;
}

int se_self_energy(const se_plan* p, const double* q_host, int64_t n, double* E_self) {
    if (!p || !E_self || n < 0 || (n > 0 && !q_host)) return SE_ERR_ARG;
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += q_host[i] * q_host[i];
    *E_self = -p->kc * p->xi / sqrt(kPi) * s;
    return SE_OK;
}

const char* se_strerror(int status) {
    switch (status) {
        case SE_OK: return "success";
        case SE_WARN_NONNEUTRAL: return "warning: the system is not charge neutral";
        case SE_ERR_ARG: return "invalid argument";
        case SE_ERR_CUDA: return "CUDA error";
        case SE_ERR_NOMEM: return "out of memory";
        case SE_ERR_UNSUPPORTED: return "unsupported parameter (odd P or P > 32)";
        case SE_ERR_CUFFT: return "cuFFT error";
        case SE_ERR_NONFINITE: return "non-finite position or charge";
        default: return "unknown status";
    }
}

int se_plan_set_timing(se_plan* p, int enable) {
    if (!p) return SE_ERR_ARG;
    if (enable && !p->ev_created) {
        for (int i = 0; i < se_plan::kRing; ++i)
            for (int s = 0; s <= se_plan::kStages; ++s)
                SE_CUDA(cudaEventCreate(&p->ev[i][s]));
        p->ev_created = true;
    }
    p->timing = enable != 0;
    return SE_OK;
}

int se_plan_get_timing(se_plan* p, double* ms, int nstages, int64_t* count, int reset) {
    if (!p || !ms || nstages < se_plan::kStages) return SE_ERR_ARG;
    if (p->ev_created)
        for (int i = 0; i < se_plan::kRing; ++i) fold_set(p, i);
    for (int s = 0; s < se_plan::kStages; ++s) ms[s] = p->stage_ms[s];
    if (count) *count = p->stage_count;
    if (reset) {
        for (int s = 0; s < se_plan::kStages; ++s) p->stage_ms[s] = 0.0;
        p->stage_count = 0;
    }
    return SE_OK;
}

int se_version(void) { return 100; }

}  // extern "C"
