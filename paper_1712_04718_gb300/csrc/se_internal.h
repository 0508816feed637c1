// se_internal.h -- types shared by the libse host code and its kernels.
// Not part of the public ABI (see include/se.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace se {

constexpr int kMaxP = 32;

// A particle as (x, y, z, q), one 16- or 32-byte load.
struct __align__(16) f4 { float x, y, z, w; };
struct __align__(32) d4 { double x, y, z, w; };
template <typename T> struct V4;
template <> struct V4<float> { using type = f4; };
template <> struct V4<double> { using type = d4; };
template <typename T> using v4_t = typename V4<T>::type;

// Per-evaluation constants passed by value to every kernel.
template <typename T>
struct KParams {
    int N;          // particles
    int M;          // grid points per dimension
    int P;          // support points per dimension (even)
    int tile;       // edge of a spreading tile, in grid cells
    int nT;         // tiles per dimension = ceil(M / tile)
    int ntiles;     // nT^3
    T L, invL;      // box and its rounded reciprocal (wrap)
    T h, invh;      // grid spacing and M / L rounded (cell index)
    T beta;         // alpha h^2, the Gaussian exponent in grid units (alpha = 2 xi^2 / eta)
    T qcg;          // c_g, folded into the spread weights
    T phi_scale;    // kc h^3 c_g
    T F_scale;      // -kc 2 alpha h^4 c_g (offsets are in grid units)
    T E3[kMaxP];    // exp(-beta (a - (P-1)/2)^2), a = 0..P-1 (fast Gaussian gridding)
};

// Device-side results of the reducing kernels; each field is overwritten by
// the last block of the kernel that produces it.
struct Acc {
    double sum_q;        // sum of charges (bin)
    double sum_absq;     // sum of |q| (bin)
    double e_grid;       // sum_k w_k G |H^_k|^2 over the half spectrum (scale)
    double e_gather;     // sum_m q_m phi_m, phi including the prefactor (gather)
    unsigned int nonfinite;  // number of particles with NaN/Inf position or charge (bin)
    int fx_shift;            // fixed-point spread: weights scaled by 2^fx_shift
    float fx_scale, fx_inv;  // 2^fx_shift and 2^-fx_shift
    double pad;
};

// launchers (se_kernels_*.cu)
template <typename T>
cudaError_t launch_bin(const T* xyz, const T* q, const KParams<T>& kp, int* tile_count,
                       int* slot, int* tile_of, int* tile_start, double* partials,
                       unsigned* ticket, Acc* acc, cudaStream_t s);
template <typename T>
cudaError_t launch_scatter(const T* xyz, const T* q, const KParams<T>& kp, const int* slot,
                           const int* tile_of, const int* tile_start, v4_t<T>* sorted,
                           int* perm, cudaStream_t s);
template <typename T>
cudaError_t launch_spread_tiled(const v4_t<T>* sorted, const int* tile_start, T* grid,
                                const KParams<T>& kp, bool comp, cudaStream_t s);
template <typename T>
cudaError_t launch_spread_direct(const v4_t<T>* sorted, T* grid, const KParams<T>& kp,
                                 cudaStream_t s);
template <typename T>
cudaError_t launch_scale(void* cgrid, const double* green, int M, T* zero_grid,
                         double* partials, unsigned* ticket, Acc* acc, double e_scale,
                         double* E_out, cudaStream_t s);
template <typename T>
cudaError_t launch_gather(const v4_t<T>* sorted, const int* perm, const T* grid, T* phi,
                          T* F, const KParams<T>& kp, double* partials, unsigned* ticket,
                          Acc* acc, double e_scale, double* E_out, const double* adj,
                          cudaStream_t s);

// ik differentiation (se_plain.cuh): scale as launch_scale, and in addition
// D_d = i k_d G/M^3 Hhat into dgrid (d = x, y, z; each an M x M x (M/2+1)
// complex half spectrum, dstride >= M^2 (M/2+1) complex values apart).
template <typename T>
cudaError_t launch_scale_ik(void* cgrid, void* dgrid, size_t dstride, const double* green, int M,
                            double L, T* zero_grid, double* partials, unsigned* ticket, Acc* acc,
                            double e_scale, double* E_out, cudaStream_t s);
// Gather with the underived window from ng grids gstride values apart:
// ng = 1 potential (and energy) only; ng = 4 potential and ik forces from
// [Ht, dHt/dx, dHt/dy, dHt/dz].  pdl: launched as a programmatic dependent.
template <typename T>
cudaError_t launch_gather_plain(int ng, const v4_t<T>* sorted, const int* perm, const T* grid,
                                size_t gstride, T* phi, T* F, const KParams<T>& kp,
                                double* partials, unsigned* ticket, Acc* acc, double e_scale,
                                double* E_out, bool pdl, cudaStream_t s);

// Kernel parameters for an FP64 evaluation without a plan (se_plan.cu).
int make_kparams_f64(int64_t N, double L, double xi, int M, int P, int tile, KParams<double>* out);

// single-precision pipeline without cuFFT (se_fast.cuh)
struct FastBufs {
    long long* g64;       // M^3 fixed-point spread grid (the float grid when unsorted)
    void* cgrid;          // M x M x (M/2+1) float2
    float* rgrid;         // M^3 real grid after the inverse transform
    const void* tw;       // M twiddles (cos, sin)(2 pi r / M), float2
    const double* green;  // G(k) on the half spectrum
    const float* green_f; // the same table rounded to float
    int* tile_count;
    void* bucket;         // f4 [ntiles * cap]: particles by tile
    int* bucket_idx;      // [ntiles * cap]: their input positions
    int* tile_n;          // [ntiles + 1]: particles in each bucket, then the overflow count
    int cap;              // bucket capacity
    int* over_idx;        // [N] particles that found their bucket full
    void* wrapped;        // f4 [N]: wrapped (x, y, z, q) in input order, for the gather
    double* partials;     // bin: [0, 3*1024), its max |q| per block as words at [3*1024, ...);
                          // gather: [4*1024, 5*1024); x pass: [5*1024, 7*1024)
    unsigned* tickets;    // [0] unsorted spread, [1] x pass, [2] gather, [3] overflow
                          // CTAs, [4] overflow count
    Acc* acc;
    bool unsorted;        // spread unsorted into a float grid (k_fdirect)
    void* part;           // variant 5: float4 [P][N], each particle's share of each x-plane
};
cudaError_t fast_spread(const float* xyz, const float* q, const KParams<float>& kp,
                        const FastBufs& b, cudaStream_t s, bool marks, void (*mark)(void*, int),
                        void* ctx);
bool fast_gather_tiled(const KParams<float>& kp);
cudaError_t fast_gather(const KParams<float>& kp, const FastBufs& b, float* phi, float* F,
                        double* partials, unsigned* ticket, double e_scale, double* E_out,
                        const double* adj, cudaStream_t s);
// forward transform, x pass (scaling, grid energy partials) and, with
// inverse, the inverse transform into b.rgrid (variant 5 fuses the inverse
// with its gather instead)
cudaError_t fast_transform(const KParams<float>& kp, const FastBufs& b, double e_scale,
                           double* E_grid, cudaStream_t s, bool marks, void (*mark)(void*, int),
                           void* ctx, bool inverse = true);
// the inverse transform alone (the real grid of variant 5 on request)
cudaError_t fast_inverse(const KParams<float>& kp, const FastBufs& b, double e_scale,
                         double* E_grid, cudaStream_t s);
// variant 5: the grid energy from the x pass's partials (energy only), and
// the inverse transform fused with the gather, then the sum of the shares
cudaError_t fast_grid_energy(const KParams<float>& kp, const FastBufs& b, double e_scale,
                             double* E_out, cudaStream_t s);
// whether variant 5's shared memory (the inverse transform's regions and
// the real plane) fits one CTA on the current device for this M
bool fast_slab_gather_ok(int M);
cudaError_t fast_gather_slab(const KParams<float>& kp, const FastBufs& b, float* phi, float* F,
                             double* partials, unsigned* ticket, double e_scale, double* E_out,
                             const double* adj, cudaStream_t s);
cudaError_t fast_to_real(const FastBufs& b, int M, float* dst, cudaStream_t s);
cudaError_t launch_gather_pdl(const f4* sorted, const int* perm, const float* grid, float* phi,
                              float* F, const KParams<float>& kp, double* partials,
                              unsigned* ticket, Acc* acc, double e_scale, double* E_out,
                              const double* adj, cudaStream_t s);

constexpr int kMaxPartials = 1024;   // blocks of the reducing kernels

// Lanes per particle: a particle's P z-points are split over G = P / D lanes
// (D points each); D is the smallest divisor of P that keeps >= 85% of the
// warp's lanes busy.
__host__ __device__ constexpr int pick_d(int P) {
    for (int d = 1; d <= P; ++d) {
        if (P % d) continue;
        int g = P / d;
        if (g > 32) continue;
        if (g * (32 / g) * 100 >= 85 * 32) return d;
    }
    return P;
}
constexpr int kFastMaxM = 128;       // largest grid of the single-precision pipeline
constexpr int kScanLimit = 8192;     // tiles scanned in shared memory
constexpr size_t kSmemBudget = 200 * 1024;  // dynamic shared memory for a spreading tile
constexpr size_t kSlabSmemFloor = 116 * 1024;  // > half of an SM's 228 KB: one slab CTA per SM
constexpr size_t kTileGatherSmem = 64 * 1024;  // largest tile region staged by the tile gather

}  // namespace se
