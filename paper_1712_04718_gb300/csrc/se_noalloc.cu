// se_noalloc.cu -- se_spread_noalloc: the spreading step of se_spread for
// callers that cannot allocate device memory (no counterpart in the paper).
//
// Some callers can't call cudaMalloc: a host program that reserves all of its
// device memory at start-up and forbids allocation inside its time-step loop,
// or a library that lives inside a framework whose own caching allocator owns
// the device and must not see raw cudaMalloc/cudaFree.  For them this entry
// point spreads onto a grid they own, with every intermediate buffer (tile
// counts and offsets, per-particle slots, the tile-sorted particle copy, the
// reduction partials) inside one file-scope device array of fixed size.
//
// That array is reserved on every GPU that loads the library, for the life
// of the process: kScratchBytes (about 1.5 MB).  All calls on a device share
// it, so two calls that overlap on the GPU (different streams, or different
// host threads) race and corrupt each other's results: issue them on one
// stream, one after another.  The array's device address is looked up once
// per device and kept: after a cudaDeviceReset it is stale, and this entry
// point must not be called on that device again.  Non-finite inputs are not
// reported (no status is read back).
#include <mutex>

#include "../../include/se.h"
#include "se_internal.h"

namespace {

constexpr int64_t kNoAllocMaxN = 32768;   // particles
constexpr int kNoAllocTile = 8;           // spreading tile edge (cells)
constexpr int kNoAllocMaxTiles = 4096;    // (M/8)^3 tiles: M <= 128
constexpr int kMaxDevices = 64;

constexpr size_t up256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t kOffCount = 0;
constexpr size_t kOffStart = up256(kOffCount + sizeof(int) * kNoAllocMaxTiles);
constexpr size_t kOffSlot = up256(kOffStart + sizeof(int) * (kNoAllocMaxTiles + 1));
constexpr size_t kOffTileOf = up256(kOffSlot + sizeof(int) * kNoAllocMaxN);
constexpr size_t kOffPerm = up256(kOffTileOf + sizeof(int) * kNoAllocMaxN);
constexpr size_t kOffSorted = up256(kOffPerm + sizeof(int) * kNoAllocMaxN);
constexpr size_t kOffPartials = up256(kOffSorted + sizeof(se::d4) * kNoAllocMaxN);
constexpr size_t kOffTickets = up256(kOffPartials + sizeof(double) * 3 * se::kMaxPartials);
constexpr size_t kOffAcc = up256(kOffTickets + sizeof(unsigned) * 4);
constexpr size_t kScratchBytes = up256(kOffAcc + sizeof(se::Acc));

std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {};

}  // namespace

// The scratch itself.  In host code this name is only a host-side stand-in
// for the device symbol: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of the scratch on the current device (looked up once per
// device, with that device current).
static int scratch_address(int dev, unsigned char** out) {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return SE_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
    return SE_OK;
}

extern "C" int se_spread_noalloc(const double* xyz, const double* q, int64_t N, double L,
                                 double xi, int M, int P, double* H, void* stream) {
    if (!H || N < 0 || (N > 0 && (!xyz || !q))) return SE_ERR_ARG;
    if (N > kNoAllocMaxN || M < 2 || M > 128) return SE_ERR_ARG;   // beyond the static scratch
    if (P < 2 || P > M) return SE_ERR_ARG;
    if ((P & 1) || P > se::kMaxP) return SE_ERR_UNSUPPORTED;
    se::KParams<double> kp;
    if (se::make_kparams_f64(N, L, xi, M, P, kNoAllocTile, &kp) != SE_OK) return SE_ERR_ARG;
    if (kp.ntiles > kNoAllocMaxTiles) return SE_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SE_ERR_CUDA;
    unsigned char* base = nullptr;
    if (scratch_address(dev, &base) != SE_OK) return SE_ERR_CUDA;
    int* tile_count = reinterpret_cast<int*>(base + kOffCount);
    int* tile_start = reinterpret_cast<int*>(base + kOffStart);
    int* slot = reinterpret_cast<int*>(base + kOffSlot);
    int* tile_of = reinterpret_cast<int*>(base + kOffTileOf);
    int* perm = reinterpret_cast<int*>(base + kOffPerm);
    se::d4* sorted = reinterpret_cast<se::d4*>(base + kOffSorted);
    double* partials = reinterpret_cast<double*>(base + kOffPartials);
    unsigned* tickets = reinterpret_cast<unsigned*>(base + kOffTickets);
    se::Acc* acc = reinterpret_cast<se::Acc*>(base + kOffAcc);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t M3 = (size_t)M * M * M;
    // what must start at zero: the tile counters, the block ticket, the output grid
    if (cudaMemsetAsync(tile_count, 0, sizeof(int) * kp.ntiles, s) != cudaSuccess ||
        cudaMemsetAsync(tickets, 0, sizeof(unsigned) * 4, s) != cudaSuccess ||
        cudaMemsetAsync(H, 0, sizeof(double) * M3, s) != cudaSuccess)
        return SE_ERR_CUDA;
    if (se::launch_bin<double>(xyz, q, kp, tile_count, slot, tile_of, tile_start, partials,
                               tickets, acc, s) != cudaSuccess)
        return SE_ERR_CUDA;
    if (se::launch_scatter<double>(xyz, q, kp, slot, tile_of, tile_start, sorted, perm, s) !=
        cudaSuccess)
        return SE_ERR_CUDA;
    if (N > 0 && se::launch_spread_tiled<double>(sorted, tile_start, H, kp, false, s) != cudaSuccess)
        return SE_ERR_CUDA;
    return SE_OK;
}
