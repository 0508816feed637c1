// se_probe.cu -- throughput probes for the roofline denominators of the
// benchmark: the FP32 and FP64 FMA rate and the shared-memory atomic add rate
// of the current GPU, each from a short timed kernel (bounded loops, no
// waits).  The spread, gather and transform kernels are bound by these units
// rather than by HBM; copy bandwidth and tensor throughput come from the
// measured peaks file instead.  The paper has no counterpart.
#include <cuda_runtime.h>

#include "../../include/se.h"

namespace {

constexpr int kThreads = 256;
constexpr int kFmaIters = 2048;      // per thread, 8 independent chains each
constexpr int kAtomIters = 2048;     // shared atomics per thread
constexpr int kAtomWords = 4096;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_probe_fma(T* out, T a) {
    T x0 = (T)threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
    T x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    for (int i = 0; i < kFmaIters; ++i) {
        x0 = x0 * a + (T)1;
        x1 = x1 * a + (T)1;
        x2 = x2 * a + (T)1;
        x3 = x3 * a + (T)1;
        x4 = x4 * a + (T)1;
        x5 = x5 * a + (T)1;
        x6 = x6 * a + (T)1;
        x7 = x7 * a + (T)1;
    }
    const T s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
    if (s == (T)-1) out[blockIdx.x] = s;   // keeps the chains alive
}

// Non-returning shared-memory atomic adds: in every step the 32 lanes of a
// warp hit 32 consecutive words (no bank conflict), the warps of a block
// different words.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_probe_smem_atomic(T* out) {
    __shared__ T s[kAtomWords];
    for (int i = threadIdx.x; i < kAtomWords; i += blockDim.x) s[i] = (T)0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int base = warp * 32 * 5;
    for (int i = 0; i < kAtomIters; ++i) {
        atomicAdd(&s[(base + lane) & (kAtomWords - 1)], (T)1);
        base += 32 * 3;
    }
    __syncthreads();
    if (threadIdx.x == 0 && s[7] == (T)-1) out[blockIdx.x] = s[7];
}

template <typename K, typename... A>
int time_kernel(K kern, int grid, cudaStream_t st, double* ms, A... args) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return SE_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return SE_ERR_CUDA;
    }
    int rc = SE_OK;
    kern<<<grid, kThreads, 0, st>>>(args...);   // warm-up
    cudaEventRecord(e0, st);
    for (int r = 0; r < 5; ++r) kern<<<grid, kThreads, 0, st>>>(args...);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) rc = SE_ERR_CUDA;
    float t = 0.f;
    if (rc == SE_OK && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) rc = SE_ERR_CUDA;
    *ms = t / 5.0;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

}  // namespace

extern "C" int se_probe_peak(int kind, double* out) {
    if (!out || kind < 0 || kind > 3) return SE_ERR_ARG;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SE_ERR_CUDA;
    const int grid = nsm * 8;   // 2048 threads per SM
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return SE_ERR_CUDA;
    void* buf = nullptr;
    int rc = cudaMalloc(&buf, (size_t)grid * sizeof(double)) == cudaSuccess ? SE_OK : SE_ERR_NOMEM;
    double ms = 0.0, work = 0.0;
    const double threads = (double)grid * kThreads;
    if (rc == SE_OK) {
        switch (kind) {
            case SE_PROBE_FP32_FMA:
                rc = time_kernel(k_probe_fma<float>, grid, st, &ms, (float*)buf, 0.999f);
                work = threads * kFmaIters * 8 * 2;
                break;
            case SE_PROBE_FP64_FMA:
                rc = time_kernel(k_probe_fma<double>, grid, st, &ms, (double*)buf, 0.999);
                work = threads * kFmaIters * 8 * 2;
                break;
            case SE_PROBE_SMEM_ATOMIC_U32:
                rc = time_kernel(k_probe_smem_atomic<unsigned>, grid, st, &ms, (unsigned*)buf);
                work = threads * kAtomIters;
                break;
            default:
                rc = time_kernel(k_probe_smem_atomic<float>, grid, st, &ms, (float*)buf);
                work = threads * kAtomIters;
                break;
        }
    }
    if (buf) cudaFree(buf);
    cudaStreamDestroy(st);
    if (rc != SE_OK) return rc;
    if (!(ms > 0.0)) return SE_ERR_CUDA;
    *out = work / (ms * 1e-3);
    return SE_OK;
}
