// Measurement probe: sustained rate of fire-and-forget 64-bit integer
// reductions (red.global.add.u64) served by the L2, the operation the
// contribution kernel issues once per in-window sample. The rate is the
// denominator of that kernel's atomic roofline; no vendor figure exists for it.
//
// Every thread of a GPU-filling grid issues `per_thread` reductions into a
// 64 MiB buffer (L2-resident), with one of two address patterns:
//   0: each warp's 32 lanes hit 32 consecutive words (256 B, two 128 B lines),
//      the warp moving to another line group each iteration;
//   1: every lane a pseudo-random word (an integer hash of thread and
//      iteration), as scattered as possible.
// The kernel is timed with CUDA events after a warm-up launch.
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/tsdf.h"

namespace {

constexpr size_t kWords = (64u << 20) / 8;   // 64 MiB of uint64

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    // integer finaliser (xor-shift-multiply), only used to spread addresses
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

__global__ void __launch_bounds__(256) red_probe_kernel(unsigned long long* buf, int pattern, int per_thread) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t warp = tid >> 5, lane = tid & 31u;
    const uint32_t mask = (uint32_t)kWords - 1u;
    for (int i = 0; i < per_thread; ++i) {
        uint32_t w;
        if (pattern == 0) w = ((mix32(warp * 1024u + (uint32_t)i) << 5) | lane) & mask;
        else w = mix32(tid * 4096u + (uint32_t)i) & mask;
        atomicAdd(buf + w, 1ull);   // result unused: compiled to a reduction
    }
}

}  // namespace

extern "C" int tsdf_probe_reduction_rate(int32_t pattern, double* per_second, void* stream) {
    if ((pattern != 0 && pattern != 1) || !per_second) return TSDF_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    unsigned long long* buf = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&buf, kWords * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, kWords * sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    const int grid = sms * 8, per_thread = 256;
    float ms = 0.f;
    if (e == cudaSuccess) {
        red_probe_kernel<<<grid, 256, 0, s>>>(buf, pattern, per_thread);   // warm-up
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(t0, s);
    if (e == cudaSuccess) {
        red_probe_kernel<<<grid, 256, 0, s>>>(buf, pattern, per_thread);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(t1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (buf) cudaFree(buf);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? TSDF_ERR_OOM : TSDF_ERR_CUDA;
    *per_second = (double)grid * 256.0 * per_thread / ((double)ms * 1e-3);
    return TSDF_OK;
}
