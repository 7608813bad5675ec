// Peak probes of the current GPU for the roofline figures the benchmark reports beside each kernel
// (no counterpart in the paper): the FP32 FMA rate of a register-only loop, and the bandwidth of a
// streaming read from HBM over a buffer larger than L2.  Neither touches a context.
#include "fdirw_internal.h"

#include "fdirw.h"

#include <string>

namespace fdirw {
namespace {

constexpr int kChains = 16;              // independent FMA chains per thread

__global__ void __launch_bounds__(512) fma_probe_kernel(float a, float b, int iters, float* sink) {
    float x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; i++) x[i] = 1e-3f * (float)threadIdx.x + (float)i;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int i = 0; i < kChains; i++) x[i] = fmaf(x[i], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; i++) s += x[i];
    if (s == -1.0f) sink[0] = s;         // never true for these inputs; keeps the loop
}

__global__ void __launch_bounds__(512) read_probe_kernel(const uint4* __restrict__ p, int64_t n16, unsigned* sink) {
    unsigned acc = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n16; i += 4 * stride) {      // four independent 16-byte loads in flight
        const uint4 v0 = __ldcs(p + i), v1 = __ldcs(p + i + stride);
        const uint4 v2 = __ldcs(p + i + 2 * stride), v3 = __ldcs(p + i + 3 * stride);
        acc ^= v0.x ^ v0.y ^ v0.z ^ v0.w ^ v1.x ^ v1.y ^ v1.z ^ v1.w ^ v2.x ^ v2.y ^ v2.z ^ v2.w ^ v3.x ^ v3.y ^ v3.z ^ v3.w;
    }
    for (; i < n16; i += stride) {
        const uint4 v = __ldcs(p + i);
        acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
    if (acc == 0x9E3779B9u) sink[0] = acc;   // the buffer is zero, so never true; keeps the loads
}

}  // namespace
}  // namespace fdirw

extern "C" FDIRW_API int fdirw_probe_peaks(int32_t device, double* fp32_flops, double* read_bytes_per_s) {
    using namespace fdirw;
    int prev = 0;
    cudaGetDevice(&prev);
    if (device >= 0 && cudaSetDevice(device) != cudaSuccess)
        return set_thread_error(FDIRW_ERR_CUDA, "fdirw_probe_peaks: cannot select the device");
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t bytes = (size_t)4 << 30;
    void* buf = nullptr;
    float* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    std::string err;
    cudaError_t e = cudaMalloc(&buf, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&sink, 16);
    if (e == cudaSuccess) e = cudaMemset(buf, 0, bytes);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best_fma = 1e30f, best_read = 1e30f;
    const int iters = 1 << 15, fma_grid = sms * 4;
    for (int rep = 0; rep < 4 && e == cudaSuccess; rep++) {
        float ms = 0.f;
        cudaEventRecord(e0);
        fma_probe_kernel<<<fma_grid, 512>>>(0.9999999f, 1e-7f, iters, sink);
        cudaEventRecord(e1);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && ms < best_fma) best_fma = ms;     // the first run warms up
        cudaEventRecord(e0);
        read_probe_kernel<<<sms * 4, 512>>>(reinterpret_cast<const uint4*>(buf), (int64_t)(bytes / 16),
                                            reinterpret_cast<unsigned*>(sink));
        cudaEventRecord(e1);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && ms < best_read) best_read = ms;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(buf);
    cudaFree(sink);
    if (device >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess)
        return set_thread_error(e == cudaErrorMemoryAllocation ? FDIRW_ERR_NOMEM : FDIRW_ERR_CUDA,
                                std::string("fdirw_probe_peaks: ") + cudaGetErrorString(e));
    if (fp32_flops) *fp32_flops = 2.0 * kChains * (double)iters * fma_grid * 512 / (best_fma * 1e-3);
    if (read_bytes_per_s) *read_bytes_per_s = (double)bytes / (best_read * 1e-3);
    return FDIRW_OK;
}
