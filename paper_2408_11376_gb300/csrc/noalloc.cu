// fdirw_mass_noalloc: the FP64 mass budget of a device field, computed without allocating any memory.
//
// Who needs it: code that may not call cudaMalloc at the moment it wants the budget -- a host framework
// that owns and pre-partitions all device memory and forbids libraries from allocating, a real-time
// loop where an allocation (and the device synchronisation it can imply) is not allowed, or a caller
// holding no fdirw context at all.  fdirw_mass needs a context, whose creation allocates its reduction
// scratch; this entry point keeps that scratch in a fixed array compiled into the library instead.
//
// Scratch: g_mass_scratch, kMaxChunks doubles in device memory, one partial sum per chunk of kChunk
// cells, so fields of up to kMaxChunks * kChunk = 2^30 cells are accepted.  Every GPU that loads the
// library holds this 128 KiB array until the process exits.  Calls share it: two calls whose kernels
// overlap on the GPU (different streams, or host threads, without ordering between them) race on it and
// may return wrong totals.  Each call writes every partial it later reads, so nothing has to be cleared.
//
// The reduction order is fixed (chunk by chunk, then the partials in index order through one block), so
// the result is bitwise reproducible for a given n; it may differ from fdirw_mass in the last bits
// because fdirw_mass splits the field into a fixed number of chunks instead.
#include "fdirw.h"
#include "fdirw_internal.h"

#include <mutex>
#include <string>

namespace {

constexpr int64_t kChunk = 1 << 16;          // cells per partial sum
constexpr int kMaxChunks = 1 << 14;          // partial sums held by the scratch array
constexpr int kMaxDevices = 64;
constexpr int kFinalThreads = 1024;

__device__ __align__(256) double g_mass_scratch[kMaxChunks];

std::mutex g_setup_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Block b sums cells [b*kChunk, min(n, (b+1)*kChunk)): thread-strided, then a fixed xor-butterfly tree.
__global__ void __launch_bounds__(256) chunk_sum_kernel(const double* __restrict__ c, int64_t n,
                                                        double* __restrict__ partials) {
    __shared__ double sh[8];
    const int64_t lo = (int64_t)blockIdx.x * kChunk;
    const int64_t hi = lo + kChunk < n ? lo + kChunk : n;
    double acc = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) acc += c[i];
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (threadIdx.x == 0) partials[blockIdx.x] = v;
    }
}

// One block: thread t sums partials t, t + 1024, ... in order, then a fixed tree; writes *out.
__global__ void __launch_bounds__(kFinalThreads) partials_sum_kernel(const double* __restrict__ partials, int nb,
                                                                     double* __restrict__ out) {
    __shared__ double sh[kFinalThreads / 32];
    double v = 0.0;
    for (int i = threadIdx.x; i < nb; i += kFinalThreads) v += partials[i];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double w = sh[threadIdx.x];
        for (int off = 16; off > 0; off >>= 1) w += __shfl_xor_sync(0xffffffffu, w, off);
        if (threadIdx.x == 0) *out = w;
    }
}

bool is_device_memory(const void* p, int device) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
    return (a.type == cudaMemoryTypeDevice && a.device == device) || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" FDIRW_API int fdirw_mass_noalloc(const double* c, int64_t n, double* mass_out, void* stream) {
    if (n < 0 || n > (int64_t)kMaxChunks * kChunk)
        return fdirw::set_thread_error(FDIRW_ERR_ARG, "fdirw_mass_noalloc: n = " + std::to_string(n) +
                                                          " is outside [0, 2^30], the capacity of its fixed scratch");
    if ((!c && n > 0) || !mass_out)
        return fdirw::set_thread_error(FDIRW_ERR_ARG, "fdirw_mass_noalloc: NULL c or mass_out");
    if (((reinterpret_cast<uintptr_t>(c) | reinterpret_cast<uintptr_t>(mass_out)) & 7u) != 0)
        return fdirw::set_thread_error(FDIRW_ERR_ARG, "fdirw_mass_noalloc: c and mass_out must be 8-byte aligned");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fdirw::set_thread_error(FDIRW_ERR_CUDA, std::string("fdirw_mass_noalloc: no usable current device: ") +
                                                           cudaGetErrorString(e));
    if ((n > 0 && !is_device_memory(c, dev)) || !is_device_memory(mass_out, dev))
        return fdirw::set_thread_error(FDIRW_ERR_ARG,
                                       "fdirw_mass_noalloc: c and mass_out must be device memory of the current device");
    // Set-up, once per device with that device current: the host-side name of the array is only a
    // stand-in, so the kernels get the device address from cudaGetSymbolAddress.
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_setup_mu);
        if (!g_scratch_addr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_mass_scratch);
            if (e != cudaSuccess)
                return fdirw::set_thread_error(FDIRW_ERR_CUDA, std::string("fdirw_mass_noalloc: cudaGetSymbolAddress: ") +
                                                                   cudaGetErrorString(e));
            g_scratch_addr[dev] = static_cast<double*>(p);
        }
        scratch = g_scratch_addr[dev];
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int nb = (int)((n + kChunk - 1) / kChunk);
    // The launch status is read right after each launch that was issued (an empty field launches only the
    // final kernel, which writes 0), so an earlier call's error left on this thread is not reported here.
    e = cudaSuccess;
    if (nb > 0) {
        chunk_sum_kernel<<<nb, 256, 0, st>>>(c, n, scratch);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        partials_sum_kernel<<<1, kFinalThreads, 0, st>>>(scratch, nb, mass_out);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        return fdirw::set_thread_error(FDIRW_ERR_CUDA, std::string("fdirw_mass_noalloc: launch: ") + cudaGetErrorString(e));
    return FDIRW_OK;
}
