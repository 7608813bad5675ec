// The context behind the C ABI (internal to libfdirw; shared by api.cu and surrogate.cu).
#pragma once

#include <cmath>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "fdirw.h"
#include "fdirw_internal.h"

namespace fdirw {
struct Batch;   // batch of structures with per-source window radii (batch.cu)
struct Coarse;  // coarse-mesh FDiRW (coarse.cu)
}

struct fdirw_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    fdirw::Grid g{};
    double h = 1.0, dt_macro = 0.0, dt_sub = 0.0, lam = 0.0, max_face_sum = 0.0;
    int R = 0, n_sub = 0;
    int prec = FDIRW_FP32;
    fdirw::Store store = fdirw::Store::F32;
    int num_sms = 0;
    int parts_req = 0, parts_used = 0;
    uint64_t mem_limit = 0, allocated = 0;
    void* coef[3] = {nullptr, nullptr, nullptr};   // lam * g: float (mixed) or double (FP64)
    void* coefb[3] = {nullptr, nullptr, nullptr};  // convection: upper-into-lower face coefficients (flow.cu)
    bool flow = false;                              // coef / coefb hold direction-dependent coefficients
    void* Q = nullptr;
    uint64_t q_bytes = 0;
    double* sigma = nullptr;
    void* chat = nullptr;                           // padded sigma*c: double or float2
    double* cbuf = nullptr;                         // staging for host fields
    double* partials = nullptr;                     // 2 * kMassBlocks
    double* dmass = nullptr;                        // 1 double
    double* dfix = nullptr;                         // FDIRW_ACCUM_FP32: [M_in, f, max drift] of the mass restoration
    int slab_T = 0;                                 // > 0: the cache holds slab_T destination z-planes (streamed)
    double* obuf = nullptr;                         // streamed steps: output of the step being computed
    int accum = 0;                                  // fdirw_accum
    double* Dd = nullptr;                           // device copy of D (surrogate features)
    uint16_t* feat0 = nullptr;                      // surrogate feature channel 0 per cell (BF16 bits), made on first use
    int64_t* dsrc = nullptr;
    double* dkout = nullptr;
    int64_t kcap = 0;
    bool kernels_ready = false;
    bool kernels_timed = false, gather_timed = false;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    double window_cells = 0.0;
    double mass_in = NAN, mass_out = NAN;
    fdirw::Batch* batch = nullptr;                  // non-null for fdirw_create_batch contexts
    fdirw::Coarse* coarse = nullptr;                // non-null for fdirw_create_coarse contexts
    std::string err;
};

namespace fdirw {

// Host helpers of the C ABI (api.cu).
namespace host {
// Records msg on the context (or as the thread's last error when c is NULL) and returns code.
int fail(fdirw_ctx* c, int code, const std::string& msg);
std::string cuda_msg(const char* what, cudaError_t e);
// Makes `dev` current for the duration of a call and restores the caller's device afterwards.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (dev >= 0 && dev != prev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() { if (prev >= 0) cudaSetDevice(prev); }
};
enum class Kind { Host, Device, Foreign };
// Host (pageable or pinned) vs device memory of `device`; managed memory counts as device.
Kind classify(const void* p, int device);
bool grid_ok(const fdirw_grid* g);
// cudaMalloc that honours the context's mem_limit and keeps its byte count.
int dalloc(fdirw_ctx* c, void** p, uint64_t bytes, const char* what);
void dfree(void*& p);
}  // namespace host

#define FDIRW_CUDA(ctx, call)                                                                     \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            cudaGetLastError();   /* a failed call must not surface again in a later check */    \
            return fdirw::host::fail((ctx), FDIRW_ERR_CUDA, fdirw::host::cuda_msg(#call, e_));    \
        }                                                                                         \
    } while (0)

// Batch contexts (batch.cu): the entry points of the C ABI forward to these when c->batch is set.
int batch_kernels(fdirw_ctx* c);
int batch_step(fdirw_ctx* c, const double* c_in, double* c_out, int32_t n_steps, double* mass_out);
int batch_read_kernels(fdirw_ctx* c, const int64_t* sources, int64_t n, double* out);
int batch_info(fdirw_ctx* c, fdirw_info* out);
void batch_release(fdirw_ctx* c);
// Structures of a batch context: grid, first global cell, lam and h of each.
void batch_structures(const fdirw_ctx* c, std::vector<Grid>& grids, std::vector<int64_t>& base,
                      std::vector<double>& lams, std::vector<double>& hs);
void batch_invalidate(fdirw_ctx* c);           // the kernels must be rebuilt (new coefficients)

// Coarse-mesh contexts (coarse.cu).
int coarse_kernels(fdirw_ctx* c);
int coarse_step(fdirw_ctx* c, const double* c_in, double* c_out, int32_t n_steps, double* mass_out);
int coarse_info(fdirw_ctx* c, fdirw_info* out);
void coarse_release(fdirw_ctx* c);
const uint8_t* coarse_liquid(fdirw_ctx* c);    // the coarse context's liquid mask (device)
const float* coarse_open_faces(fdirw_ctx* c);  // lam * open-face conductance per cell, or NULL (no far field)
void coarse_invalidate(fdirw_ctx* c);          // the coarse matrix and P_BC must be rebuilt

// Allocates (once) and zeroes the kernel cache of a context; honours mem_limit, and falls back to a
// cache of z-slabs of destinations (slab_T) when the whole cache does not fit.
int ensure_cache(fdirw_ctx* c);
// March arguments of a uniform context (every source, the whole cache).
MarchArgs march_args(const fdirw_ctx* c);
// n_steps macro steps of a uniform context with a streamed cache (slab_T > 0).
int step_slabs(fdirw_ctx* c, const double* src, double* dst, int n_steps);
}  // namespace fdirw
