// The context behind the C ABI (internal to libfdirw; shared by api.cu and surrogate.cu).
#pragma once

#include <cmath>
#include <string>

#include <cuda_runtime.h>

#include "fdirw.h"
#include "fdirw_internal.h"

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
    void* Q = nullptr;
    uint64_t q_bytes = 0;
    double* sigma = nullptr;
    void* chat = nullptr;                           // padded sigma*c: double or float2
    double* cbuf = nullptr;                         // staging for host fields
    double* partials = nullptr;                     // kMassBlocks
    double* dmass = nullptr;                        // 1 double
    double* Dd = nullptr;                           // device copy of D (surrogate features)
    int64_t* dsrc = nullptr;
    double* dkout = nullptr;
    int64_t kcap = 0;
    bool kernels_ready = false;
    bool kernels_timed = false, gather_timed = false;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    double window_cells = 0.0;
    double mass_in = NAN, mass_out = NAN;
    std::string err;
};

namespace fdirw {
// Allocates (once) and zeroes the kernel cache of a context; honours mem_limit.
int ensure_cache(fdirw_ctx* c);
}  // namespace fdirw
