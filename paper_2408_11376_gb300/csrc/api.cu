// C ABI of libfdirw: context lifetime, argument checking, device memory, stream ordering.
// Every step of the path runs in the kernels of setup.cu, march.cu and superpose.cu; this file only
// validates, allocates, copies and launches.
#include "fdirw.h"
#include "fdirw_internal.h"
#include "ctx.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

using fdirw::Grid;
using fdirw::Store;


namespace fdirw {
namespace host {

thread_local std::string g_err;

int fail(fdirw_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg; else g_err = msg;
    return code;
}

std::string cuda_msg(const char* what, cudaError_t e) {
    return std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
}

// Host (pageable or pinned) vs device memory of `device`; managed memory counts as device.
Kind classify(const void* p, int device) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return Kind::Host; }
    if (a.type == cudaMemoryTypeManaged) return Kind::Device;
    if (a.type == cudaMemoryTypeDevice) return a.device == device ? Kind::Device : Kind::Foreign;
    return Kind::Host;
}

bool grid_ok(const fdirw_grid* g) {
    return g && g->nx >= 1 && g->ny >= 1 && g->nz >= 1 && std::isfinite(g->h) && g->h > 0.0 &&
           (double)g->nx * g->ny * g->nz < 9.0e15;
}

int dalloc(fdirw_ctx* c, void** p, uint64_t bytes, const char* what) {
    *p = nullptr;
    if (bytes == 0) return FDIRW_OK;
    if (c->mem_limit && c->allocated + bytes > c->mem_limit)
        return fail(c, FDIRW_ERR_NOMEM, std::string("allocating ") + what + " (" + std::to_string(bytes) +
                                            " bytes) would exceed mem_limit " + std::to_string(c->mem_limit));
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        *p = nullptr;
        return fail(c, FDIRW_ERR_NOMEM, std::string("cudaMalloc of ") + what + " (" + std::to_string(bytes) + " bytes) failed");
    }
    if (e != cudaSuccess) { *p = nullptr; return fail(c, FDIRW_ERR_CUDA, cuda_msg("cudaMalloc", e)); }
    c->allocated += bytes;
    return FDIRW_OK;
}

void dfree(void*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

}  // namespace host
}  // namespace fdirw

using namespace fdirw::host;

namespace {

// Sum over one axis of the clipped window extents: sum_x (min(x+R, n-1) - max(x-R, 0) + 1).
double axis_window_sum(int n, int R) {
    double s = 0.0;
    for (int x = 0; x < n; x++) s += (double)(std::min(x + R, n - 1) - std::max(x - R, 0) + 1);
    return s;
}

// D on the device (copied if host), FP64 face conductances, max face sum, invalid count.
int conductances(fdirw_ctx* c, const double* D, double* g3[3], double* max_sum) {
    const Grid& g = c->g;
    const Kind k = classify(D, c->device);
    if (k == Kind::Foreign) return fail(c, FDIRW_ERR_ARG, "D_map is device memory of another device");
    if ((reinterpret_cast<uintptr_t>(D) & 7u) != 0) return fail(c, FDIRW_ERR_ARG, "D_map is not 8-byte aligned");
    void* dD = nullptr;
    int rc;
    for (int a = 0; a < 3; a++) {
        if ((rc = dalloc(c, reinterpret_cast<void**>(&g3[a]), (uint64_t)g.n * 8, "conductances")) != FDIRW_OK) return rc;
    }
    unsigned long long* flags = nullptr;
    if ((rc = dalloc(c, reinterpret_cast<void**>(&flags), 16, "flags")) != FDIRW_OK) return rc;
    const double* Dd = D;
    if (k == Kind::Host) {
        if ((rc = dalloc(c, &dD, (uint64_t)g.n * 8, "D staging")) != FDIRW_OK) { cudaFree(flags); return rc; }
        cudaError_t e = cudaMemcpyAsync(dD, D, (size_t)g.n * 8, cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) { cudaFree(dD); cudaFree(flags); return fail(c, FDIRW_ERR_CUDA, cuda_msg("copy D_map", e)); }
        Dd = reinterpret_cast<const double*>(dD);
    }
    unsigned long long h[2] = {0ull, 0ull};
    cudaError_t e = cudaMemsetAsync(flags, 0, 16, c->stream);
    if (e == cudaSuccess) e = fdirw::launch_conductance(Dd, g, g3[0], g3[1], g3[2], flags, flags + 1, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, flags, 16, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (dD) { cudaFree(dD); c->allocated -= (uint64_t)g.n * 8; }
    cudaFree(flags);
    c->allocated -= 16;
    if (e != cudaSuccess) return fail(c, FDIRW_ERR_CUDA, cuda_msg("conductance kernel", e));
    if (h[1] != 0ull)
        return fail(c, FDIRW_ERR_ARG, "D_map holds " + std::to_string(h[1]) + " NaN, infinite or negative values");
    double m;
    std::memcpy(&m, &h[0], 8);
    *max_sum = m;
    return FDIRW_OK;
}

void release(fdirw_ctx* c) {
    fdirw::batch_release(c);
    fdirw::coarse_release(c);
    for (auto& p : c->coef) dfree(p);
    for (auto& p : c->coefb) dfree(p);
    dfree(c->Q);
    void* p;
    p = c->sigma; dfree(p); c->sigma = nullptr;
    dfree(c->chat);
    p = c->cbuf; dfree(p); c->cbuf = nullptr;
    p = c->partials; dfree(p); c->partials = nullptr;
    p = c->dmass; dfree(p); c->dmass = nullptr;
    p = c->dfix; dfree(p); c->dfix = nullptr;
    p = c->obuf; dfree(p); c->obuf = nullptr;
    p = c->Dd; dfree(p); c->Dd = nullptr;
    p = c->feat0; dfree(p); c->feat0 = nullptr;
    p = c->dsrc; dfree(p); c->dsrc = nullptr;
    p = c->dkout; dfree(p); c->dkout = nullptr;
    for (auto& e : c->ev) if (e) { cudaEventDestroy(e); e = nullptr; }
}

}  // namespace

// The kernel cache: all N destinations when they fit the device's free memory (less a reserve) and the
// context's mem_limit; otherwise slab streaming, a cache of T destination z-planes (as many as fit next
// to an output field) that every macro step refills slab by slab: the kernels are marched again each
// step, for the sources within R planes of the slab.
int fdirw::ensure_cache(fdirw_ctx* c) {
    if (c->Q) return FDIRW_OK;
    const uint64_t W = (uint64_t)(2 * c->R + 1) * (2 * c->R + 1) * (2 * c->R + 1);
    const uint64_t plane = W * (uint64_t)c->g.nx * (uint64_t)c->g.ny * (uint64_t)fdirw::store_bytes(c->store);
    const uint64_t full = plane * (uint64_t)c->g.nz;
    size_t free_b = 0, total_b = 0;
    uint64_t budget = ~0ull;
    constexpr uint64_t kReserve = 1ull << 30;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) budget = free_b > kReserve ? free_b - kReserve : 0;
    else cudaGetLastError();                                   // unknown: let the allocation decide
    if (c->mem_limit) budget = std::min<uint64_t>(budget, c->mem_limit > c->allocated ? c->mem_limit - c->allocated : 0);
    const uint64_t obytes = (uint64_t)c->g.n * 8;
    int T = c->g.nz;
    if (full > budget) {
        const uint64_t rest = budget > obytes ? budget - obytes : 0;
        T = (int)std::min<uint64_t>(rest / plane, (uint64_t)c->g.nz);
    }
    // Largest slab that allocates: the whole grid when it fits, else halving after a failed allocation
    // (free memory can be fragmented or taken meanwhile).
    while (T >= 1) {
        const bool streamed = T < c->g.nz;
        if (streamed && !c->obuf) {
            const int rc = dalloc(c, reinterpret_cast<void**>(&c->obuf), obytes, "streamed step output");
            if (rc != FDIRW_OK) return rc;
        }
        const int rc = dalloc(c, &c->Q, plane * (uint64_t)T, "kernel cache");
        if (rc == FDIRW_OK) {
            c->q_bytes = plane * (uint64_t)T;
            c->slab_T = streamed ? T : 0;
            if (!streamed && c->obuf) {
                void* p = c->obuf; dfree(p); c->obuf = nullptr;
                c->allocated -= obytes;
            }
            // Entries whose source lies outside the domain are never written by the march: zero them once.
            FDIRW_CUDA(c, cudaMemsetAsync(c->Q, 0, c->q_bytes, c->stream));
            return FDIRW_OK;
        }
        if (rc != FDIRW_ERR_NOMEM) return rc;
        T = streamed ? T / 2 : std::min(T - 1, std::max(c->g.nz / 2, 1));
    }
    return fail(c, FDIRW_ERR_NOMEM, "the kernel cache does not fit, not even one z-plane of destinations (" +
                                        std::to_string(plane) + " bytes)");
}

// March arguments of a uniform context: every source, the whole cache.
fdirw::MarchArgs fdirw::march_args(const fdirw_ctx* c) {
    MarchArgs a{};
    a.g = c->g;
    a.R = c->R;
    a.Rq = c->R;
    a.q_stride = c->g.n;
    a.n_sub = c->n_sub;
    if (c->store == Store::F64) {
        a.dx = reinterpret_cast<const double*>(c->coef[0]);
        a.dy = reinterpret_cast<const double*>(c->coef[1]);
        a.dz = reinterpret_cast<const double*>(c->coef[2]);
    } else {
        a.ax = reinterpret_cast<const float*>(c->coef[0]);
        a.ay = reinterpret_cast<const float*>(c->coef[1]);
        a.az = reinterpret_cast<const float*>(c->coef[2]);
    }
    a.Q = c->Q;
    a.store = c->store;
    a.sigma = c->sigma;
    a.src_begin = 0;
    a.src_end = c->g.n;
    a.list = nullptr;
    if (c->flow) {                                    // convection: direction-dependent faces (mapping 5)
        a.bx = reinterpret_cast<const float*>(c->coefb[0]);
        a.by = reinterpret_cast<const float*>(c->coefb[1]);
        a.bz = reinterpret_cast<const float*>(c->coefb[2]);
    }
    return a;
}

// Macro steps with a streamed cache: per step and slab of T destination planes, the march of the sources
// within R planes of the slab (only the slab's destinations stored, sigma of every marched source), the
// scaled field of those sources, and the gather of the slab into a buffer other than the step's input;
// then the mass restoration (FP32 accumulation).  Results equal the resident cache's bit for bit.
int fdirw::step_slabs(fdirw_ctx* c, const double* src, double* dst, int n_steps) {
    const int T = c->slab_T, nz = c->g.nz, R = c->R;
    const int64_t nxy = (int64_t)c->g.nx * c->g.ny;
    const bool fp32acc = c->accum == FDIRW_ACCUM_FP32;
    const int mode = c->store == Store::F64 ? 0 : fp32acc ? 2 : 1;
    if (fp32acc) {
        FDIRW_CUDA(c, fdirw::launch_mass(src, c->g.n, c->partials, c->dfix, c->stream));
        FDIRW_CUDA(c, cudaMemsetAsync(c->dfix + 2, 0, 8, c->stream));
    }
    MarchArgs a = march_args(c);
    a.q_stride = (int64_t)T * nxy;
    const double* cur = src;
    for (int t = 0; t < n_steps; t++) {
        // The step writes a buffer other than its input; the last one lands in dst unless dst is the input.
        double* out = ((n_steps - 1 - t) % 2 == 0) ? dst : c->obuf;
        if (out == cur) out = (out == dst) ? c->obuf : dst;
        for (int z0 = 0; z0 < nz; z0 += T) {
            const int zn = std::min(T, nz - z0);
            const int zs0 = std::max(z0 - R, 0), zs1 = std::min(z0 + zn + R, nz);
            a.src_begin = (int64_t)zs0 * nxy;
            a.src_end = (int64_t)zs1 * nxy;
            a.dest_lo = (int64_t)z0 * nxy;
            a.dest_hi = (int64_t)(z0 + zn) * nxy;
            FDIRW_CUDA(c, launch_march(a, c->num_sms, c->parts_req, c->stream, &c->parts_used));
            FDIRW_CUDA(c, launch_scale(cur, c->sigma, c->g, R, c->chat, mode, c->stream, zs0, zs1 - zs0));
            FDIRW_CUDA(c, launch_gather_slab(c->Q, c->store, (int64_t)T * nxy, a.dest_lo, c->chat, c->g, R, mode, z0,
                                             zn, out, c->stream));
        }
        if (fp32acc) FDIRW_CUDA(c, fdirw::launch_restore_mass(out, c->g.n, c->partials, c->dfix, c->stream));
        cur = out;
    }
    if (cur != dst) FDIRW_CUDA(c, cudaMemcpyAsync(dst, cur, (size_t)c->g.n * 8, cudaMemcpyDeviceToDevice, c->stream));
    return FDIRW_OK;
}

int fdirw::set_thread_error(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

extern "C" {

const char* fdirw_last_error(const fdirw_ctx* ctx) {
    return ctx ? ctx->err.c_str() : g_err.c_str();
}

int fdirw_stable_dt(const fdirw_grid* grid, const double* D_map, int32_t device, double* dt_sub_max) {
    if (!grid_ok(grid)) return fail(nullptr, FDIRW_ERR_ARG, "invalid grid (dimensions >= 1, finite h > 0)");
    if (!D_map || !dt_sub_max) return fail(nullptr, FDIRW_ERR_ARG, "NULL D_map or dt_sub_max");
    DeviceGuard dg(device);
    if (!dg.ok) return fail(nullptr, FDIRW_ERR_CUDA, "cannot select CUDA device " + std::to_string(device));
    fdirw_ctx tmp;
    cudaGetDevice(&tmp.device);
    tmp.g = Grid{grid->nx, grid->ny, grid->nz, (int64_t)grid->nx * grid->ny * grid->nz};
    double* g3[3] = {nullptr, nullptr, nullptr};
    double m = 0.0;
    const int rc = conductances(&tmp, D_map, g3, &m);
    for (auto& p : g3) if (p) cudaFree(p);
    if (rc != FDIRW_OK) return fail(nullptr, rc, tmp.err);
    *dt_sub_max = m > 0.0 ? grid->h * grid->h / m : HUGE_VAL;
    return FDIRW_OK;
}

int fdirw_create(const fdirw_grid* grid, const double* D_map, double dt_macro, int32_t window_R, int32_t n_sub,
                 const fdirw_opts* opts, fdirw_ctx** out) {
    if (!out) return fail(nullptr, FDIRW_ERR_ARG, "NULL out");
    *out = nullptr;
    if (!grid_ok(grid)) return fail(nullptr, FDIRW_ERR_ARG, "invalid grid (dimensions >= 1, finite h > 0)");
    if (!D_map) return fail(nullptr, FDIRW_ERR_ARG, "NULL D_map");
    if (!(std::isfinite(dt_macro) && dt_macro >= 0.0)) return fail(nullptr, FDIRW_ERR_ARG, "dt_macro must be finite and >= 0");
    if (window_R < 0 || window_R > fdirw::kMaxR)
        return fail(nullptr, FDIRW_ERR_ARG, "window_R must be in [0, " + std::to_string(fdirw::kMaxR) + "]");
    if (n_sub < 0) return fail(nullptr, FDIRW_ERR_ARG, "n_sub must be >= 0");
    fdirw_opts o{FDIRW_FP32, -1, nullptr, 0, 0, 0};
    if (opts) o = *opts;
    if (o.prec < FDIRW_FP64 || o.prec > FDIRW_FP32_STORE_BF16) return fail(nullptr, FDIRW_ERR_ARG, "unknown prec");
    if (o.march_parts < 0 || o.march_parts > 7) return fail(nullptr, FDIRW_ERR_ARG, "march_parts must be in [0, 7]");
    if (o.accum != FDIRW_ACCUM_FF && o.accum != FDIRW_ACCUM_FP32) return fail(nullptr, FDIRW_ERR_ARG, "unknown accum");
    if (o.accum == FDIRW_ACCUM_FP32 && o.prec == FDIRW_FP64)
        return fail(nullptr, FDIRW_ERR_ARG, "FDIRW_ACCUM_FP32 needs an FP32-march precision");
    if (o.prec == FDIRW_FP64 && window_R > fdirw::kMaxR64)
        return fail(nullptr, FDIRW_ERR_ARG, "FDIRW_FP64 supports window_R <= " + std::to_string(fdirw::kMaxR64));

    DeviceGuard dg(o.device);
    if (!dg.ok) return fail(nullptr, FDIRW_ERR_CUDA, "cannot select CUDA device " + std::to_string(o.device));
    fdirw_ctx* c = new fdirw_ctx();
    cudaGetDevice(&c->device);
    c->stream = reinterpret_cast<cudaStream_t>(o.stream);
    c->mem_limit = o.mem_limit;
    c->parts_req = o.march_parts;
    c->accum = o.accum;
    c->g = Grid{grid->nx, grid->ny, grid->nz, (int64_t)grid->nx * grid->ny * grid->nz};
    c->h = grid->h;
    c->dt_macro = dt_macro;
    c->R = window_R;
    c->n_sub = n_sub;
    c->prec = o.prec;
    c->store = o.prec == FDIRW_FP64 ? Store::F64 : o.prec == FDIRW_FP32 ? Store::F32
             : o.prec == FDIRW_FP32_STORE_FP16 ? Store::F16 : Store::BF16;
    c->dt_sub = n_sub > 0 ? dt_macro / n_sub : 0.0;
    c->lam = c->dt_sub / (grid->h * grid->h);
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);

    auto bail = [&](int rc) {
        std::string msg = c->err;
        release(c);
        delete c;
        return fail(nullptr, rc, msg);
    };

    double* g3[3] = {nullptr, nullptr, nullptr};
    int rc = conductances(c, D_map, g3, &c->max_face_sum);
    if (rc != FDIRW_OK) {
        for (auto& p : g3) if (p) cudaFree(p);
        return bail(rc);
    }
    for (int a = 0; a < 3; a++) c->coef[a] = g3[a];
    if (c->lam * c->max_face_sum > 1.0 + 1e-12) {
        char buf[256];
        std::snprintf(buf, sizeof buf, "unstable: dt_sub*max(sum g)/h^2 = %.17g > 1 (largest stable dt_sub = %.17g)",
                      c->lam * c->max_face_sum, c->max_face_sum > 0 ? c->h * c->h / c->max_face_sum : HUGE_VAL);
        c->err = buf;
        return bail(FDIRW_ERR_UNSTABLE);
    }
    const uint64_t n = (uint64_t)c->g.n;
    if (c->store == Store::F64) {
        for (int a = 0; a < 3; a++) {
            cudaError_t e = fdirw::launch_coef_f64(reinterpret_cast<double*>(c->coef[a]), c->lam, c->g.n, c->stream);
            if (e != cudaSuccess) { c->err = cuda_msg("coefficient kernel", e); return bail(FDIRW_ERR_CUDA); }
        }
    } else {
        for (int a = 0; a < 3; a++) {
            void* f = nullptr;
            if ((rc = dalloc(c, &f, n * 4, "coefficients")) != FDIRW_OK) return bail(rc);
            cudaError_t e = fdirw::launch_coef_f32(reinterpret_cast<double*>(c->coef[a]), c->lam, c->g.n,
                                                   reinterpret_cast<float*>(f), c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) { cudaFree(f); c->err = cuda_msg("coefficient kernel", e); return bail(FDIRW_ERR_CUDA); }
            cudaFree(c->coef[a]);
            c->allocated -= n * 8;
            c->coef[a] = f;
        }
    }
    const fdirw::Pad pad = fdirw::make_pad(c->g, c->R);
    if ((rc = dalloc(c, reinterpret_cast<void**>(&c->Dd), n * 8, "D copy")) != FDIRW_OK) return bail(rc);
    {
        cudaError_t e = cudaMemcpyAsync(c->Dd, D_map, n * 8, cudaMemcpyDefault, c->stream);
        if (e != cudaSuccess) { c->err = cuda_msg("copy D_map", e); return bail(FDIRW_ERR_CUDA); }
    }
    if ((rc = dalloc(c, reinterpret_cast<void**>(&c->sigma), n * 8, "sigma")) != FDIRW_OK) return bail(rc);
    if ((rc = dalloc(c, &c->chat, (uint64_t)pad.n * 8, "scaled field")) != FDIRW_OK) return bail(rc);
    if ((rc = dalloc(c, reinterpret_cast<void**>(&c->cbuf), n * 8, "field staging")) != FDIRW_OK) return bail(rc);
    if ((rc = dalloc(c, reinterpret_cast<void**>(&c->partials), 2 * fdirw::kMassBlocks * 8, "mass partials")) != FDIRW_OK) return bail(rc);
    if ((rc = dalloc(c, reinterpret_cast<void**>(&c->dmass), 8, "mass")) != FDIRW_OK) return bail(rc);
    if ((rc = dalloc(c, reinterpret_cast<void**>(&c->dfix), 24, "mass restoration")) != FDIRW_OK) return bail(rc);
    cudaError_t e = cudaMemsetAsync(c->chat, 0, (size_t)pad.n * 8, c->stream);
    for (int i = 0; i < 4 && e == cudaSuccess; i++) e = cudaEventCreate(&c->ev[i]);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) { c->err = cuda_msg("context setup", e); return bail(FDIRW_ERR_CUDA); }
    c->window_cells = axis_window_sum(c->g.nx, c->R) * axis_window_sum(c->g.ny, c->R) * axis_window_sum(c->g.nz, c->R);
    *out = c;
    return FDIRW_OK;
}

int fdirw_kernels(fdirw_ctx* c) {
    if (!c) return fail(nullptr, FDIRW_ERR_ARG, "NULL context");
    DeviceGuard dg(c->device);
    if (c->batch) return fdirw::batch_kernels(c);
    if (c->coarse) return fdirw::coarse_kernels(c);
    if (c->R == 0) { c->kernels_ready = true; return FDIRW_OK; }
    const int rc = fdirw::ensure_cache(c);
    if (rc != FDIRW_OK) return rc;
    if (c->slab_T) { c->kernels_ready = true; return FDIRW_OK; }   // streamed: marched by every step
    fdirw::MarchArgs a = fdirw::march_args(c);
    FDIRW_CUDA(c, cudaEventRecord(c->ev[0], c->stream));
    FDIRW_CUDA(c, fdirw::launch_march(a, c->num_sms, c->parts_req, c->stream, &c->parts_used));
    FDIRW_CUDA(c, cudaEventRecord(c->ev[1], c->stream));
    c->kernels_timed = true;
    c->kernels_ready = true;
    return FDIRW_OK;
}

int fdirw_step(fdirw_ctx* c, const double* c_in, double* c_out, int32_t n_steps, double* mass_out) {
    if (!c) return fail(nullptr, FDIRW_ERR_ARG, "NULL context");
    if (!c_in || !c_out) return fail(c, FDIRW_ERR_ARG, "NULL c_in or c_out");
    if (n_steps < 0) return fail(c, FDIRW_ERR_ARG, "n_steps must be >= 0");
    if (((reinterpret_cast<uintptr_t>(c_in) | reinterpret_cast<uintptr_t>(c_out)) & 7u) != 0)
        return fail(c, FDIRW_ERR_ARG, "c_in and c_out must be 8-byte aligned");
    DeviceGuard dg(c->device);
    if (c->batch) return fdirw::batch_step(c, c_in, c_out, n_steps, mass_out);
    if (c->coarse) return fdirw::coarse_step(c, c_in, c_out, n_steps, mass_out);
    const Kind kin = classify(c_in, c->device), kout = classify(c_out, c->device);
    if (kin == Kind::Foreign || kout == Kind::Foreign)
        return fail(c, FDIRW_ERR_ARG, "c_in/c_out are device memory of another device");
    if (!c->kernels_ready) {
        const int rc = fdirw_kernels(c);
        if (rc != FDIRW_OK) return rc;
    }
    const size_t bytes = (size_t)c->g.n * 8;
    const double* src = c_in;
    if (kin == Kind::Host) {
        FDIRW_CUDA(c, cudaMemcpyAsync(c->cbuf, c_in, bytes, cudaMemcpyHostToDevice, c->stream));
        src = c->cbuf;
    }
    double* dst = kout == Kind::Device ? c_out : c->cbuf;
    if (mass_out) {
        FDIRW_CUDA(c, fdirw::launch_mass(src, c->g.n, c->partials, c->dmass, c->stream));
        FDIRW_CUDA(c, cudaMemcpyAsync(&c->mass_in, c->dmass, 8, cudaMemcpyDeviceToHost, c->stream));
    }
    const bool identity = c->R == 0 || n_steps == 0;
    if (identity) {
        if (dst != src) FDIRW_CUDA(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, c->stream));
    } else if (c->slab_T) {
        const int rc = fdirw::step_slabs(c, src, dst, n_steps);
        if (rc != FDIRW_OK) return rc;
    } else {
        const bool fp32acc = c->accum == FDIRW_ACCUM_FP32;
        const int mode = c->store == Store::F64 ? 0 : fp32acc ? 2 : 1;
        // FDIRW_ACCUM_FP32: the FP64 total of the call's input, the target of every step's restoration.
        if (fp32acc) {
            FDIRW_CUDA(c, fdirw::launch_mass(src, c->g.n, c->partials, c->dfix, c->stream));
            FDIRW_CUDA(c, cudaMemsetAsync(c->dfix + 2, 0, 8, c->stream));
        }
        const double* cur = src;
        for (int t = 0; t < n_steps; t++) {
            FDIRW_CUDA(c, fdirw::launch_scale(cur, c->sigma, c->g, c->R, c->chat, mode, c->stream));
            const bool last = t + 1 == n_steps;
            if (last) FDIRW_CUDA(c, cudaEventRecord(c->ev[2], c->stream));
            if (fp32acc) {
                FDIRW_CUDA(c, fdirw::launch_gather_fp32(c->Q, c->store, reinterpret_cast<const float*>(c->chat), c->g,
                                                        c->R, dst, c->stream));
            } else {
                FDIRW_CUDA(c, fdirw::launch_gather(c->Q, c->store, c->chat, c->g, c->R, dst, c->stream));
            }
            if (last) FDIRW_CUDA(c, cudaEventRecord(c->ev[3], c->stream));
            if (fp32acc) FDIRW_CUDA(c, fdirw::launch_restore_mass(dst, c->g.n, c->partials, c->dfix, c->stream));
            cur = dst;
        }
        c->gather_timed = true;
    }
    if (mass_out) {
        FDIRW_CUDA(c, fdirw::launch_mass(dst, c->g.n, c->partials, c->dmass, c->stream));
        FDIRW_CUDA(c, cudaMemcpyAsync(&c->mass_out, c->dmass, 8, cudaMemcpyDeviceToHost, c->stream));
    }
    if (kout == Kind::Host) FDIRW_CUDA(c, cudaMemcpyAsync(c_out, dst, bytes, cudaMemcpyDeviceToHost, c->stream));
    if (mass_out || kout == Kind::Host) FDIRW_CUDA(c, cudaStreamSynchronize(c->stream));
    if (mass_out) *mass_out = c->mass_out;
    return FDIRW_OK;
}

int fdirw_mass(fdirw_ctx* c, const double* field, double* mass_out) {
    if (!c) return fail(nullptr, FDIRW_ERR_ARG, "NULL context");
    if (!field || !mass_out) return fail(c, FDIRW_ERR_ARG, "NULL field or mass_out");
    if ((reinterpret_cast<uintptr_t>(field) & 7u) != 0) return fail(c, FDIRW_ERR_ARG, "field must be 8-byte aligned");
    DeviceGuard dg(c->device);
    const Kind k = classify(field, c->device);
    if (k == Kind::Foreign) return fail(c, FDIRW_ERR_ARG, "field is device memory of another device");
    const double* src = field;
    if (k == Kind::Host) {
        FDIRW_CUDA(c, cudaMemcpyAsync(c->cbuf, field, (size_t)c->g.n * 8, cudaMemcpyHostToDevice, c->stream));
        src = c->cbuf;
    }
    double m = 0.0;
    FDIRW_CUDA(c, fdirw::launch_mass(src, c->g.n, c->partials, c->dmass, c->stream));
    FDIRW_CUDA(c, cudaMemcpyAsync(&m, c->dmass, 8, cudaMemcpyDeviceToHost, c->stream));
    FDIRW_CUDA(c, cudaStreamSynchronize(c->stream));
    *mass_out = m;
    return FDIRW_OK;
}

int fdirw_read_kernels(fdirw_ctx* c, const int64_t* sources, int64_t n, double* out) {
    if (!c) return fail(nullptr, FDIRW_ERR_ARG, "NULL context");
    if (n < 0 || (n > 0 && (!sources || !out))) return fail(c, FDIRW_ERR_ARG, "bad sources/out");
    for (int64_t q = 0; q < n; q++)
        if (sources[q] < 0 || sources[q] >= c->g.n) return fail(c, FDIRW_ERR_ARG, "source index out of range");
    if (c->coarse) return fail(c, FDIRW_ERR_ARG, "a coarse-mesh context has no per-source kernels (fdirw_read_coarse)");
    if (!c->kernels_ready) return fail(c, FDIRW_ERR_STATE, "kernel cache not built (call fdirw_kernels)");
    if (c->slab_T) return fail(c, FDIRW_ERR_STATE, "the kernel cache is streamed by z-slabs: no kernel stays resident");
    if (n == 0) return FDIRW_OK;
    if (c->batch) {
        DeviceGuard dg(c->device);
        return fdirw::batch_read_kernels(c, sources, n, out);
    }
    if (c->R == 0) {
        for (int64_t q = 0; q < n; q++) out[q] = 1.0;
        return FDIRW_OK;
    }
    DeviceGuard dg(c->device);
    const int64_t W = (int64_t)(2 * c->R + 1) * (2 * c->R + 1) * (2 * c->R + 1);
    if (n > c->kcap) {
        void* p = c->dsrc; dfree(p); c->dsrc = nullptr;
        p = c->dkout; dfree(p); c->dkout = nullptr;
        c->allocated -= (uint64_t)c->kcap * (8 + 8 * W);
        c->kcap = 0;
        int rc = dalloc(c, reinterpret_cast<void**>(&c->dsrc), (uint64_t)n * 8, "source list");
        if (rc != FDIRW_OK) return rc;
        rc = dalloc(c, reinterpret_cast<void**>(&c->dkout), (uint64_t)n * W * 8, "kernel readback");
        if (rc != FDIRW_OK) return rc;
        c->kcap = n;
    }
    FDIRW_CUDA(c, cudaMemcpyAsync(c->dsrc, sources, (size_t)n * 8, cudaMemcpyHostToDevice, c->stream));
    FDIRW_CUDA(c, fdirw::launch_read_kernels(c->Q, c->store, c->sigma, c->g, c->R, c->dsrc, n, c->dkout, c->stream));
    FDIRW_CUDA(c, cudaMemcpyAsync(out, c->dkout, (size_t)(n * W) * 8, cudaMemcpyDeviceToHost, c->stream));
    FDIRW_CUDA(c, cudaStreamSynchronize(c->stream));
    return FDIRW_OK;
}

int fdirw_get_info(fdirw_ctx* c, fdirw_info* out) {
    if (!c || !out) return fail(c, FDIRW_ERR_ARG, "NULL context or out");
    DeviceGuard dg(c->device);
    std::memset(out, 0, sizeof *out);
    out->n_cells = c->g.n;
    out->window_R = c->R;
    out->n_sub = c->n_sub;
    out->prec = c->prec;
    out->kernels_ready = c->kernels_ready ? 1 : 0;
    out->dt_sub = c->dt_sub;
    out->lam = c->lam;
    out->max_face_sum = c->max_face_sum;
    out->cache_bytes = c->q_bytes;
    out->device_bytes = c->allocated;
    out->window_cells = c->window_cells;
    out->last_mass_in = c->mass_in;
    out->last_mass_out = c->mass_out;
    out->march_parts = c->parts_used;
    out->accum = c->accum;
    float ms = 0.f;
    if (c->kernels_timed) {
        FDIRW_CUDA(c, cudaEventSynchronize(c->ev[1]));
        FDIRW_CUDA(c, cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
        out->kernels_ms = ms;
    }
    if (c->gather_timed) {
        FDIRW_CUDA(c, cudaEventSynchronize(c->ev[3]));
        FDIRW_CUDA(c, cudaEventElapsedTime(&ms, c->ev[2], c->ev[3]));
        out->last_gather_ms = ms;
    }
    if (c->batch) return fdirw::batch_info(c, out);
    if (c->coarse) return fdirw::coarse_info(c, out);
    if (c->accum == FDIRW_ACCUM_FP32 && c->dfix) {
        FDIRW_CUDA(c, cudaMemcpyAsync(&out->last_restore_drift, c->dfix + 2, 8, cudaMemcpyDeviceToHost, c->stream));
        FDIRW_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    out->n_chunks = c->slab_T ? (c->g.nz + c->slab_T - 1) / c->slab_T : 1;   // z-slabs of a streamed cache
    return FDIRW_OK;
}

void fdirw_destroy(fdirw_ctx* c) {
    if (!c) return;
    {
        DeviceGuard dg(c->device);
        if (c->stream) cudaStreamSynchronize(c->stream); else cudaDeviceSynchronize();
        release(c);
    }
    delete c;
}

}  // extern "C"
