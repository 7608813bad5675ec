// Internal declarations shared by the CUDA translation units of libfdirw (not part of the C ABI).
#pragma once

#include <cstdint>
#include <string>

#include <cuda_runtime.h>

namespace fdirw {

// Largest window radius: the FP32 march supports R <= 10 (window 21^3), the FP64 march R <= 8.
constexpr int kMaxR = 10;
constexpr int kMaxR64 = 8;

enum class Store : int { F64 = 0, F32 = 1, F16 = 2, BF16 = 3 };

inline int store_bytes(Store s) { return s == Store::F64 ? 8 : s == Store::F32 ? 4 : 2; }

struct Grid {
    int nx, ny, nz;
    int64_t n;     // nx*ny*nz
};

// Records msg as this host thread's last error (what fdirw_last_error(NULL) returns); returns code.
int set_thread_error(int code, const std::string& msg);

// ---------------------------------------------------------------- setup.cu
// Checks D (finite, >= 0), computes FP64 harmonic-mean face conductances gx/gy/gz (+x/+y/+z face of each
// cell, 0 across the domain edge), the maximum per-cell face sum (as the bit pattern of a non-negative
// double, for atomicMax) and the number of invalid D values.  *max_bits and *bad must be zeroed first.
cudaError_t launch_conductance(const double* D, Grid g, double* gx, double* gy, double* gz,
                               unsigned long long* max_bits, unsigned long long* bad, cudaStream_t st);
// coef = lam * g (FP32, one rounding from FP64).
cudaError_t launch_coef_f32(const double* g, double lam, int64_t n, float* coef, cudaStream_t st);
// coef = lam * g in place (FP64).
cudaError_t launch_coef_f64(double* g, double lam, int64_t n, cudaStream_t st);

// ---------------------------------------------------------------- march.cu
struct MarchArgs {
    Grid g;
    int R;                // window radius of the marched sources
    int Rq;               // radius of the cache layout (Rq >= R; equal for a uniform window)
    int n_sub;
    const float* ax; const float* ay; const float* az;     // FP32 path: lam*g
    const double* dx; const double* dy; const double* dz;  // FP64 path: lam*g
    void* Q;              // kernel cache, (2Rq+1)^3 planes
    Store store;
    double* sigma;        // N: 1 / FP64 sum of the stored values of each source
    int64_t src_begin, src_end;
    const int64_t* list;  // nullable: march sources list[src_begin..src_end) instead of that range
    // Batch of structures (nstruct > 0, FP32 march only): sources and coefficients index the
    // concatenation; structure i holds global cells [s_base[i], s_base[i+1]) of dimensions s_dims[i].
    int nstruct;
    const int64_t* s_base;
    const int4* s_dims;
    const int64_t* s_qbase;   // nullable: first cache column of each structure (destination-indexed layout)
    // Q index = plane * q_stride + column; the column is the destination cell (src_major = 0: the cell's
    // index within its structure plus s_qbase, or the global cell without s_qbase) or the source's
    // position in [src_begin, src_end) (src_major = 1).
    int64_t q_stride;
    int src_major;
    // Coarse-mesh march (coarse_B > 0, mapping 5 only): list holds coarse block indices; see coarse.cu.
    int coarse_B, coarse_Rc;
    int ncx, ncy, ncz;
    int64_t coarse_n;            // ncx * ncy * ncz
    const uint8_t* liquid;       // N: 1 = liquid cell
    const int32_t* ccount;       // coarse_n: liquid cells per block
    double* Qc;                  // (2 Rc + 1)^3 planes of coarse_n values, destination-indexed
    const float* abnd;           // nullable: lam * open-face conductance of each cell (far-field boundary)
    // Convection (nullable; mapping 5 only): ax/ay/az then hold the coefficient of the lower cell in the
    // upper cell's update across each +face, bx/by/bz that of the upper cell in the lower cell's update.
    const float* bx; const float* by; const float* bz;
    // Slab streaming of a uniform context (dest_hi > dest_lo): only destinations in [dest_lo, dest_hi)
    // are stored, at column dest - dest_lo; the others are rounded (for sigma) but not stored.
    int64_t dest_lo, dest_hi;
};
// Coarse-mesh march of the blocks a.list[src_begin..src_end): window radius R = window_R + (B - 1) / 2
// (1..10), one source per CTA.
cudaError_t launch_march_coarse(const MarchArgs& a, int R, int num_sms, cudaStream_t st);
// parts_req: FP32 march thread mapping (1..3 threads per window column, 4 = 2x2 column blocks with TMEM
// faces, 5 = one column per thread with TMEM lateral faces), or 0 to autotune (timed once per device, R
// and storage, then cached); parts_used receives the mapping launched.
cudaError_t launch_march(const MarchArgs& a, int num_sms, int parts_req, cudaStream_t st, int* parts_used);
// The thread mapping launch_march would use for parts_req (timing the candidates on `a`'s sources when
// autotuning and nothing is cached, which synchronises st and overwrites part of a.Q); launches nothing
// else, so that the following launches can be captured into a graph.
cudaError_t tune_march(const MarchArgs& a, int num_sms, int parts_req, cudaStream_t st, int* parts);

// ---------------------------------------------------------------- superpose.cu
// Padded layout of the scaled field chat = sigma * c: (nx+2R) x (ny+2R) x (nz+2R), zero halo.
struct Pad {
    int px, py, pz;
    int64_t n;
};
inline Pad make_pad(const Grid& g, int R) {
    Pad p{g.nx + 2 * R, g.ny + 2 * R, g.nz + 2 * R, 0};
    p.n = (int64_t)p.px * p.py * p.pz;
    return p;
}
// chat = sigma * c into the interior of the padded buffer (zero halo of R cells): mode 0 FP64, mode 1 a
// float2 (hi, lo) pair with hi = fp32(v), lo = fp32(v - hi), mode 2 fp32(v).  Cells of the z-planes
// [z0, z0 + zn) only (zn < 0: all planes).
cudaError_t launch_scale(const double* c, const double* sigma, Grid g, int R, void* chat, int mode,
                         cudaStream_t st, int z0 = 0, int zn = -1);
// c_out(x) = sum_o Q[o][x] * chat(x - o).
cudaError_t launch_gather(const void* Q, Store store, const void* chat, Grid g, int R, double* c_out,
                          cudaStream_t st);
// The radius-R part of the gather for one grid whose chat is padded with a halo of Rp >= R cells and
// whose Q planes are qs values apart: c_out(x) = [c_out(x) +] sum_{|o| <= R} Q[o][x] * chat(x - o), the
// rows (o_z, o_y) in ascending order as in launch_gather.
cudaError_t launch_gather_part(const void* Q, Store store, int64_t qs, const void* chat, int Rp, Grid g, int R,
                               bool accumulate, double* c_out, cudaStream_t st);
// Deterministic FP64 total: partials[kMassBlocks] then one block.  partials must hold kMassBlocks doubles.
constexpr int kMassBlocks = 1024;
cudaError_t launch_mass(const double* c, int64_t n, double* partials, double* out, cudaStream_t st);
// FDIRW_ACCUM_FP32 superposition of a uniform context: FP32 chat (launch_scale mode 2), FP32 products
// and row sums, double-float row accumulation.
cudaError_t launch_gather_fp32(const void* Q, Store store, const float* chat, Grid g, int R, double* c_out,
                               cudaStream_t st);
// Restores the FP64 total of c to *m_in: c[i] += f |c[i]|, f = (m_in - sum c) / sum |c| (0 when the
// field is zero), both sums in a fixed order.  partials: 2 * kMassBlocks doubles; fix: 2 doubles
// (fix[0] = m_in on entry, fix[1] = f on exit).
cudaError_t launch_restore_mass(double* c, int64_t n, double* partials, double* fix, cudaStream_t st);
// The destinations of the z-planes [z0, z0 + zn) of a uniform context whose cache holds only those
// destinations (column = cell - qoff, plane stride qs): mode 0 FP64, 1 float-float, 2 FP32 arithmetic.
cudaError_t launch_gather_slab(const void* Q, Store store, int64_t qs, int64_t qoff, const void* chat, Grid g, int R,
                               int mode, int z0, int zn, double* c_out, cudaStream_t st);
// launch_gather_part with the FDIRW_ACCUM_FP32 arithmetic (FP32 chat with a halo of Rp).
cudaError_t launch_gather_part_fp32(const void* Q, Store store, int64_t qs, const float* chat, int Rp, Grid g, int R,
                                    bool accumulate, double* c_out, cudaStream_t st);
// Per-structure mass restoration of structures [s0, s1) whose cells are [base[i], base[i + 1]) (base on
// the device): launch_seg_target stores each structure's FP64 total of c in fix[2 i]; launch_seg_restore
// then adds f_i |c| to every cell of structure i, f_i = (fix[2 i] - sum c) / sum |c|.  partials holds
// 2 * kSegBlocks doubles per structure of the range.
constexpr int kSegBlocks = 32;
cudaError_t launch_seg_target(const double* c, const int64_t* base, int s0, int s1, double* partials, double* fix,
                              cudaStream_t st);
cudaError_t launch_seg_restore(double* c, const int64_t* base, int s0, int s1, double* partials, double* fix,
                               cudaStream_t st);
// Renormalised kernels of listed sources on the (2R+1)^3 offset layout.
cudaError_t launch_read_kernels(const void* Q, Store store, const double* sigma, Grid g, int R,
                                const int64_t* sources, int64_t n_src, double* out, cudaStream_t st);

}  // namespace fdirw
