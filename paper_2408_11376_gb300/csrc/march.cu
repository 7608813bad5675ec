// Per-source windowed explicit FD march (Sec. 3.1: column s of p is the explicit-FD solution from a
// unit point source at s) and FP64 renormalisation of the stored kernel.
//
// Work decomposition (persistent grid, batches of SPB sources per CTA):
//   - one thread per z-column (ci, cj) of a source's (2R+1)^3 window; the column's 2R+1 cells live in
//     registers for the whole march;
//   - the FP32 path also keeps the 6 face coefficients of each cell in registers (they are constant over
//     the march), so a substep costs 1 MUL + 6 FMA + 1 ADD per cell; the z neighbours are in the same thread and
//     the x/y neighbours are read from a double-buffered shared-memory copy of every column (one
//     __syncthreads per substep);
//   - the FP64 path (the plain FP64 baseline) keeps u and the diagonal in registers and the face
//     coefficients in shared memory (FP64 registers would not fit), same exchange scheme;
//   - after the march each thread rounds its cells to the storage type, writes them into the
//     destination-indexed cache Q[o][s + o] and sums the stored values in FP64; a fixed-order block
//     reduction gives sigma_s = 1 / sum.
// Window cells outside the domain carry no coefficients, so they stay 0; faces leaving the window or
// the domain have coefficient 0 (zero flux).  Bound: FP32 pipe + shared-memory bandwidth (FP32 path),
// FP64 pipe (FP64 path).  HBM traffic is only the coefficient loads (L2-resident) and the cache writes.
#include "fdirw_internal.h"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

namespace fdirw {

namespace {

template <int R>
struct Shape {
    static constexpr int W1 = 2 * R + 1;
    static constexpr int COLS = W1 * W1;
    static constexpr int W = W1 * W1 * W1;
    static constexpr int SPB = (512 / COLS) > 0 ? (512 / COLS) : 1;
    // FP64 path: 2 exchange buffers + 3 face arrays of SPB*W doubles must fit in ~200 KB.
    static constexpr int SPB64_CAP = 200000 / (5 * W * 8);
    static constexpr int SPB64 = SPB64_CAP < 1 ? 1 : (SPB64_CAP < SPB ? SPB64_CAP : SPB);
    static constexpr int THREADS64 = ((SPB64 * COLS + 31) / 32) * 32;
};

// FP32 path thread mapping: P threads per window z-column, each owning KS consecutive cells.
template <int R, int P>
struct Map32 {
    static constexpr int W1 = 2 * R + 1;
    static constexpr int COLS = W1 * W1;
    static constexpr int KS = (W1 + P - 1) / P;
    static constexpr int TPS = P * COLS;                       // threads per source
    static constexpr int SPB = (512 / TPS) > 0 ? (512 / TPS) : 1;    // sources per CTA
    static constexpr int THREADS = ((SPB * TPS + 31) / 32) * 32;
    // Split mappings aim at ~1024 resident threads per SM; the single-column mapping needs the
    // registers of a whole SM for one CTA (6 coefficients + state per cell, 2R+1 cells per thread).
    static constexpr int MIN_BLOCKS = P == 1 ? 1 : ((1024 / THREADS) > 0 ? 1024 / THREADS : 1);
    static constexpr int BUF = SPB * COLS * W1;                // floats per exchange buffer
    static constexpr size_t SMEM = (size_t)((2 * BUF * 4 + 15) / 16) * 16 + (size_t)SPB * COLS * 8;
};

// Plane of the kernel cache for window cell (x, y, k) of a radius-R window: the cache is laid out for
// radius a.Rq >= R (offset o = (x - R, y - R, k - R), plane (ox + Rq) + Wq ((oy + Rq) + Wq (oz + Rq))).
__device__ __forceinline__ int64_t qplane(const MarchArgs& a, int R, int x, int y, int k) {
    const int Wq = 2 * a.Rq + 1, d = a.Rq - R;
    return (int64_t)(x + d) + (int64_t)Wq * ((y + d) + (int64_t)Wq * (k + d));
}

// Structure holding a source: its dimensions and first global cell (a batch concatenates structures;
// a single grid is structure 0 with base 0).  s becomes the source's index within its structure.
// qbase: first column of the structure in a destination-indexed cache (s_qbase, or base without it).
struct SrcLoc {
    int nx, ny, nz;
    int64_t base, qbase;
};
__device__ __forceinline__ SrcLoc locate(const MarchArgs& a, bool ok, int64_t& s) {
    SrcLoc L{a.g.nx, a.g.ny, a.g.nz, 0, 0};
    if (ok && a.nstruct > 0) {
        int lo = 0, hi = a.nstruct - 1;               // last structure whose first cell is <= s
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(a.s_base + mid) <= s) lo = mid; else hi = mid - 1;
        }
        const int4 d = __ldg(a.s_dims + lo);
        const int64_t b = __ldg(a.s_base + lo);
        L = SrcLoc{d.x, d.y, d.z, b, a.s_qbase ? __ldg(a.s_qbase + lo) : b};
        s -= L.base;
    }
    return L;
}

// Column of the kernel cache for a stored value: the destination cell (destination-indexed layout) or
// the source's position in the launch's source range (source-indexed layout of the radius buckets).
__device__ __forceinline__ int64_t qcol(const MarchArgs& a, int64_t dest, int64_t pos) {
    return a.src_major ? pos - a.src_begin : dest;
}

// Rounds v to the storage type, writes it to Q[idx] and returns the stored value widened to float
// (exact for every storage type).  Q == nullptr: round only.
__device__ __forceinline__ float put(void* Q, Store st, int64_t idx, float v) {
    if (st == Store::F32) {
        if (Q) reinterpret_cast<float*>(Q)[idx] = v;
        return v;
    } else if (st == Store::F16) {
        const __half h = __float2half_rn(v);
        if (Q) reinterpret_cast<__half*>(Q)[idx] = h;
        return __half2float(h);
    } else {
        const __nv_bfloat16 b = __float2bfloat16_rn(v);
        if (Q) reinterpret_cast<__nv_bfloat16*>(Q)[idx] = b;
        return __bfloat162float(b);
    }
}

// Stores the march's value for destination `dest` at `plane` (put), or, for a destination outside the
// streamed slab, only rounds it to the storage type (sigma still sums it).
__device__ __forceinline__ float store_q(const MarchArgs& a, int64_t plane, int64_t dest, int64_t pos, float v) {
    if (a.dest_hi > a.dest_lo) {
        if (dest < a.dest_lo || dest >= a.dest_hi) return put(nullptr, a.store, 0, v);
        dest -= a.dest_lo;
    }
    return put(a.Q, a.store, plane * a.q_stride + qcol(a, dest, pos), v);
}

// sigma_s = 1 / (sum of the per-column FP64 partials of slot) for every slot of the batch, fixed order:
// warp w takes slots w, w + nwarps, ...; lane l sums columns l, l + 32, ...; then a xor-butterfly.
template <int COLS, int SPB>
__device__ __forceinline__ void finish_sigma(const double* red, int64_t batch_first, int64_t src_end,
                                             const int64_t* list, double* sigma) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int slot = warp; slot < SPB; slot += nwarps) {
        double acc = 0.0;
        for (int c = lane; c < COLS; c += 32) acc += red[slot * COLS + c];
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        const int64_t s = batch_first + slot;
        if (lane == 0 && s < src_end) sigma[list ? list[s] : s] = acc > 0.0 ? 1.0 / acc : 0.0;
    }
}

template <int R, int P>
__global__ void __launch_bounds__(Map32<R, P>::THREADS, Map32<R, P>::MIN_BLOCKS) march_f32_kernel(MarchArgs a) {
    using M = Map32<R, P>;
    constexpr int W1 = M::W1, COLS = M::COLS, KS = M::KS, TPS = M::TPS, SPB = M::SPB, BUF = M::BUF;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* xbuf = reinterpret_cast<float*>(smem_raw);                                  // [2][SPB*COLS][W1]
    double* red = reinterpret_cast<double*>(smem_raw + ((2 * BUF * 4 + 15) / 16) * 16);  // [SPB*COLS]

    const int t = threadIdx.x;
    const bool active = t < SPB * TPS;
    const int slot = active ? t / TPS : 0;
    const int rr = active ? t - slot * TPS : 0;
    const int part = rr / COLS;
    const int col = rr - part * COLS;
    const int ci = col % W1, cj = col / W1;
    const int k0 = part * KS;                                  // first own cell of the column
    const int kn = (W1 - k0) < KS ? (W1 - k0) : KS;            // number of own cells
    const int64_t nbatch = (a.src_end - a.src_begin + SPB - 1) / SPB;

    const int base = (slot * COLS + col) * W1;
    const int xm = ci > 0 ? base - W1 : base;
    const int xp = ci < 2 * R ? base + W1 : base;
    const int ym = cj > 0 ? base - W1 * W1 : base;
    const int yp = cj < 2 * R ? base + W1 * W1 : base;
    const int kbelow = k0 > 0 ? k0 - 1 : k0;                   // cell read for the -z face of cell k0
    const int kabove = k0 + kn < W1 ? k0 + kn : k0;            // cell read for the +z face of the last cell

    for (int64_t b = blockIdx.x; b < nbatch; b += gridDim.x) {
        const int64_t first = a.src_begin + b * SPB;
        int64_t s = first + slot;
        const bool src_ok = active && s < a.src_end;
        if (src_ok && a.list) s = a.list[s];       // explicit source list (e.g. the surrogate's rejects)
        const int64_t pos = first + slot;                     // position of the source in the launch range
        const SrcLoc L = locate(a, src_ok, s);
        const int nx = L.nx, ny = L.ny, nz = L.nz;
        const int64_t nxy = (int64_t)nx * ny;
        const float* ax = a.ax + L.base;   // coefficients of the source's structure
        const float* ay = a.ay + L.base;
        const float* az = a.az + L.base;
        int sx = 0, sy = 0, sz = 0;
        if (src_ok) {
            sx = (int)(s % nx);
            const int64_t r = s / nx;
            sy = (int)(r % ny);
            sz = (int)(r / ny);
        }
        const int x = sx - R + ci, y = sy - R + cj;
        const bool col_ok = src_ok && x >= 0 && x < nx && y >= 0 && y < ny;

        // am = -(sum of the cell's face coefficients): the update is u += am*u + sum c*u_nb, i.e. the
        // increment is formed at full FP32 relative precision before it is added (1 - sum c rounded
        // once would bias near-delta kernels by half an ulp of 1 every substep).
        // cz[j] is the +z face of own cell j; czb is the -z face of own cell 0.
        float u[KS], am[KS], cxm[KS], cxp[KS], cym[KS], cyp[KS], cz[KS];
        float czb = 0.f;
#pragma unroll
        for (int j = 0; j < KS; j++) {
            const int k = k0 + j;
            const int z = sz - R + k;
            const bool ok = col_ok && j < kn && z >= 0 && z < nz;
            float vxm = 0.f, vxp = 0.f, vym = 0.f, vyp = 0.f, vz = 0.f;
            if (ok) {
                const int64_t i = (int64_t)x + (int64_t)nx * y + nxy * z;
                if (ci > 0 && x > 0) vxm = __ldg(ax + i - 1);
                if (ci < 2 * R && x + 1 < nx) vxp = __ldg(ax + i);
                if (cj > 0 && y > 0) vym = __ldg(ay + i - nx);
                if (cj < 2 * R && y + 1 < ny) vyp = __ldg(ay + i);
                if (k < 2 * R && z + 1 < nz) vz = __ldg(az + i);
                if (j == 0 && k > 0 && z > 0) czb = __ldg(az + i - nxy);
            }
            cxm[j] = vxm; cxp[j] = vxp; cym[j] = vym; cyp[j] = vyp; cz[j] = vz;
            u[j] = (src_ok && ci == R && cj == R && k == R) ? 1.f : 0.f;
        }
#pragma unroll
        for (int j = 0; j < KS; j++) {
            const float zm = j > 0 ? cz[j - 1] : czb;
            am[j] = -(((cxm[j] + cxp[j]) + (cym[j] + cyp[j])) + (zm + cz[j]));
        }

        for (int it = 0; it < a.n_sub; it++) {
            float* buf = xbuf + (it & 1) * BUF;
            if (active) {
#pragma unroll
                for (int j = 0; j < KS; j++)
                    if (j < kn) buf[base + k0 + j] = u[j];
            }
            __syncthreads();
            float prev = buf[base + kbelow];        // z-neighbour below own cell 0 (coefficient 0 if none)
            const float next_last = buf[base + kabove];
#pragma unroll
            for (int j = 0; j < KS; j++) {
                if (j < kn) {                      // the last part of a column may own fewer cells
                    const float cur = u[j];
                    const int k = k0 + j;
                    float v = am[j] * cur;
                    v = fmaf(cxm[j], buf[xm + k], v);
                    v = fmaf(cxp[j], buf[xp + k], v);
                    v = fmaf(cym[j], buf[ym + k], v);
                    v = fmaf(cyp[j], buf[yp + k], v);
                    v = fmaf(j > 0 ? cz[j - 1] : czb, prev, v);
                    v = fmaf(cz[j], (j + 1 < KS) ? (j + 1 < kn ? u[j + 1] : next_last) : next_last, v);
                    prev = cur;
                    u[j] = __fadd_rn(cur, v);
                }
            }
        }

        // Epilogue: round to storage and write Q[o][x] (x = s + o, the cell itself); the stored values
        // (exact in FP32) go back to shared memory so that each column is summed in k order by one
        // thread, whatever P is.
        float* sbuf = xbuf + (a.n_sub & 1) * BUF;   // not the buffer the last substep read
        if (active) {
#pragma unroll
            for (int j = 0; j < KS; j++) {
                if (j < kn) {
                    const int k = k0 + j;
                    const int z = sz - R + k;
                    float st = 0.f;
                    if (col_ok && z >= 0 && z < nz) {
                        const int64_t i = (int64_t)x + (int64_t)nx * y + nxy * z;
                        st = store_q(a, qplane(a, R, ci, cj, k), L.qbase + i, pos, u[j]);
                    }
                    sbuf[base + k] = st;
                }
            }
        }
        __syncthreads();
        for (int c = t; c < SPB * COLS; c += blockDim.x) {
            double colsum = 0.0;
#pragma unroll
            for (int k = 0; k < W1; k++) colsum += (double)sbuf[c * W1 + k];
            red[c] = colsum;
        }
        __syncthreads();
        finish_sigma<COLS, SPB>(red, first, a.src_end, a.list, a.sigma);
        __syncthreads();   // red and xbuf are reused by the next batch
    }
}

template <int R>
__global__ void __launch_bounds__(Shape<R>::THREADS64, 1) march_f64_kernel(MarchArgs a) {
    using S = Shape<R>;
    constexpr int W1 = S::W1, COLS = S::COLS, SPB = S::SPB64;
    constexpr int BUF = SPB * COLS * W1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* xbuf = reinterpret_cast<double*>(smem_raw);   // [2][BUF]
    double* fx = xbuf + 2 * BUF;                           // +x face coefficient of each window cell
    double* fy = fx + BUF;                                 // +y
    double* fz = fy + BUF;                                 // +z
    double* red = fz + BUF;                                // [SPB*COLS]

    const int t = threadIdx.x;
    const bool active = t < SPB * COLS;
    const int slot = active ? t / COLS : 0;
    const int col = active ? t - slot * COLS : 0;
    const int ci = col % W1, cj = col / W1;
    const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
    const int64_t nxy = (int64_t)nx * ny;
    const int64_t nbatch = (a.src_end - a.src_begin + SPB - 1) / SPB;

    const int base = (slot * COLS + col) * W1;
    const int xm = ci > 0 ? base - W1 : base;
    const int xp = ci < 2 * R ? base + W1 : base;
    const int ym = cj > 0 ? base - W1 * W1 : base;
    const int yp = cj < 2 * R ? base + W1 * W1 : base;

    for (int64_t b = blockIdx.x; b < nbatch; b += gridDim.x) {
        const int64_t first = a.src_begin + b * SPB;
        int64_t s = first + slot;
        const bool src_ok = active && s < a.src_end;
        if (src_ok && a.list) s = a.list[s];       // explicit source list (e.g. the surrogate's rejects)
        int sx = 0, sy = 0, sz = 0;
        if (src_ok) {
            sx = (int)(s % nx);
            const int64_t r = s / nx;
            sy = (int)(r % ny);
            sz = (int)(r / ny);
        }
        const int x = sx - R + ci, y = sy - R + cj;
        const bool col_ok = src_ok && x >= 0 && x < nx && y >= 0 && y < ny;

        double u[W1];
#pragma unroll
        for (int k = 0; k < W1; k++) {
            const int z = sz - R + k;
            const bool ok = col_ok && z >= 0 && z < nz;
            double vxp = 0.0, vyp = 0.0, vz = 0.0;
            if (ok) {
                const int64_t i = (int64_t)x + (int64_t)nx * y + nxy * z;
                if (ci < 2 * R && x + 1 < nx) vxp = __ldg(a.dx + i);
                if (cj < 2 * R && y + 1 < ny) vyp = __ldg(a.dy + i);
                if (k < 2 * R && z + 1 < nz) vz = __ldg(a.dz + i);
            }
            if (active) { fx[base + k] = vxp; fy[base + k] = vyp; fz[base + k] = vz; }
            u[k] = (src_ok && ci == R && cj == R && k == R) ? 1.0 : 0.0;
        }
        __syncthreads();
        double a0[W1];
#pragma unroll
        for (int k = 0; k < W1; k++) {
            const double vxm = ci > 0 ? fx[xm + k] : 0.0;
            const double vym = cj > 0 ? fy[ym + k] : 0.0;
            const double vzm = k > 0 ? fz[base + k - 1] : 0.0;
            a0[k] = 1.0 - (((vxm + fx[base + k]) + (vym + fy[base + k])) + (vzm + fz[base + k]));
        }

        for (int it = 0; it < a.n_sub; it++) {
            double* buf = xbuf + (it & 1) * BUF;
            if (active) {
#pragma unroll
                for (int k = 0; k < W1; k++) buf[base + k] = u[k];
            }
            __syncthreads();
            double prev = 0.0;
#pragma unroll
            for (int k = 0; k < W1; k++) {
                const double cur = u[k];
                double v = a0[k] * cur;
                if (ci > 0) v = fma(fx[xm + k], buf[xm + k], v);
                v = fma(fx[base + k], buf[xp + k], v);
                if (cj > 0) v = fma(fy[ym + k], buf[ym + k], v);
                v = fma(fy[base + k], buf[yp + k], v);
                if (k > 0) v = fma(fz[base + k - 1], prev, v);
                if (k + 1 < W1) v = fma(fz[base + k], u[k + 1], v);
                prev = cur;
                u[k] = v;
            }
        }

        double colsum = 0.0;
        if (col_ok) {
#pragma unroll
            for (int k = 0; k < W1; k++) {
                const int z = sz - R + k;
                if (z >= 0 && z < nz) {
                    const int64_t i = (int64_t)x + (int64_t)nx * y + nxy * z;
                    if (a.dest_hi <= a.dest_lo || (i >= a.dest_lo && i < a.dest_hi))
                        reinterpret_cast<double*>(a.Q)[qplane(a, R, ci, cj, k) * a.q_stride + (i - a.dest_lo)] = u[k];
                    colsum += u[k];
                }
            }
        }
        if (active) red[t] = colsum;
        __syncthreads();
        finish_sigma<COLS, SPB>(red, first, a.src_end, a.list, a.sigma);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------------------
// 2x2-block mapping with TMEM-resident coefficients (mapping id 4).
//
// Each thread owns a 2x2 block of window columns (4*(2R+1) cells, u in registers), so the halo it
// exchanges through shared memory per substep drops from 5 to 3 words per cell.  The 12 x/y face
// coefficients of a block level (and the 4 diagonals, while they fit) no longer fit in registers; they
// live in Tensor Memory, one TMEM lane per thread, and are streamed back level by level with
// tcgen05.ld while the previous level computes (TMEM is read at ~2.5x the shared-memory rate on GB300).
// The z faces and the remaining diagonals stay in registers.  The FP32 operations per cell and their
// order are the same as in march_f32_kernel, so the results are bitwise identical.
//
// One CTA of 256 threads per SM (two threads per TMEM lane, 256 columns each; the CTA allocates all 512
// columns once and frees them before it exits, and its shared-memory request keeps a second CTA off the
// SM so an allocation never waits).
// Where the stored values of one source of a CTA batch go (written by the source's first thread, read by
// every thread of the CTA in the epilogue).
struct SlotInfo {
    int64_t qbase, pos, nxy;
    int sx, sy, sz, nx, ny, nz, ok, pad;
};

template <int R>
struct MapTm {
    static constexpr int W1 = 2 * R + 1;
    static constexpr int COLS = W1 * W1;
    static constexpr int NB = R + 1;                      // blocks per window axis (last one half padding)
    static constexpr int TPS = NB * NB;                   // threads per source
    // R <= 8: 256 threads, two per TMEM lane (256 columns each); R = 9, 10: one source of 100 or 121
    // threads per CTA, one per lane, so that every level's 16 words fit its 512 columns.
    static constexpr int THREADS = TPS <= 81 ? 256 : 128;
    static constexpr int TCOLS = THREADS == 256 ? 256 : 512;   // TMEM columns per thread
    static constexpr int SPB = THREADS / TPS;
    static constexpr int LEVEL = 4 * THREADS;             // floats per level: [sub-column][thread]
    static constexpr int BUF = W1 * LEVEL;                // floats per exchange buffer
    static constexpr int LA0 = (TCOLS - 12 * W1) / 4;
    static constexpr int LA = LA0 < W1 ? LA0 : W1;        // levels whose diagonals live in TMEM
    static constexpr int NR = W1 - LA;                    // levels whose diagonals live in registers
    static constexpr size_t SMEM_USED = (size_t)2 * BUF * 4 + (size_t)SPB * COLS * 8 + (size_t)SPB * sizeof(SlotInfo);
    static constexpr size_t SMEM = SMEM_USED > 120 * 1024 ? SMEM_USED : 120 * 1024;
};

__device__ __forceinline__ void tm_st16(uint32_t a, const uint32_t (&v)[16]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
                 :: "r"(a), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
                    "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]) : "memory");
}
__device__ __forceinline__ void tm_st8(uint32_t a, const uint32_t* v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
                 :: "r"(a), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]) : "memory");
}
__device__ __forceinline__ void tm_st4(uint32_t a, const uint32_t* v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};"
                 :: "r"(a), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]) : "memory");
}
__device__ __forceinline__ void tm_ld16(uint32_t a, uint32_t (&r)[16]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(a));
}
__device__ __forceinline__ void tm_ld12(uint32_t a8, uint32_t a4, uint32_t (&r)[16]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(a8));
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]) : "r"(a4));
}
// Waits for every outstanding tcgen05.ld of the thread; the registers are in-out operands so that no
// use of them is scheduled before the wait.
__device__ __forceinline__ void tm_wait_ld(uint32_t (&r)[16]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
                 :: "memory");
}

// TMEM word offsets of a block level: levels < LA hold 16 words [12 faces, 4 diagonals] at 16k; the
// remaining levels hold their 12 faces as 8 words in region A and 4 words in region B (every access is
// aligned to its width).
template <int R>
__device__ __forceinline__ void tm_level_offsets(int k, uint32_t& o16, uint32_t& o8, uint32_t& o4) {
    using M = MapTm<R>;
    o16 = (uint32_t)(16 * k);
    o8 = (uint32_t)(16 * M::LA + 8 * (k - M::LA));
    o4 = (uint32_t)(16 * M::LA + 8 * M::NR + 4 * (k - M::LA));
}

template <int R>
__device__ __forceinline__ void tm_load_level(uint32_t tbase, int k, uint32_t (&r)[16]) {
    uint32_t o16, o8, o4;
    tm_level_offsets<R>(k, o16, o8, o4);
    if (k < MapTm<R>::LA) tm_ld16(tbase + o16, r);
    else tm_ld12(tbase + o8, tbase + o4, r);
}

template <int R>
__global__ void __launch_bounds__(MapTm<R>::THREADS, 1) march_tm_kernel(MarchArgs a) {
    using M = MapTm<R>;
    constexpr int W1 = M::W1, COLS = M::COLS, NB = M::NB, TPS = M::TPS, SPB = M::SPB;
    constexpr int LEVEL = M::LEVEL, PLANE = M::THREADS, BUF = M::BUF, LA = M::LA, NR = M::NR;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* xbuf = reinterpret_cast<float*>(smem_raw);                         // [2][W1][4][256]
    double* red = reinterpret_cast<double*>(smem_raw + (size_t)2 * BUF * 4);  // [SPB*COLS]
    SlotInfo* sinfo = reinterpret_cast<SlotInfo*>(red + SPB * COLS);           // [SPB]
    __shared__ uint32_t s_taddr;

    const int t = threadIdx.x;
    const int warp = t >> 5;
    if (warp == 0) {
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&s_taddr);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" :: "r"(dst) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = s_taddr;
    const uint32_t tbase = taddr + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(256 * (warp >> 2));

    const bool active = t < SPB * TPS;
    const int slot = active ? t / TPS : 0;
    const int b = active ? t - slot * TPS : 0;
    const int bi = b % NB, bj = b / NB;
    // Neighbour blocks; the own index at the window edge (the matching faces are 0) and for idle threads.
    const int tl = (active && bi > 0) ? t - 1 : t;
    const int tr = (active && bi < NB - 1) ? t + 1 : t;
    const int tb = (active && bj > 0) ? t - NB : t;
    const int tt = (active && bj < NB - 1) ? t + NB : t;
    const int64_t nbatch = (a.src_end - a.src_begin + SPB - 1) / SPB;

    for (int64_t bt = blockIdx.x; bt < nbatch; bt += gridDim.x) {
        const int64_t first = a.src_begin + bt * SPB;
        int64_t s = first + slot;
        const bool src_ok = active && s < a.src_end;
        if (src_ok && a.list) s = a.list[s];       // explicit source list (e.g. the surrogate's rejects)
        const int64_t pos = first + slot;                     // position of the source in the launch range
        const SrcLoc L = locate(a, src_ok, s);
        const int nx = L.nx, ny = L.ny, nz = L.nz;
        const int64_t nxy = (int64_t)nx * ny;
        const float* ax = a.ax + L.base;   // coefficients of the source's structure
        const float* ay = a.ay + L.base;
        const float* az = a.az + L.base;
        int sx = 0, sy = 0, sz = 0;
        if (src_ok) {
            sx = (int)(s % nx);
            const int64_t r = s / nx;
            sy = (int)(r % ny);
            sz = (int)(r / ny);
        }
        // Window cell (x, y, k) -> global cell; validity; face coefficients (0 outside window/domain).
        auto cell_ok = [&](int x, int y, int k) -> bool {
            const int gx = sx - R + x, gy = sy - R + y, gz = sz - R + k;
            return src_ok && x >= 0 && x < W1 && y >= 0 && y < W1 && k >= 0 && k < W1 &&
                   gx >= 0 && gx < nx && gy >= 0 && gy < ny && gz >= 0 && gz < nz;
        };
        auto gidx = [&](int x, int y, int k) -> int64_t {
            return (int64_t)(sx - R + x) + (int64_t)nx * (sy - R + y) + nxy * (sz - R + k);
        };
        auto xface = [&](int x, int y, int k) -> float {   // face between window x and x+1
            return (x + 1 < W1 && cell_ok(x, y, k) && sx - R + x + 1 < nx) ? __ldg(ax + gidx(x, y, k)) : 0.f;
        };
        auto yface = [&](int x, int y, int k) -> float {
            return (y + 1 < W1 && cell_ok(x, y, k) && sy - R + y + 1 < ny) ? __ldg(ay + gidx(x, y, k)) : 0.f;
        };
        auto zface = [&](int x, int y, int k) -> float {
            return (k + 1 < W1 && cell_ok(x, y, k) && sz - R + k + 1 < nz) ? __ldg(az + gidx(x, y, k)) : 0.f;
        };
        if (active && b == 0)
            sinfo[slot] = SlotInfo{L.qbase, pos, nxy, sx, sy, sz, nx, ny, nz, src_ok ? 1 : 0, 0};

        // Registers: state u[sub][k], z faces cz[sub][k] (+z face of the cell), diagonals of the levels
        // whose TMEM slot has no room for them.  Sub-column sc = sxb + 2*syb at window (2bi+sxb, 2bj+syb).
        float u[4][W1], cz[4][W1], amr[NR > 0 ? NR : 1][4];
#pragma unroll
        for (int sc = 0; sc < 4; sc++) {
            const int x = 2 * bi + (sc & 1), y = 2 * bj + (sc >> 1);
#pragma unroll
            for (int k = 0; k < W1; k++) {
                cz[sc][k] = zface(x, y, k);
                u[sc][k] = (src_ok && x == R && y == R && k == R) ? 1.f : 0.f;
            }
        }
#pragma unroll
        for (int k = 0; k < W1; k++) {
            // faces of the level: rows (syb) for x, columns (sxb) for y
            float f[16];
            const int x0 = 2 * bi, y0 = 2 * bj;
            f[0] = bi > 0 ? xface(x0 - 1, y0, k) : 0.f;       // L0
            f[1] = xface(x0, y0, k);                           // I0
            f[2] = xface(x0 + 1, y0, k);                       // R0
            f[3] = bi > 0 ? xface(x0 - 1, y0 + 1, k) : 0.f;   // L1
            f[4] = xface(x0, y0 + 1, k);                       // I1
            f[5] = xface(x0 + 1, y0 + 1, k);                   // R1
            f[6] = bj > 0 ? yface(x0, y0 - 1, k) : 0.f;       // B0
            f[7] = yface(x0, y0, k);                           // J0
            f[8] = yface(x0, y0 + 1, k);                       // T0
            f[9] = bj > 0 ? yface(x0 + 1, y0 - 1, k) : 0.f;   // B1
            f[10] = yface(x0 + 1, y0, k);                      // J1
            f[11] = yface(x0 + 1, y0 + 1, k);                  // T1
            // diagonals, same association as march_f32_kernel: -(((cxm+cxp)+(cym+cyp))+(czm+czp))
            const float cxm[4] = {f[0], f[1], f[3], f[4]}, cxp[4] = {f[1], f[2], f[4], f[5]};
            const float cym[4] = {f[6], f[9], f[7], f[10]}, cyp[4] = {f[7], f[10], f[8], f[11]};
#pragma unroll
            for (int sc = 0; sc < 4; sc++) {
                const float zm = k > 0 ? cz[sc][k - 1] : 0.f;
                f[12 + sc] = -(((cxm[sc] + cxp[sc]) + (cym[sc] + cyp[sc])) + (zm + cz[sc][k]));
            }
            uint32_t w[16];
#pragma unroll
            for (int q = 0; q < 16; q++) w[q] = __float_as_uint(f[q]);
            uint32_t o16, o8, o4;
            tm_level_offsets<R>(k, o16, o8, o4);
            if (k < LA) {
                tm_st16(tbase + o16, w);
            } else {
                tm_st8(tbase + o8, w);
                tm_st4(tbase + o4, w + 8);
#pragma unroll
                for (int sc = 0; sc < 4; sc++) amr[(k - LA) < NR ? k - LA : 0][sc] = f[12 + sc];
            }
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");

        #pragma unroll(R <= 8 ? 2 : 1)   // two substeps per iteration: no register copies at the back edge
        for (int it = 0; it < a.n_sub; it++) {
            float* buf = xbuf + (it & 1) * BUF;
            if (active) {
#pragma unroll
                for (int k = 0; k < W1; k++)
#pragma unroll
                    for (int sc = 0; sc < 4; sc++) buf[k * LEVEL + sc * PLANE + t] = u[sc][k];
            }
            __syncthreads();
            // cb[k & 1]: coefficients of level k (ready); cb[(k + 1) & 1]: level k+1, loaded while level k
            // computes (the loop is unrolled, so the two buffers are fixed registers and nothing is copied).
            uint32_t cb[2][16];
            tm_load_level<R>(tbase, 0, cb[0]);
            tm_wait_ld(cb[0]);
            float prev[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < W1; k++) {
                uint32_t (&cc)[16] = cb[k & 1];
                uint32_t (&cn)[16] = cb[(k + 1) & 1];
                if (k + 1 < W1) tm_load_level<R>(tbase, k + 1, cn);
                const float* lv = buf + k * LEVEL;
                const float l0 = lv[1 * PLANE + tl], l1 = lv[3 * PLANE + tl];
                const float r0 = lv[0 * PLANE + tr], r1 = lv[2 * PLANE + tr];
                const float b0 = lv[2 * PLANE + tb], b1 = lv[3 * PLANE + tb];
                const float t0 = lv[0 * PLANE + tt], t1 = lv[1 * PLANE + tt];
                float c[16];
#pragma unroll
                for (int q = 0; q < 16; q++) c[q] = __uint_as_float(cc[q]);
                const float cxm[4] = {c[0], c[1], c[3], c[4]}, cxp[4] = {c[1], c[2], c[4], c[5]};
                const float cym[4] = {c[6], c[9], c[7], c[10]}, cyp[4] = {c[7], c[10], c[8], c[11]};
                const float uxm[4] = {l0, u[0][k], l1, u[2][k]}, uxp[4] = {u[1][k], r0, u[3][k], r1};
                const float uym[4] = {b0, b1, u[0][k], u[1][k]}, uyp[4] = {u[2][k], u[3][k], t0, t1};
                float nu[4];
#pragma unroll
                for (int sc = 0; sc < 4; sc++) {
                    const float cur = u[sc][k];
                    const float am = k < LA ? c[12 + sc] : amr[(k - LA) >= 0 ? k - LA : 0][sc];
                    float v = am * cur;
                    v = fmaf(cxm[sc], uxm[sc], v);
                    v = fmaf(cxp[sc], uxp[sc], v);
                    v = fmaf(cym[sc], uym[sc], v);
                    v = fmaf(cyp[sc], uyp[sc], v);
                    v = fmaf(k > 0 ? cz[sc][k > 0 ? k - 1 : 0] : 0.f, prev[sc], v);
                    v = fmaf(cz[sc][k], k + 1 < W1 ? u[sc][k + 1 < W1 ? k + 1 : k] : 0.f, v);
                    nu[sc] = __fadd_rn(cur, v);
                }
#pragma unroll
                for (int sc = 0; sc < 4; sc++) { prev[sc] = u[sc][k]; u[sc][k] = nu[sc]; }
                if (k + 1 < W1) tm_wait_ld(cn);
            }
        }

        // Epilogue: round to the storage type, then per-column FP64 sums in k order (same order as
        // march_f32_kernel) and the cache stores.
        float* sbuf = xbuf + (a.n_sub & 1) * BUF;
        if (active) {
#pragma unroll
            for (int sc = 0; sc < 4; sc++) {
                const int x = 2 * bi + (sc & 1), y = 2 * bj + (sc >> 1);
#pragma unroll
                for (int k = 0; k < W1; k++) sbuf[k * LEVEL + sc * PLANE + t] = cell_ok(x, y, k) ? put(nullptr, a.store, 0, u[sc][k]) : 0.f;
            }
        }
        __syncthreads();
        // Stores with the batch's sources fastest: a cell's SPB sources have adjacent destinations in the
        // same plane, so one warp store covers about 32 / SPB cells instead of 32 planes.  The values are
        // already rounded, so storing rounds nothing further.
        for (int w = t; w < SPB * W1 * W1 * W1; w += blockDim.x) {
            const int sl = w % SPB, c3 = w / SPB;
            const int x = c3 % W1, y = (c3 / W1) % W1, k = c3 / (W1 * W1);
            const SlotInfo& si = sinfo[sl];
            const int gx = si.sx - R + x, gy = si.sy - R + y, gz = si.sz - R + k;
            if (!si.ok || gx < 0 || gx >= si.nx || gy < 0 || gy >= si.ny || gz < 0 || gz >= si.nz) continue;
            const float v = sbuf[k * LEVEL + ((x & 1) + 2 * (y & 1)) * PLANE + sl * TPS + (x >> 1) + NB * (y >> 1)];
            store_q(a, qplane(a, R, x, y, k), si.qbase + gx + (int64_t)si.nx * gy + si.nxy * gz, si.pos, v);
        }
        for (int c = t; c < SPB * COLS; c += blockDim.x) {
            const int sl = c / COLS, cc = c - sl * COLS;
            const int x = cc % W1, y = cc / W1;
            const int tt2 = sl * TPS + (x >> 1) + NB * (y >> 1);
            const int sc = (x & 1) + 2 * (y & 1);
            double colsum = 0.0;
#pragma unroll
            for (int k = 0; k < W1; k++) colsum += (double)sbuf[k * LEVEL + sc * PLANE + tt2];
            red[c] = colsum;
        }
        __syncthreads();
        finish_sigma<COLS, SPB>(red, first, a.src_end, a.list, a.sigma);
        __syncthreads();
    }

    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" :: "r"(taddr) : "memory");
}

template <int R>
cudaError_t launch_tm(const MarchArgs& a, int num_sms, cudaStream_t st) {
    using M = MapTm<R>;
    static_assert(M::SPB >= 1, "a source must fit one CTA");
    const int64_t nsrc = a.src_end - a.src_begin;
    if (nsrc <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(march_tm_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)M::SMEM);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, march_tm_kernel<R>, M::THREADS, M::SMEM);
    if (e != cudaSuccess) return e;
    if (per_sm != 1) return cudaErrorInvalidConfiguration;   // TMEM allocation assumes one CTA per SM
    const int64_t nbatch = (nsrc + M::SPB - 1) / M::SPB;
    const int64_t grid = nbatch < (int64_t)num_sms ? nbatch : (int64_t)num_sms;
    march_tm_kernel<R><<<(unsigned)grid, M::THREADS, M::SMEM, st>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------------
// Column pairs with TMEM-resident faces and diagonals (mapping id 7; any R <= 10, made for R = 9, 10).
//
// Each thread owns two x-adjacent window columns (2 (2R+1) cells; the last pair of a window row is half
// padding), so the halo it exchanges through shared memory per substep is 4 words per cell (its two new
// values, the outer x neighbours and the y neighbours of both columns) instead of 5.  The 7 lateral faces
// of a pair's level (3 x, 4 y) and its 2 diagonals live in the thread's TMEM lane (8 + 1 words, loaded one
// level ahead); u and the z faces stay in registers, which leaves room below the register cap of a
// 256-thread CTA at R = 10 (mapping 5 runs 448 threads there and spills under a 128-register cap).  One
// CTA of 256 threads per SM, two threads per TMEM lane; the FP32 operations and their order are those of
// march_f32_kernel, so the results are bitwise those of every other mapping.
template <int R>
struct MapTmx {
    static constexpr int W1 = 2 * R + 1;
    static constexpr int COLS = W1 * W1;
    static constexpr int NBX = R + 1;                     // column pairs per window row
    static constexpr int TPS = NBX * W1;                  // threads per source
    static constexpr int THREADS = 256;
    static constexpr int SPB = THREADS / TPS;
    static constexpr int LEVEL = 2 * THREADS;             // floats per level: [sub-column][thread]
    static constexpr int BUF = W1 * LEVEL;
    static constexpr size_t SMEM_USED = (size_t)2 * BUF * 4 + (size_t)SPB * COLS * 8;
    static constexpr size_t SMEM = SMEM_USED > 120 * 1024 ? SMEM_USED : 120 * 1024;
    static_assert(SPB >= 1 && 9 * W1 <= 256, "a source must fit a CTA and its coefficients 256 TMEM columns");
};

__device__ __forceinline__ void tm_st1(uint32_t a, uint32_t v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" :: "r"(a), "r"(v) : "memory");
}
// The 9 words of a pair's level: 8 at a8, 1 at a1.
__device__ __forceinline__ void tm_ld9(uint32_t a8, uint32_t a1, uint32_t (&r)[9]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(a8));
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r[8]) : "r"(a1));
}
__device__ __forceinline__ void tm_wait_ld9(uint32_t (&r)[9]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]) :: "memory");
}

template <int R>
__global__ void __launch_bounds__(MapTmx<R>::THREADS, 1) march_tmx_kernel(MarchArgs a) {
    using M = MapTmx<R>;
    constexpr int W1 = M::W1, COLS = M::COLS, NBX = M::NBX, TPS = M::TPS, SPB = M::SPB;
    constexpr int LEVEL = M::LEVEL, PLANE = M::THREADS, BUF = M::BUF;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* xbuf = reinterpret_cast<float*>(smem_raw);                         // [2][W1][2][256]
    double* red = reinterpret_cast<double*>(smem_raw + (size_t)2 * BUF * 4);  // [SPB*COLS]
    __shared__ uint32_t s_taddr;

    const int t = threadIdx.x;
    const int warp = t >> 5;
    if (warp == 0) {
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&s_taddr);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" :: "r"(dst) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = s_taddr;
    const uint32_t tbase = taddr + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(256 * (warp >> 2));
    const uint32_t regA = tbase, regB = tbase + (uint32_t)(8 * W1);      // level k: 8 words at 8k, 1 at 8 W1 + k

    const bool active = t < SPB * TPS;
    const int slot = active ? t / TPS : 0;
    const int b = active ? t - slot * TPS : 0;
    const int bi = b % NBX, bj = b / NBX;
    const int tl = (active && bi > 0) ? t - 1 : t;
    const int tr = (active && bi < NBX - 1) ? t + 1 : t;
    const int tb = (active && bj > 0) ? t - NBX : t;
    const int tt = (active && bj < W1 - 1) ? t + NBX : t;
    const int64_t nbatch = (a.src_end - a.src_begin + SPB - 1) / SPB;

    for (int64_t bt = blockIdx.x; bt < nbatch; bt += gridDim.x) {
        const int64_t first = a.src_begin + bt * SPB;
        int64_t s = first + slot;
        const bool src_ok = active && s < a.src_end;
        if (src_ok && a.list) s = a.list[s];
        const int64_t pos = first + slot;
        const SrcLoc L = locate(a, src_ok, s);
        const int nx = L.nx, ny = L.ny, nz = L.nz;
        const int64_t nxy = (int64_t)nx * ny;
        const float* ax = a.ax + L.base;
        const float* ay = a.ay + L.base;
        const float* az = a.az + L.base;
        int sx = 0, sy = 0, sz = 0;
        if (src_ok) {
            sx = (int)(s % nx);
            const int64_t r = s / nx;
            sy = (int)(r % ny);
            sz = (int)(r / ny);
        }
        auto cell_ok = [&](int x, int y, int k) -> bool {
            const int gx = sx - R + x, gy = sy - R + y, gz = sz - R + k;
            return src_ok && x >= 0 && x < W1 && y >= 0 && y < W1 && k >= 0 && k < W1 &&
                   gx >= 0 && gx < nx && gy >= 0 && gy < ny && gz >= 0 && gz < nz;
        };
        auto gidx = [&](int x, int y, int k) -> int64_t {
            return (int64_t)(sx - R + x) + (int64_t)nx * (sy - R + y) + nxy * (sz - R + k);
        };
        auto xface = [&](int x, int y, int k) -> float {
            return (x + 1 < W1 && cell_ok(x, y, k) && sx - R + x + 1 < nx) ? __ldg(ax + gidx(x, y, k)) : 0.f;
        };
        auto yface = [&](int x, int y, int k) -> float {
            return (y + 1 < W1 && cell_ok(x, y, k) && sy - R + y + 1 < ny) ? __ldg(ay + gidx(x, y, k)) : 0.f;
        };
        auto zface = [&](int x, int y, int k) -> float {
            return (k + 1 < W1 && cell_ok(x, y, k) && sz - R + k + 1 < nz) ? __ldg(az + gidx(x, y, k)) : 0.f;
        };

        // Sub-column sc at window (2 bi + sc, bj): state u[sc][k] and +z faces cz[sc][k] in registers.
        float u[2][W1], cz[2][W1];
#pragma unroll
        for (int sc = 0; sc < 2; sc++) {
            const int x = 2 * bi + sc, y = bj;
#pragma unroll
            for (int k = 0; k < W1; k++) {
                cz[sc][k] = zface(x, y, k);
                u[sc][k] = (src_ok && x == R && y == R && k == R) ? 1.f : 0.f;
            }
        }
#pragma unroll
        for (int k = 0; k < W1; k++) {
            const int x0 = 2 * bi, y = bj;
            float f[9];
            f[0] = bi > 0 ? xface(x0 - 1, y, k) : 0.f;        // -x face of sub-column 0
            f[1] = xface(x0, y, k);                            // between the two sub-columns
            f[2] = xface(x0 + 1, y, k);                        // +x face of sub-column 1
            f[3] = bj > 0 ? yface(x0, y - 1, k) : 0.f;        // -y face of sub-column 0
            f[4] = yface(x0, y, k);                            // +y face of sub-column 0
            f[5] = bj > 0 ? yface(x0 + 1, y - 1, k) : 0.f;    // -y face of sub-column 1
            f[6] = yface(x0 + 1, y, k);                        // +y face of sub-column 1
            // diagonals, same association as march_f32_kernel: -(((cxm+cxp)+(cym+cyp))+(czm+czp))
            f[7] = -(((f[0] + f[1]) + (f[3] + f[4])) + ((k > 0 ? cz[0][k > 0 ? k - 1 : 0] : 0.f) + cz[0][k]));
            f[8] = -(((f[1] + f[2]) + (f[5] + f[6])) + ((k > 0 ? cz[1][k > 0 ? k - 1 : 0] : 0.f) + cz[1][k]));
            uint32_t w[9];
#pragma unroll
            for (int q = 0; q < 9; q++) w[q] = __float_as_uint(f[q]);
            tm_st8(regA + (uint32_t)(8 * k), w);
            tm_st1(regB + (uint32_t)k, w[8]);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");

        #pragma unroll(2)   // two substeps per iteration: no register copies at the back edge
        for (int it = 0; it < a.n_sub; it++) {
            float* buf = xbuf + (it & 1) * BUF;
            if (active) {
#pragma unroll
                for (int k = 0; k < W1; k++)
#pragma unroll
                    for (int sc = 0; sc < 2; sc++) buf[k * LEVEL + sc * PLANE + t] = u[sc][k];
            }
            __syncthreads();
            uint32_t cb[2][9];
            tm_ld9(regA, regB, cb[0]);
            tm_wait_ld9(cb[0]);
            float prev[2] = {0.f, 0.f};
#pragma unroll
            for (int k = 0; k < W1; k++) {
                uint32_t (&cc)[9] = cb[k & 1];
                uint32_t (&cn)[9] = cb[(k + 1) & 1];
                if (k + 1 < W1) tm_ld9(regA + (uint32_t)(8 * (k + 1)), regB + (uint32_t)(k + 1), cn);
                const float* lv = buf + k * LEVEL;
                const float l = lv[1 * PLANE + tl], r = lv[0 * PLANE + tr];
                const float b0 = lv[0 * PLANE + tb], b1 = lv[1 * PLANE + tb];
                const float t0 = lv[0 * PLANE + tt], t1 = lv[1 * PLANE + tt];
                float c[9];
#pragma unroll
                for (int q = 0; q < 9; q++) c[q] = __uint_as_float(cc[q]);
                const float cxm[2] = {c[0], c[1]}, cxp[2] = {c[1], c[2]};
                const float cym[2] = {c[3], c[5]}, cyp[2] = {c[4], c[6]};
                const float amv[2] = {c[7], c[8]};
                const float uxm[2] = {l, u[0][k]}, uxp[2] = {u[1][k], r};
                const float uym[2] = {b0, b1}, uyp[2] = {t0, t1};
                float nu[2];
#pragma unroll
                for (int sc = 0; sc < 2; sc++) {
                    const float cur = u[sc][k];
                    float v = amv[sc] * cur;
                    v = fmaf(cxm[sc], uxm[sc], v);
                    v = fmaf(cxp[sc], uxp[sc], v);
                    v = fmaf(cym[sc], uym[sc], v);
                    v = fmaf(cyp[sc], uyp[sc], v);
                    v = fmaf(k > 0 ? cz[sc][k > 0 ? k - 1 : 0] : 0.f, prev[sc], v);
                    v = fmaf(cz[sc][k], k + 1 < W1 ? u[sc][k + 1 < W1 ? k + 1 : k] : 0.f, v);
                    nu[sc] = __fadd_rn(cur, v);
                }
#pragma unroll
                for (int sc = 0; sc < 2; sc++) { prev[sc] = u[sc][k]; u[sc][k] = nu[sc]; }
                if (k + 1 < W1) tm_wait_ld9(cn);
            }
        }

        // Epilogue: store, then per-column FP64 sums in k order (same order as march_f32_kernel).
        float* sbuf = xbuf + (a.n_sub & 1) * BUF;
        if (active) {
#pragma unroll
            for (int sc = 0; sc < 2; sc++) {
                const int x = 2 * bi + sc, y = bj;
#pragma unroll
                for (int k = 0; k < W1; k++) {
                    float stv = 0.f;
                    if (cell_ok(x, y, k)) stv = store_q(a, qplane(a, R, x, y, k), L.qbase + gidx(x, y, k), pos, u[sc][k]);
                    sbuf[k * LEVEL + sc * PLANE + t] = stv;
                }
            }
        }
        __syncthreads();
        for (int c = t; c < SPB * COLS; c += blockDim.x) {
            const int sl = c / COLS, cc = c - sl * COLS;
            const int x = cc % W1, y = cc / W1;
            const int tt2 = sl * TPS + (x >> 1) + NBX * y;
            const int sc = x & 1;
            double colsum = 0.0;
#pragma unroll
            for (int k = 0; k < W1; k++) colsum += (double)sbuf[k * LEVEL + sc * PLANE + tt2];
            red[c] = colsum;
        }
        __syncthreads();
        finish_sigma<COLS, SPB>(red, first, a.src_end, a.list, a.sigma);
        __syncthreads();
    }

    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" :: "r"(taddr) : "memory");
}

template <int R>
cudaError_t launch_tmx(const MarchArgs& a, int num_sms, cudaStream_t st) {
    using M = MapTmx<R>;
    const int64_t nsrc = a.src_end - a.src_begin;
    if (nsrc <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(march_tmx_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)M::SMEM);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, march_tmx_kernel<R>, M::THREADS, M::SMEM);
    if (e != cudaSuccess) return e;
    if (per_sm != 1) return cudaErrorInvalidConfiguration;   // TMEM allocation assumes one CTA per SM
    const int64_t nbatch = (nsrc + M::SPB - 1) / M::SPB;
    const int64_t grid = nbatch < (int64_t)num_sms ? nbatch : (int64_t)num_sms;
    march_tmx_kernel<R><<<(unsigned)grid, M::THREADS, M::SMEM, st>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------------
// One thread per window column with the lateral face coefficients in TMEM (mapping id 5; any R <= 10).
//
// For R = 9, 10 a column of 2R+1 cells with 6 coefficients each no longer fits in registers next to
// enough threads.  Here u, the diagonal and the z faces stay in registers and the 4 lateral faces of the
// column (4(2R+1) words) live in the thread's TMEM lane, in groups of 4 cells (16 words, one
// tcgen05.ld.32x32b.x16 each) fetched one group ahead of the compute.  Up to 4 threads share a TMEM lane
// (128 columns each), so one CTA of up to 448 threads per SM owns all 512 columns.  The halo exchange
// and the FP32 operations (and their order) are those of march_f32_kernel.
template <int R>
struct MapTmc {
    static constexpr int W1 = 2 * R + 1;
    static constexpr int COLS = W1 * W1;
    static constexpr int THREADS = ((COLS + 31) / 32) * 32;
    static constexpr int NG = (W1 + 3) / 4;               // TMEM groups of 4 cells
    static constexpr int BUF = COLS * W1;
    static constexpr size_t SMEM_USED = (size_t)((2 * BUF * 4 + 15) / 16) * 16 + (size_t)COLS * 8;
    static constexpr size_t SMEM = SMEM_USED > 120 * 1024 ? SMEM_USED : 120 * 1024;
    static_assert(16 * NG <= 128, "lateral faces of a column must fit a 128-column TMEM slot");
    static_assert(THREADS <= 512, "at most 4 threads per TMEM lane");
    // Coarse mode adds the per-block sums (at most W1^3 blocks in a window, plus the total).
    static constexpr size_t SMEM_COARSE_USED = SMEM_USED + (size_t)(W1 * W1 * W1 + 1) * 8;
    static constexpr size_t SMEM_COARSE = SMEM_COARSE_USED > SMEM ? SMEM_COARSE_USED : SMEM;
};

// Coarse epilogue (Eq. 11 applied to the marched unit of block J): S[d] = FP64 sum of the marched field
// over the liquid cells of block J + d inside the window (z, y, x order; sbuf holds 0 elsewhere), m =
// sum of S in a fixed order, and column J of P: Qc[d][J + d] = N_J S[d] / (m N_{J+d}), or S[d] / N_{J+d}
// when the phase has open faces (a.abnd) and the column keeps the mass that stays (0 where block J + d
// has no liquid).  Every thread of the CTA takes part; S follows red in shared memory.
template <int R>
__device__ void coarse_epilogue(const MarchArgs& a, const float* sbuf, double* S, int64_t first) {
    constexpr int W1 = 2 * R + 1;
    const bool valid = first < a.src_end;                 // uniform over the CTA
    const int64_t J = valid ? (a.list ? a.list[first] : first) : 0;
    const int B = a.coarse_B, Rc = a.coarse_Rc, Wc = 2 * Rc + 1, Wc3 = Wc * Wc * Wc, bh = (B - 1) / 2;
    const int bx = (int)(J % a.ncx), by = (int)((J / a.ncx) % a.ncy), bz = (int)(J / ((int64_t)a.ncx * a.ncy));
    const int sx = bx * B + bh, sy = by * B + bh, sz = bz * B + bh;
    const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
    for (int d = threadIdx.x; d < Wc3; d += blockDim.x) {
        double acc = 0.0;
        if (valid) {
            const int cx = bx + d % Wc - Rc, cy = by + (d / Wc) % Wc - Rc, cz = bz + d / (Wc * Wc) - Rc;
            const int x0 = max(max(cx * B, sx - R), 0), x1 = min(min(cx * B + B - 1, sx + R), nx - 1);
            const int y0 = max(max(cy * B, sy - R), 0), y1 = min(min(cy * B + B - 1, sy + R), ny - 1);
            const int z0 = max(max(cz * B, sz - R), 0), z1 = min(min(cz * B + B - 1, sz + R), nz - 1);
            for (int z = z0; z <= z1; z++)
                for (int y = y0; y <= y1; y++)
                    for (int x = x0; x <= x1; x++)
                        acc += (double)sbuf[((x - (sx - R)) + W1 * (y - (sy - R))) * W1 + (z - (sz - R))];
        }
        S[d] = acc;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        double m = 0.0;
        for (int d = threadIdx.x; d < Wc3; d += 32) m += S[d];
        for (int off = 16; off > 0; off >>= 1) m += __shfl_xor_sync(0xffffffffu, m, off);
        if (threadIdx.x == 0) S[Wc3] = m;
    }
    __syncthreads();
    const double m = S[Wc3];
    if (valid) {
        const double NJ = (double)a.ccount[J];
        for (int d = threadIdx.x; d < Wc3; d += blockDim.x) {
            const int cx = bx + d % Wc - Rc, cy = by + (d / Wc) % Wc - Rc, cz = bz + d / (Wc * Wc) - Rc;
            if (cx < 0 || cx >= a.ncx || cy < 0 || cy >= a.ncy || cz < 0 || cz >= a.ncz) continue;
            const int64_t I = cx + (int64_t)a.ncx * (cy + (int64_t)a.ncy * cz);
            const int NI = a.ccount[I];
            // Closed phase: renormalise the column to carry N_J; open faces: keep the mass that stays.
            double v = 0.0;
            if (NI > 0 && m > 0.0) v = a.abnd ? S[d] / (double)NI : (NJ * S[d]) / (m * (double)NI);
            a.Qc[(int64_t)d * a.coarse_n + I] = v;
        }
    }
}

// COARSE: the source is coarse block a.list[pos] (Eqs. 10-15): its window is centred on the block's
// centre cell (radius R = window_R + (B - 1) / 2), the march starts from 1 on the block's liquid cells,
// and the epilogue maps the marched field onto the blocks of the window (column J of the coarse matrix,
// written destination-indexed) instead of storing a kernel.
// ADV: the face coefficients differ by direction (convection): a.ax/ay/az hold the coefficient of the
// lower cell in the upper cell's update and a.bx/by/bz that of the upper cell in the lower one's; the
// diagonal is minus the sum of the cell's outflow coefficients.  Without ADV both are a.ax/ay/az.
template <int R, bool COARSE, bool ADV>
__global__ void __launch_bounds__(MapTmc<R>::THREADS, 1) march_tmc_kernel(MarchArgs a) {
    using M = MapTmc<R>;
    constexpr int W1 = M::W1, COLS = M::COLS, NG = M::NG, BUF = M::BUF;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* xbuf = reinterpret_cast<float*>(smem_raw);                                  // [2][COLS][W1]
    double* red = reinterpret_cast<double*>(smem_raw + ((2 * BUF * 4 + 15) / 16) * 16);  // [COLS]
    __shared__ uint32_t s_taddr;

    const int t = threadIdx.x, warp = t >> 5;
    if (warp == 0) {
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&s_taddr);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" :: "r"(dst) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = s_taddr;
    const uint32_t tbase = taddr + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(128 * (warp >> 2));

    const bool active = t < COLS;
    const int col = active ? t : 0;
    const int ci = col % W1, cj = col / W1;
    const int64_t nbatch = a.src_end - a.src_begin;
    const int base = col * W1;
    const int xm = ci > 0 ? base - W1 : base;
    const int xp = ci < 2 * R ? base + W1 : base;
    const int ym = cj > 0 ? base - W1 * W1 : base;
    const int yp = cj < 2 * R ? base + W1 * W1 : base;

    for (int64_t b = blockIdx.x; b < nbatch; b += gridDim.x) {
        const int64_t first = a.src_begin + b;
        int64_t s = first;
        const bool src_ok = active && s < a.src_end;
        if (src_ok && a.list) s = a.list[s];
        const int64_t pos = first;                     // position of the source in the launch range
        const SrcLoc L = locate(a, src_ok, s);
        const int nx = L.nx, ny = L.ny, nz = L.nz;
        const int64_t nxy = (int64_t)nx * ny;
        const float* ax = a.ax + L.base;   // coefficients of the source's structure
        const float* ay = a.ay + L.base;
        const float* az = a.az + L.base;
        int sx = 0, sy = 0, sz = 0;
        int bx = 0, by = 0, bz = 0;
        const int bh = COARSE ? (a.coarse_B - 1) / 2 : 0;
        if (src_ok) {
            if constexpr (COARSE) {
                bx = (int)(s % a.ncx);
                by = (int)((s / a.ncx) % a.ncy);
                bz = (int)(s / ((int64_t)a.ncx * a.ncy));
                sx = bx * a.coarse_B + bh;       // centre of the block (may lie past a clipped domain edge)
                sy = by * a.coarse_B + bh;
                sz = bz * a.coarse_B + bh;
            } else {
                sx = (int)(s % nx);
                const int64_t r = s / nx;
                sy = (int)(r % ny);
                sz = (int)(r / ny);
            }
        }
        const int x = sx - R + ci, y = sy - R + cj;
        const bool col_ok = src_ok && x >= 0 && x < nx && y >= 0 && y < ny;

        float u[W1], am[W1], cz[W1];
        float czb[ADV ? W1 : 1];              // ADV: coefficient of the upper z neighbour (cz: of the lower)
        float zprev = 0.f, zprevb = 0.f;
        const float* bxp = ADV ? a.bx + L.base : nullptr;
        const float* byp = ADV ? a.by + L.base : nullptr;
        const float* bzp = ADV ? a.bz + L.base : nullptr;
#pragma unroll
        for (int g = 0; g < NG; g++) {
            uint32_t w[16];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int k = 4 * g + q;
                float vxm = 0.f, vxp = 0.f, vym = 0.f, vyp = 0.f, vz = 0.f;
                float oxm = 0.f, oxp = 0.f, oym = 0.f, oyp = 0.f, vzb = 0.f;   // ADV: outflows, upper-z inflow
                if (k < W1) {
                    const int z = sz - R + k;
                    const bool ok = col_ok && z >= 0 && z < nz;
                    float u0 = (!COARSE && src_ok && ci == R && cj == R && k == R) ? 1.f : 0.f;
                    float vb = 0.f;                       // open faces of the cell (coarse, far field)
                    if (ok) {
                        const int64_t i = (int64_t)x + (int64_t)nx * y + nxy * z;
                        if (COARSE && a.liquid[i] && abs(ci - R) <= bh && abs(cj - R) <= bh && abs(k - R) <= bh) u0 = 1.f;
                        if (COARSE && a.abnd) vb = __ldg(a.abnd + i);
                        if (ci > 0 && x > 0) vxm = __ldg(ax + i - 1);
                        if (ci < 2 * R && x + 1 < nx) vxp = __ldg(ADV ? bxp + i : ax + i);
                        if (cj > 0 && y > 0) vym = __ldg(ay + i - nx);
                        if (cj < 2 * R && y + 1 < ny) vyp = __ldg(ADV ? byp + i : ay + i);
                        if (k < 2 * R && z + 1 < nz) vz = __ldg(az + i);
                        if constexpr (ADV) {
                            if (ci > 0 && x > 0) oxm = __ldg(bxp + i - 1);
                            if (ci < 2 * R && x + 1 < nx) oxp = __ldg(ax + i);
                            if (cj > 0 && y > 0) oym = __ldg(byp + i - nx);
                            if (cj < 2 * R && y + 1 < ny) oyp = __ldg(ay + i);
                            if (k < 2 * R && z + 1 < nz) vzb = __ldg(bzp + i);
                        }
                    }
                    cz[k < W1 ? k : 0] = vz;
                    if constexpr (ADV) {
                        // outflow through the -z face: the lower cell's upper-z inflow coefficient
                        czb[k < W1 ? k : 0] = vzb;
                        const float diag = ((oxm + oxp) + (oym + oyp)) + (zprevb + vz);
                        am[k < W1 ? k : 0] = COARSE ? -(diag + vb) : -diag;
                        zprevb = vzb;
                    } else if constexpr (COARSE) {
                        am[k < W1 ? k : 0] = -((((vxm + vxp) + (vym + vyp)) + (zprev + vz)) + vb);
                    } else {
                        am[k < W1 ? k : 0] = -(((vxm + vxp) + (vym + vyp)) + (zprev + vz));
                    }
                    u[k < W1 ? k : 0] = u0;
                    zprev = vz;
                }
                w[4 * q + 0] = __float_as_uint(vxm);
                w[4 * q + 1] = __float_as_uint(vxp);
                w[4 * q + 2] = __float_as_uint(vym);
                w[4 * q + 3] = __float_as_uint(vyp);
            }
            tm_st16(tbase + (uint32_t)(16 * g), w);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");

        for (int it = 0; it < a.n_sub; it++) {
            float* buf = xbuf + (it & 1) * BUF;
            if (active) {
#pragma unroll
                for (int k = 0; k < W1; k++) buf[base + k] = u[k];
            }
            __syncthreads();
            uint32_t cb[2][16];                        // group g in cb[g & 1], g + 1 loading into the other
            tm_ld16(tbase, cb[0]);
            tm_wait_ld(cb[0]);
            float prev = 0.f;
#pragma unroll
            for (int g = 0; g < NG; g++) {
                uint32_t (&cc)[16] = cb[g & 1];
                uint32_t (&cn)[16] = cb[(g + 1) & 1];
                if (g + 1 < NG) tm_ld16(tbase + (uint32_t)(16 * (g + 1)), cn);
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const int k = 4 * g + q;
                    if (k < W1) {
                        const float cxm = __uint_as_float(cc[4 * q + 0]), cxp = __uint_as_float(cc[4 * q + 1]);
                        const float cym = __uint_as_float(cc[4 * q + 2]), cyp = __uint_as_float(cc[4 * q + 3]);
                        const float cur = u[k];
                        float v = am[k] * cur;
                        v = fmaf(cxm, buf[xm + k], v);
                        v = fmaf(cxp, buf[xp + k], v);
                        v = fmaf(cym, buf[ym + k], v);
                        v = fmaf(cyp, buf[yp + k], v);
                        v = fmaf(k > 0 ? cz[k > 0 ? k - 1 : 0] : 0.f, prev, v);
                        v = fmaf(ADV ? czb[ADV ? k : 0] : cz[k], k + 1 < W1 ? u[k + 1 < W1 ? k + 1 : k] : 0.f, v);
                        prev = cur;
                        u[k] = __fadd_rn(cur, v);
                    }
                }
                if (g + 1 < NG) tm_wait_ld(cn);
            }
        }

        float* sbuf = xbuf + (a.n_sub & 1) * BUF;
        if constexpr (COARSE) {
            if (active) {
#pragma unroll
                for (int k = 0; k < W1; k++) {
                    const int z = sz - R + k;
                    const bool ok = col_ok && z >= 0 && z < nz && a.liquid[(int64_t)x + (int64_t)nx * y + nxy * z];
                    sbuf[base + k] = ok ? u[k] : 0.f;
                }
            }
            __syncthreads();
            coarse_epilogue<R>(a, sbuf, red + COLS, first);
        } else {
            if (active) {
#pragma unroll
                for (int k = 0; k < W1; k++) {
                    const int z = sz - R + k;
                    float stv = 0.f;
                    if (col_ok && z >= 0 && z < nz) {
                        const int64_t i = (int64_t)x + (int64_t)nx * y + nxy * z;
                        stv = store_q(a, qplane(a, R, ci, cj, k), L.qbase + i, pos, u[k]);
                    }
                    sbuf[base + k] = stv;
                }
            }
            __syncthreads();
            for (int c = t; c < COLS; c += blockDim.x) {
                double colsum = 0.0;
#pragma unroll
                for (int k = 0; k < W1; k++) colsum += (double)sbuf[c * W1 + k];
                red[c] = colsum;
            }
            __syncthreads();
            finish_sigma<COLS, 1>(red, first, a.src_end, a.list, a.sigma);
        }
        __syncthreads();
    }

    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" :: "r"(taddr) : "memory");
}

template <int R, bool COARSE = false, bool ADV = false>
cudaError_t launch_tmc(const MarchArgs& a, int num_sms, cudaStream_t st) {
    using M = MapTmc<R>;
    const int64_t nsrc = a.src_end - a.src_begin;
    if (nsrc <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(march_tmc_kernel<R, COARSE, ADV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(COARSE ? M::SMEM_COARSE : M::SMEM));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, march_tmc_kernel<R, COARSE, ADV>, M::THREADS, (COARSE ? M::SMEM_COARSE : M::SMEM));
    if (e != cudaSuccess) return e;
    if (per_sm != 1) return cudaErrorInvalidConfiguration;   // TMEM allocation assumes one CTA per SM
    const int64_t grid = nsrc < (int64_t)num_sms ? nsrc : (int64_t)num_sms;
    march_tmc_kernel<R, COARSE, ADV><<<(unsigned)grid, M::THREADS, (COARSE ? M::SMEM_COARSE : M::SMEM), st>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------------
// Mapping 6: one window column per thread for a PAIR of sources, every FP32 operation packed (f32x2).
//
// The two sources of a pair have the same window shape, so each thread marches the same column of
// both: the state, the diagonals and the z faces are register pairs (source A in the low half, B in
// the high half), the exchange buffer holds one 8-byte pair per cell, and the four lateral faces of
// both sources live in TMEM as aligned pairs (8 words per cell, 2 cells per 16-word load).  Each
// packed mul.rn / fma.rn / add.rn.f32x2 rounds each half exactly like the scalar instruction, and the
// operations come in the order of march_f32_kernel, so the kernels are bitwise those of mappings 1-5.
// Per cell-substep of a pair: 1 store + 4 loads of 8 bytes and 8 packed FP32 instructions.
template <int R>
struct MapTmp {
    static constexpr int W1 = 2 * R + 1;
    static constexpr int COLS = W1 * W1;
    static constexpr int PAIRS = (384 / COLS) > 0 ? (384 / COLS) : 1;   // source pairs per CTA
    static constexpr int THREADS = ((PAIRS * COLS + 31) / 32) * 32;
    static constexpr int SLOTS = (THREADS / 32 + 3) / 4;                // threads per TMEM lane
    static constexpr int SLOT_COLS = (512 / SLOTS) / 16 * 16;           // TMEM columns per thread
    static constexpr int NG = (W1 + 1) / 2;                             // 16-word groups of 2 cells
    static constexpr int BUF = PAIRS * COLS * W1;                       // 8-byte pairs per buffer
    static constexpr size_t SMEM_USED = (size_t)2 * BUF * 8 + (size_t)2 * PAIRS * COLS * 8;
    static constexpr size_t SMEM = SMEM_USED > 120 * 1024 ? SMEM_USED : 120 * 1024;
    static_assert(16 * NG <= SLOT_COLS, "the lateral faces of a column pair must fit the thread's TMEM slot");
    static_assert(R <= 8, "mapping 6 covers R <= 8");
};

__device__ __forceinline__ uint64_t f2pack(float lo, float hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ uint64_t u2pack(uint32_t lo, uint32_t hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "r"(lo), "r"(hi));
    return r;
}
__device__ __forceinline__ float f2lo(uint64_t v) { return __uint_as_float((uint32_t)(v & 0xffffffffull)); }
__device__ __forceinline__ float f2hi(uint64_t v) { return __uint_as_float((uint32_t)(v >> 32)); }
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

template <int R>
__global__ void __launch_bounds__(MapTmp<R>::THREADS, 1) march_tmp_kernel(MarchArgs a) {
    using M = MapTmp<R>;
    constexpr int W1 = M::W1, COLS = M::COLS, NG = M::NG, BUF = M::BUF, PAIRS = M::PAIRS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t* xbuf = reinterpret_cast<uint64_t*>(smem_raw);                        // [2][PAIRS*COLS][W1]
    double* red = reinterpret_cast<double*>(smem_raw + (size_t)2 * BUF * 8);      // [2*PAIRS][COLS]
    __shared__ uint32_t s_taddr;

    const int t = threadIdx.x, warp = t >> 5;
    if (warp == 0) {
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&s_taddr);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" :: "r"(dst) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = s_taddr;
    const uint32_t tbase = taddr + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(M::SLOT_COLS * (warp >> 2));

    const bool active = t < PAIRS * COLS;
    const int pair = active ? t / COLS : 0;
    const int col = active ? t - pair * COLS : 0;
    const int ci = col % W1, cj = col / W1;
    const int64_t nbatch = (a.src_end - a.src_begin + 2 * PAIRS - 1) / (2 * PAIRS);
    const int base = (pair * COLS + col) * W1;
    const int xm = ci > 0 ? base - W1 : base;
    const int xp = ci < 2 * R ? base + W1 : base;
    const int ym = cj > 0 ? base - W1 * W1 : base;
    const int yp = cj < 2 * R ? base + W1 * W1 : base;

    for (int64_t b = blockIdx.x; b < nbatch; b += gridDim.x) {
        const int64_t first = a.src_begin + b * 2 * PAIRS;
        // Per source of the pair (h = 0: low half, h = 1: high half): geometry and validity.
        int64_t pos[2], sidx[2];
        bool src_ok[2], col_ok[2];
        int sx[2], sy[2], sz[2], xs[2], ys[2], nzs[2], nxs[2], nys[2];
        int64_t nxy[2], cbase[2], qb[2];
#pragma unroll
        for (int h = 0; h < 2; h++) {
            pos[h] = first + 2 * pair + h;
            src_ok[h] = active && pos[h] < a.src_end;
            int64_t s = pos[h];
            if (src_ok[h] && a.list) s = a.list[s];
            const SrcLoc L = locate(a, src_ok[h], s);
            nxs[h] = L.nx; nys[h] = L.ny; nzs[h] = L.nz;
            nxy[h] = (int64_t)L.nx * L.ny;
            cbase[h] = L.base;
            qb[h] = L.qbase;
            sidx[h] = s;
            sx[h] = sy[h] = sz[h] = 0;
            if (src_ok[h]) {
                sx[h] = (int)(s % L.nx);
                const int64_t r = s / L.nx;
                sy[h] = (int)(r % L.ny);
                sz[h] = (int)(r / L.ny);
            }
            xs[h] = sx[h] - R + ci;
            ys[h] = sy[h] - R + cj;
            col_ok[h] = src_ok[h] && xs[h] >= 0 && xs[h] < L.nx && ys[h] >= 0 && ys[h] < L.ny;
        }

        uint64_t u[W1], am[W1], cz[W1];
        float zprev[2] = {0.f, 0.f};
#pragma unroll
        for (int g = 0; g < NG; g++) {
            uint32_t w[16];
#pragma unroll
            for (int q = 0; q < 2; q++) {
                const int k = 2 * g + q;
                float f[2][5] = {{0.f, 0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f, 0.f}};   // xm xp ym yp z+
                if (k < W1) {
                    float amv[2], uv[2];
#pragma unroll
                    for (int h = 0; h < 2; h++) {
                        const int z = sz[h] - R + k;
                        const bool ok = col_ok[h] && z >= 0 && z < nzs[h];
                        if (ok) {
                            const int64_t i = cbase[h] + (int64_t)xs[h] + (int64_t)nxs[h] * ys[h] + nxy[h] * z;
                            if (ci > 0 && xs[h] > 0) f[h][0] = __ldg(a.ax + i - 1);
                            if (ci < 2 * R && xs[h] + 1 < nxs[h]) f[h][1] = __ldg(a.ax + i);
                            if (cj > 0 && ys[h] > 0) f[h][2] = __ldg(a.ay + i - nxs[h]);
                            if (cj < 2 * R && ys[h] + 1 < nys[h]) f[h][3] = __ldg(a.ay + i);
                            if (k < 2 * R && z + 1 < nzs[h]) f[h][4] = __ldg(a.az + i);
                        }
                        amv[h] = -(((f[h][0] + f[h][1]) + (f[h][2] + f[h][3])) + (zprev[h] + f[h][4]));
                        uv[h] = (src_ok[h] && ci == R && cj == R && k == R) ? 1.f : 0.f;
                        zprev[h] = f[h][4];
                    }
                    const int kk = k < W1 ? k : 0;
                    cz[kk] = f2pack(f[0][4], f[1][4]);
                    am[kk] = f2pack(amv[0], amv[1]);
                    u[kk] = f2pack(uv[0], uv[1]);
                }
#pragma unroll
                for (int d = 0; d < 4; d++) {
                    w[8 * q + 2 * d] = __float_as_uint(f[0][d]);
                    w[8 * q + 2 * d + 1] = __float_as_uint(f[1][d]);
                }
            }
            tm_st16(tbase + (uint32_t)(16 * g), w);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");

        for (int it = 0; it < a.n_sub; it++) {
            uint64_t* buf = xbuf + (it & 1) * BUF;
            if (active) {
#pragma unroll
                for (int k = 0; k < W1; k++) buf[base + k] = u[k];
            }
            __syncthreads();
            uint32_t cb[2][16];
            tm_ld16(tbase, cb[0]);
            tm_wait_ld(cb[0]);
            uint64_t prev = 0ull;
#pragma unroll
            for (int g = 0; g < NG; g++) {
                uint32_t (&cc)[16] = cb[g & 1];
                uint32_t (&cn)[16] = cb[(g + 1) & 1];
                if (g + 1 < NG) tm_ld16(tbase + (uint32_t)(16 * (g + 1)), cn);
#pragma unroll
                for (int q = 0; q < 2; q++) {
                    const int k = 2 * g + q;
                    if (k < W1) {
                        const uint64_t cur = u[k];
                        uint64_t v = mul2(am[k], cur);
                        v = fma2(u2pack(cc[8 * q + 0], cc[8 * q + 1]), buf[xm + k], v);
                        v = fma2(u2pack(cc[8 * q + 2], cc[8 * q + 3]), buf[xp + k], v);
                        v = fma2(u2pack(cc[8 * q + 4], cc[8 * q + 5]), buf[ym + k], v);
                        v = fma2(u2pack(cc[8 * q + 6], cc[8 * q + 7]), buf[yp + k], v);
                        v = fma2(k > 0 ? cz[k > 0 ? k - 1 : 0] : 0ull, prev, v);
                        v = fma2(cz[k], k + 1 < W1 ? u[k + 1 < W1 ? k + 1 : k] : 0ull, v);
                        prev = cur;
                        u[k] = add2(cur, v);
                    }
                }
                if (g + 1 < NG) tm_wait_ld(cn);
            }
        }

        uint64_t* sbuf = xbuf + (a.n_sub & 1) * BUF;
        if (active) {
#pragma unroll
            for (int k = 0; k < W1; k++) {
                float stv[2];
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const int z = sz[h] - R + k;
                    stv[h] = 0.f;
                    if (col_ok[h] && z >= 0 && z < nzs[h]) {
                        const int64_t i = (int64_t)xs[h] + (int64_t)nxs[h] * ys[h] + nxy[h] * z;
                        stv[h] = store_q(a, qplane(a, R, ci, cj, k), qb[h] + i, pos[h], h == 0 ? f2lo(u[k]) : f2hi(u[k]));
                    }
                }
                sbuf[base + k] = f2pack(stv[0], stv[1]);
            }
        }
        __syncthreads();
        for (int c = t; c < PAIRS * COLS; c += blockDim.x) {
            const int pr = c / COLS, cl = c - pr * COLS;
            double s0 = 0.0, s1 = 0.0;
#pragma unroll
            for (int k = 0; k < W1; k++) {
                const uint64_t v = sbuf[c * W1 + k];
                s0 += (double)f2lo(v);
                s1 += (double)f2hi(v);
            }
            red[(2 * pr) * COLS + cl] = s0;
            red[(2 * pr + 1) * COLS + cl] = s1;
        }
        __syncthreads();
        finish_sigma<COLS, 2 * PAIRS>(red, first, a.src_end, a.list, a.sigma);
        __syncthreads();
    }

    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" :: "r"(taddr) : "memory");
}

template <int R>
cudaError_t launch_tmp(const MarchArgs& a, int num_sms, cudaStream_t st) {
    using M = MapTmp<R>;
    const int64_t nsrc = a.src_end - a.src_begin;
    if (nsrc <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(march_tmp_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)M::SMEM);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, march_tmp_kernel<R>, M::THREADS, M::SMEM);
    if (e != cudaSuccess) return e;
    if (per_sm != 1) return cudaErrorInvalidConfiguration;   // TMEM allocation assumes one CTA per SM
    const int64_t nbatch = (nsrc + 2 * M::PAIRS - 1) / (2 * M::PAIRS);
    const int64_t grid = nbatch < (int64_t)num_sms ? nbatch : (int64_t)num_sms;
    march_tmp_kernel<R><<<(unsigned)grid, M::THREADS, M::SMEM, st>>>(a);
    return cudaGetLastError();
}

template <int R, int P>
cudaError_t launch_f32(const MarchArgs& a, int num_sms, cudaStream_t st) {
    using M = Map32<R, P>;
    const int64_t nsrc = a.src_end - a.src_begin;
    if (nsrc <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(march_f32_kernel<R, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)M::SMEM);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, march_f32_kernel<R, P>, M::THREADS, M::SMEM);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int64_t nbatch = (nsrc + M::SPB - 1) / M::SPB;
    const int64_t grid = nbatch < (int64_t)num_sms * per_sm ? nbatch : (int64_t)num_sms * per_sm;
    march_f32_kernel<R, P><<<(unsigned)grid, M::THREADS, M::SMEM, st>>>(a);
    return cudaGetLastError();
}

template <int R>
cudaError_t launch_f32_p(const MarchArgs& a, int P, int num_sms, cudaStream_t st) {
    switch (P) {
        case 1: return launch_f32<R, 1>(a, num_sms, st);
        case 2: return launch_f32<R, 2>(a, num_sms, st);
        case 3: return launch_f32<R, 3>(a, num_sms, st);
        case 4: return launch_tm<R>(a, num_sms, st);
        case 5: return a.bx ? launch_tmc<R, false, true>(a, num_sms, st) : launch_tmc<R>(a, num_sms, st);
        case 6: return launch_tmp<R>(a, num_sms, st);
        case 7: return launch_tmx<R>(a, num_sms, st);
        default: return cudaErrorInvalidValue;
    }
}

template <int R>
cudaError_t launch_f64(const MarchArgs& a, int num_sms, cudaStream_t st) {
    using S = Shape<R>;
    const int64_t nsrc = a.src_end - a.src_begin;
    if (nsrc <= 0) return cudaSuccess;
    const size_t smem = (size_t)(5 * S::SPB64 * S::W + S::SPB64 * S::COLS) * 8;
    cudaError_t e = cudaFuncSetAttribute(march_f64_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, march_f64_kernel<R>, S::THREADS64, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int64_t nbatch = (nsrc + S::SPB64 - 1) / S::SPB64;
    const int64_t grid = nbatch < (int64_t)num_sms * per_sm ? nbatch : (int64_t)num_sms * per_sm;
    march_f64_kernel<R><<<(unsigned)grid, S::THREADS64, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t dispatch(const MarchArgs& a, int P, int num_sms, cudaStream_t st) {
    if (a.store == Store::F64) {
        switch (a.R) {
            case 1: return launch_f64<1>(a, num_sms, st);
            case 2: return launch_f64<2>(a, num_sms, st);
            case 3: return launch_f64<3>(a, num_sms, st);
            case 4: return launch_f64<4>(a, num_sms, st);
            case 5: return launch_f64<5>(a, num_sms, st);
            case 6: return launch_f64<6>(a, num_sms, st);
            case 7: return launch_f64<7>(a, num_sms, st);
            case 8: return launch_f64<8>(a, num_sms, st);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (a.R) {
        case 1: return launch_f32_p<1>(a, P, num_sms, st);
        case 2: return launch_f32_p<2>(a, P, num_sms, st);
        case 3: return launch_f32_p<3>(a, P, num_sms, st);
        case 4: return launch_f32_p<4>(a, P, num_sms, st);
        case 5: return launch_f32_p<5>(a, P, num_sms, st);
        case 6: return launch_f32_p<6>(a, P, num_sms, st);
        case 7: return launch_f32_p<7>(a, P, num_sms, st);
        case 8: return launch_f32_p<8>(a, P, num_sms, st);
        case 9: return P == 5 ? (a.bx ? launch_tmc<9, false, true>(a, num_sms, st) : launch_tmc<9>(a, num_sms, st))
                       : P == 4 ? launch_tm<9>(a, num_sms, st) : P == 7 ? launch_tmx<9>(a, num_sms, st)
                       : cudaErrorInvalidValue;
        case 10: return P == 5 ? (a.bx ? launch_tmc<10, false, true>(a, num_sms, st) : launch_tmc<10>(a, num_sms, st))
                        : P == 4 ? launch_tm<10>(a, num_sms, st) : P == 7 ? launch_tmx<10>(a, num_sms, st)
                        : cudaErrorInvalidValue;
        default: return cudaErrorInvalidValue;
    }
}

// Thread-mapping autotuner (P = threads per window column).  Each candidate is timed once on the
// context stream over a sample of the real sources (the sample's results are identical whatever P is,
// and the full launch overwrites them); the fastest is cached per (device, R, storage) for the process.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, int> g_tune;

int default_parts(int R) { return R > 8 ? 5 : R >= 4 ? 2 : 1; }

cudaError_t tune_parts(const MarchArgs& a, int num_sms, cudaStream_t st, int* best) {
    const int W1 = 2 * a.R + 1, cols = W1 * W1;
    const int64_t per_wave = (int64_t)num_sms * ((512 / cols) > 0 ? 512 / cols : 1);
    MarchArgs s = a;
    s.src_end = a.src_begin + std::min<int64_t>(a.src_end - a.src_begin, 16 * per_wave);
    MarchArgs warm = a;
    warm.src_end = a.src_begin + std::min<int64_t>(a.src_end - a.src_begin, per_wave);
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) { cudaEventDestroy(e0); return e; }
    float best_ms = 1e30f;
    *best = default_parts(a.R);
    for (int P = 1; P <= 7 && e == cudaSuccess; P++) {
        if (P <= 3 && P > W1) continue;
        if (a.R > 8 && (P < 4 || P == 6)) continue; // mappings 4, 5 and 7 cover R = 9, 10
        if (P == 5 && a.R < 6) continue;          // one CTA of < 6 warps per SM: never the fastest there
        e = dispatch(warm, P, num_sms, st);
        float ms = 1e30f;
        for (int rep = 0; rep < 2 && e == cudaSuccess; rep++) {      // the faster of two timings
            float t = 0.f;
            e = cudaEventRecord(e0, st);
            if (e == cudaSuccess) e = dispatch(s, P, num_sms, st);
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
            if (e == cudaSuccess && t < ms) ms = t;
        }
        if (e == cudaSuccess && ms < best_ms) { best_ms = ms; *best = P; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e;
}

}  // namespace

cudaError_t tune_march(const MarchArgs& a, int num_sms, int parts_req, cudaStream_t st, int* parts) {
    if (a.store == Store::F64) { *parts = 1; return cudaSuccess; }
    if (parts_req >= 1 && parts_req <= 7 && (a.R <= 8 || parts_req == 4 || parts_req == 5 || parts_req == 7)) {
        *parts = parts_req;
        return cudaSuccess;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_tuple(dev, a.R, (int)a.store);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) { *parts = it->second; return cudaSuccess; }
    }
    int P = 0;
    cudaError_t e = tune_parts(a, num_sms, st, &P);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = P;
    *parts = P;
    return cudaSuccess;
}

cudaError_t launch_march_coarse(const MarchArgs& a, int R, int num_sms, cudaStream_t st) {
    switch (R) {
        case 1: return a.bx ? launch_tmc<1, true, true>(a, num_sms, st) : launch_tmc<1, true>(a, num_sms, st);
        case 2: return a.bx ? launch_tmc<2, true, true>(a, num_sms, st) : launch_tmc<2, true>(a, num_sms, st);
        case 3: return a.bx ? launch_tmc<3, true, true>(a, num_sms, st) : launch_tmc<3, true>(a, num_sms, st);
        case 4: return a.bx ? launch_tmc<4, true, true>(a, num_sms, st) : launch_tmc<4, true>(a, num_sms, st);
        case 5: return a.bx ? launch_tmc<5, true, true>(a, num_sms, st) : launch_tmc<5, true>(a, num_sms, st);
        case 6: return a.bx ? launch_tmc<6, true, true>(a, num_sms, st) : launch_tmc<6, true>(a, num_sms, st);
        case 7: return a.bx ? launch_tmc<7, true, true>(a, num_sms, st) : launch_tmc<7, true>(a, num_sms, st);
        case 8: return a.bx ? launch_tmc<8, true, true>(a, num_sms, st) : launch_tmc<8, true>(a, num_sms, st);
        case 9: return a.bx ? launch_tmc<9, true, true>(a, num_sms, st) : launch_tmc<9, true>(a, num_sms, st);
        case 10: return a.bx ? launch_tmc<10, true, true>(a, num_sms, st) : launch_tmc<10, true>(a, num_sms, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_march(const MarchArgs& a, int num_sms, int parts_req, cudaStream_t st, int* parts_used) {
    int P = 1;
    if (a.bx && a.store != Store::F64) {          // direction-dependent coefficients: mapping 5 only
        if (parts_used) *parts_used = 5;
        return dispatch(a, 5, num_sms, st);
    }
    if (a.store != Store::F64) {
        if (parts_req >= 1 && parts_req <= 7 && (a.R <= 8 || parts_req == 4 || parts_req == 5 || parts_req == 7)) {
            P = parts_req;
        } else {
            int dev = 0;
            cudaGetDevice(&dev);
            const auto key = std::make_tuple(dev, a.R, (int)a.store);
            {
                std::lock_guard<std::mutex> lk(g_tune_mu);
                auto it = g_tune.find(key);
                if (it != g_tune.end()) P = it->second; else P = 0;
            }
            if (P == 0) {
                cudaError_t e = tune_parts(a, num_sms, st, &P);
                if (e != cudaSuccess) return e;
                std::lock_guard<std::mutex> lk(g_tune_mu);
                g_tune[key] = P;
            }
        }
    }
    if (parts_used) *parts_used = P;
    return dispatch(a, P, num_sms, st);
}

}  // namespace fdirw
