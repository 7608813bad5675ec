// One FDiRW macro step as a deterministic gather (Eq. 8 / Eq. 14 with a banded p):
//
//     chat(s)  = sigma_s * c(s)                                   (FP64 renormalisation, Sec. 3.3)
//     c'(x)    = sum_o Q[o][x] * chat(x - o),  o in [-R, R]^3 in a fixed order
//
// Q is destination-indexed (Q[o][x] = stored kernel of source x - o at offset o), so a thread that owns
// VX consecutive destinations reads VX consecutive values of each plane: 16-byte aligned vector loads,
// coalesced across the warp, every cache value read exactly once per step.  chat is stored with a zero
// halo of R cells on every side, so x - o never leaves the buffer and no bounds test is needed.
//
// Accumulation (Sec. 3.3: multiply in the storage precision, accumulate in higher precision):
//   - FP64 storage: FP64 FMA.
//   - FP32/FP16/BF16 storage: GB300 issues FP64 FMAs at 1/73 of the FP32 rate (measured), so each row of
//     2R+1 terms is summed as an unevaluated pair of FP32 values (s, c) -- error-free product (FMA
//     residual) and error-free addition (Knuth TwoSum), with chat split into hi = fp32(v),
//     lo = fp32(v - hi) -- and the rows of a destination are summed as a second FP32 pair (ff_add);
//     one FP64 addition per destination forms the result.
//   - FDIRW_ACCUM_FP32: FP32 products and row sums (one FMA per term), rows as above; the caller then
//     restores the step's FP64 mass budget (launch_restore_mass).
// The work per step is HBM-bound in the cache read (N * (2R+1)^3 * storage bytes).
#include "fdirw_internal.h"
#include "ff.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace fdirw {

namespace {

template <typename T, int VX>
struct Vec;
template <> struct Vec<double, 2> { using type = double2; };
template <> struct Vec<float, 4> { using type = float4; };
template <> struct Vec<__half, 8> { using type = uint4; };
template <> struct Vec<__nv_bfloat16, 8> { using type = uint4; };

// Loads VX consecutive stored values (16 bytes) and widens them to float.
template <typename ST, int VX>
__device__ __forceinline__ void load_q(const ST* p, float (&q)[VX]) {
    using V = typename Vec<ST, VX>::type;
    const V v = __ldcs(reinterpret_cast<const V*>(p));     // streamed: read once per step
    const ST* e = reinterpret_cast<const ST*>(&v);
#pragma unroll
    for (int j = 0; j < VX; j++) q[j] = widen(e[j]);
}

// Mixed path: ST in {float, half, bf16}, VX = 16 / sizeof(ST), chat as float2 (hi, lo).
template <typename ST, int R>
__global__ void __launch_bounds__(256) gather_ff_kernel(const ST* __restrict__ Q, const float2* __restrict__ chat,
                                                        Grid g, Pad p, int64_t qs, bool acc_in,
                                                        double* __restrict__ out, int z0, int zn, int64_t qoff) {
    constexpr int VX = 16 / sizeof(ST);
    constexpr int W1 = 2 * R + 1;
    constexpr int NC = VX + 2 * R;
    const int nxv = g.nx / VX;
    const int64_t nthreads = (int64_t)nxv * g.ny * zn;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (tid >= nthreads) return;
    const int xv = (int)(tid % nxv);
    const int64_t r = tid / nxv;
    const int y = (int)(r % g.ny);
    const int z = z0 + (int)(r / g.ny);
    const int x0 = xv * VX;
    const int64_t i0 = (int64_t)x0 + (int64_t)g.nx * y + (int64_t)g.nx * g.ny * z;

    float A[VX], B[VX];                       // running double-float sum of each destination
#pragma unroll
    for (int j = 0; j < VX; j++) { A[j] = 0.f; B[j] = 0.f; }

    for (int oz = -R; oz <= R; oz++) {
        for (int oy = -R; oy <= R; oy++) {
            // chat row of the sources x - o for ox in [-R, R]: padded x in [x0, x0 + VX + 2R).
            const float2* row = chat + ((int64_t)(z - oz + R) * p.py + (y - oy + R)) * p.px + x0;
            float2 ch[NC];
#pragma unroll
            for (int j = 0; j < NC; j++) ch[j] = __ldg(row + j);
            const ST* qrow = Q + ((int64_t)((oz + R) * W1 + (oy + R)) * W1) * qs + (i0 - qoff);
            // The FP32 pair restarts at zero on every row of 2R+1 terms, so its compensation term stays
            // within a few ulps of the row sum; the row is then added to the destination's pair.
            float s[VX], c[VX];
#pragma unroll
            for (int j = 0; j < VX; j++) { s[j] = 0.f; c[j] = 0.f; }
#pragma unroll
            for (int ox = -R; ox <= R; ox++) {
                float q[VX];
                load_q<ST, VX>(qrow + (int64_t)(ox + R) * qs, q);
#pragma unroll
                for (int j = 0; j < VX; j++) ff_madd(s[j], c[j], q[j], ch[j - ox + R]);
            }
#pragma unroll
            for (int j = 0; j < VX; j++) ff_add(A[j], B[j], s[j], c[j]);
        }
    }
#pragma unroll
    for (int j = 0; j < VX; j++) out[i0 + j] = (acc_in ? out[i0 + j] : 0.0) + ((double)A[j] + (double)B[j]);
}

// FDIRW_ACCUM_FP32: the loop of gather_ff_kernel with FP32 products and row sums (one FMA per term) and an
// FP32 chat; the rows still go into a double-float pair per destination.  The caller restores the mass.
template <typename ST, int R>
__global__ void __launch_bounds__(256) gather_fp32_kernel(const ST* __restrict__ Q, const float* __restrict__ chat,
                                                          Grid g, Pad p, int64_t qs, bool acc_in,
                                                          double* __restrict__ out, int z0, int zn, int64_t qoff) {
    constexpr int VX = 16 / sizeof(ST);
    constexpr int W1 = 2 * R + 1;
    constexpr int NC = VX + 2 * R;
    const int nxv = g.nx / VX;
    const int64_t nthreads = (int64_t)nxv * g.ny * zn;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (tid >= nthreads) return;
    const int xv = (int)(tid % nxv);
    const int64_t r = tid / nxv;
    const int y = (int)(r % g.ny);
    const int z = z0 + (int)(r / g.ny);
    const int x0 = xv * VX;
    const int64_t i0 = (int64_t)x0 + (int64_t)g.nx * y + (int64_t)g.nx * g.ny * z;

    float A[VX], B[VX];
#pragma unroll
    for (int j = 0; j < VX; j++) { A[j] = 0.f; B[j] = 0.f; }
    for (int oz = -R; oz <= R; oz++) {
        for (int oy = -R; oy <= R; oy++) {
            const float* row = chat + ((int64_t)(z - oz + R) * p.py + (y - oy + R)) * p.px + x0;
            float ch[NC];
#pragma unroll
            for (int j = 0; j < NC; j++) ch[j] = __ldg(row + j);
            const ST* qrow = Q + ((int64_t)((oz + R) * W1 + (oy + R)) * W1) * qs + (i0 - qoff);
            float s[VX];
#pragma unroll
            for (int j = 0; j < VX; j++) s[j] = 0.f;
#pragma unroll
            for (int ox = -R; ox <= R; ox++) {
                float q[VX];
                load_q<ST, VX>(qrow + (int64_t)(ox + R) * qs, q);
#pragma unroll
                for (int j = 0; j < VX; j++) s[j] = fmaf(q[j], ch[j - ox + R], s[j]);
            }
#pragma unroll
            for (int j = 0; j < VX; j++) ff_add(A[j], B[j], s[j], 0.f);
        }
    }
#pragma unroll
    for (int j = 0; j < VX; j++) out[i0 + j] = (acc_in ? out[i0 + j] : 0.0) + ((double)A[j] + (double)B[j]);
}

// FP64 path: FP64 storage, FP64 chat, FP64 FMA accumulation, VX = 2.
template <int R>
__global__ void __launch_bounds__(256) gather_f64_kernel(const double* __restrict__ Q, const double* __restrict__ chat,
                                                         Grid g, Pad p, double* __restrict__ out, int64_t qs, int z0,
                                                         int zn, int64_t qoff) {
    constexpr int VX = 2;
    constexpr int W1 = 2 * R + 1;
    constexpr int NC = VX + 2 * R;
    const int nxv = g.nx / VX;
    const int64_t nthreads = (int64_t)nxv * g.ny * zn;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (tid >= nthreads) return;
    const int xv = (int)(tid % nxv);
    const int64_t r = tid / nxv;
    const int y = (int)(r % g.ny);
    const int z = z0 + (int)(r / g.ny);
    const int x0 = xv * VX;
    const int64_t i0 = (int64_t)x0 + (int64_t)g.nx * y + (int64_t)g.nx * g.ny * z;
    double acc0 = 0.0, acc1 = 0.0;
    for (int oz = -R; oz <= R; oz++) {
        for (int oy = -R; oy <= R; oy++) {
            const double* row = chat + ((int64_t)(z - oz + R) * p.py + (y - oy + R)) * p.px + x0;
            double ch[NC];
#pragma unroll
            for (int j = 0; j < NC; j++) ch[j] = __ldg(row + j);
            const double* qrow = Q + ((int64_t)((oz + R) * W1 + (oy + R)) * W1) * qs + (i0 - qoff);
#pragma unroll
            for (int ox = -R; ox <= R; ox++) {
                const double2 q = __ldcs(reinterpret_cast<const double2*>(qrow + (int64_t)(ox + R) * qs));
                acc0 = fma(q.x, ch[0 - ox + R], acc0);
                acc1 = fma(q.y, ch[1 - ox + R], acc1);
            }
        }
    }
    out[i0] = acc0;
    out[i0 + 1] = acc1;
}

// Any nx (no vector alignment): one destination per thread, runtime R, same arithmetic as above.
template <typename ST, int MODE>
__global__ void __launch_bounds__(256) gather_scalar_kernel(const ST* __restrict__ Q, const void* __restrict__ chat,
                                                            Grid g, Pad p, int R, int64_t qs, bool acc_in,
                                                            double* __restrict__ out, int z0, int zn, int64_t qoff) {
    const int64_t nxy = (int64_t)g.nx * g.ny;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (tid >= nxy * zn) return;
    const int64_t i = z0 * nxy + tid;
    const int x = (int)(i % g.nx);
    const int64_t r = i / g.nx;
    const int y = (int)(r % g.ny);
    const int z = (int)(r / g.ny);
    double acc = (MODE == 0 && acc_in) ? out[i] : 0.0;   // FP64 path: plain FMA accumulation
    float A = 0.f, B = 0.f;                               // FP32 paths: running double-float sum
    int o = 0;
    for (int oz = -R; oz <= R; oz++)
        for (int oy = -R; oy <= R; oy++) {
            float s = 0.f, c = 0.f;
            for (int ox = -R; ox <= R; ox++, o++) {
                const int64_t pi = ((int64_t)(z - oz + R) * p.py + (y - oy + R)) * p.px + (x - ox + R);
                const ST qv = Q[(int64_t)o * qs + (i - qoff)];
                if constexpr (MODE == 1) {
                    ff_madd(s, c, widen(qv), reinterpret_cast<const float2*>(chat)[pi]);
                } else if constexpr (MODE == 2) {
                    s = fmaf(widen(qv), reinterpret_cast<const float*>(chat)[pi], s);
                } else {
                    acc = fma((double)qv, reinterpret_cast<const double*>(chat)[pi], acc);
                }
            }
            if constexpr (MODE != 0) ff_add(A, B, s, c);
        }
    if constexpr (MODE != 0) out[i] = (acc_in ? out[i] : 0.0) + ((double)A + (double)B);
    else out[i] = acc;
}

__global__ void scale_kernel(const double* __restrict__ c, const double* __restrict__ sigma, Grid g, int R, Pad p,
                             void* __restrict__ chat, int mode, int64_t i0, int64_t i1) {
    for (int64_t i = i0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < i1; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % g.nx);
        const int64_t r = i / g.nx;
        const int y = (int)(r % g.ny);
        const int z = (int)(r / g.ny);
        const int64_t pi = ((int64_t)(z + R) * p.py + (y + R)) * p.px + (x + R);
        const double v = sigma[i] * c[i];
        if (mode == 1) {
            const float hi = (float)v;
            const float lo = (float)(v - (double)hi);
            reinterpret_cast<float2*>(chat)[pi] = make_float2(hi, lo);
        } else if (mode == 2) {
            reinterpret_cast<float*>(chat)[pi] = (float)v;
        } else {
            reinterpret_cast<double*>(chat)[pi] = v;
        }
    }
}

// Fixed-order FP64 reduction, pass 1: block b sums the contiguous chunk b (thread-strided, then a tree).
__global__ void __launch_bounds__(256) mass_partial_kernel(const double* __restrict__ c, int64_t n,
                                                           double* __restrict__ partials) {
    __shared__ double sh[8];
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t lo = blockIdx.x * chunk;
    const int64_t hi = lo + chunk < n ? lo + chunk : n;
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

// Pass 2: one block of kMassBlocks threads sums the partials.
__global__ void __launch_bounds__(kMassBlocks) mass_final_kernel(const double* __restrict__ partials,
                                                                 double* __restrict__ out) {
    __shared__ double sh[kMassBlocks / 32];
    double v = partials[threadIdx.x];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double w = sh[threadIdx.x];
        for (int off = 16; off > 0; off >>= 1) w += __shfl_xor_sync(0xffffffffu, w, off);
        if (threadIdx.x == 0) *out = w;
    }
}

// Mass restoration, pass 1: block b sums c and |c| over the contiguous chunk b (as mass_partial_kernel).
__global__ void __launch_bounds__(256) mass_abs_partial_kernel(const double* __restrict__ c, int64_t n,
                                                               double* __restrict__ partials) {
    __shared__ double sh[2][8];
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t lo = blockIdx.x * chunk;
    const int64_t hi = lo + chunk < n ? lo + chunk : n;
    double acc = 0.0, aab = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const double v = c[i];
        acc += v;
        aab += fabs(v);
    }
    for (int off = 16; off > 0; off >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, off);
        aab += __shfl_xor_sync(0xffffffffu, aab, off);
    }
    if ((threadIdx.x & 31) == 0) { sh[0][threadIdx.x >> 5] = acc; sh[1][threadIdx.x >> 5] = aab; }
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? sh[0][threadIdx.x] : 0.0;
        double w = threadIdx.x < (blockDim.x >> 5) ? sh[1][threadIdx.x] : 0.0;
        for (int off = 16; off > 0; off >>= 1) {
            v += __shfl_xor_sync(0xffffffffu, v, off);
            w += __shfl_xor_sync(0xffffffffu, w, off);
        }
        if (threadIdx.x == 0) { partials[blockIdx.x] = v; partials[kMassBlocks + blockIdx.x] = w; }
    }
}

// Pass 2: one block sums both partial sets and writes f = (m_in - S) / A into fix[1] (0 when A = 0) and
// the running maximum of |m_in - S| / |m_in| into fix[2].
__global__ void __launch_bounds__(kMassBlocks) mass_fix_kernel(const double* __restrict__ partials,
                                                               double* __restrict__ fix) {
    __shared__ double sh[2][kMassBlocks / 32];
    double v = partials[threadIdx.x], w = partials[kMassBlocks + threadIdx.x];
    for (int off = 16; off > 0; off >>= 1) {
        v += __shfl_xor_sync(0xffffffffu, v, off);
        w += __shfl_xor_sync(0xffffffffu, w, off);
    }
    if ((threadIdx.x & 31) == 0) { sh[0][threadIdx.x >> 5] = v; sh[1][threadIdx.x >> 5] = w; }
    __syncthreads();
    if (threadIdx.x < 32) {
        double S = sh[0][threadIdx.x], A = sh[1][threadIdx.x];
        for (int off = 16; off > 0; off >>= 1) {
            S += __shfl_xor_sync(0xffffffffu, S, off);
            A += __shfl_xor_sync(0xffffffffu, A, off);
        }
        if (threadIdx.x == 0) {
            fix[1] = A > 0.0 ? (fix[0] - S) / A : 0.0;
            // largest relative drift of the FP32-accumulated totals before restoration since fix[2] was reset
            if (fix[0] != 0.0) fix[2] = fmax(fix[2], fabs(fix[0] - S) / fabs(fix[0]));
        }
    }
}

// Pass 3: c[i] += f |c[i]|.
__global__ void mass_apply_kernel(double* __restrict__ c, int64_t n, const double* __restrict__ fix) {
    const double f = fix[1];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        c[i] = fma(f, fabs(c[i]), c[i]);
}

// Per-structure mass restoration of batch contexts: kSegBlocks blocks per structure, block p summing the
// p-th contiguous part of its cells (c and |c|); then one warp per structure sums the parts in order.
__global__ void __launch_bounds__(256) seg_sums_kernel(const double* __restrict__ c, const int64_t* __restrict__ base,
                                                       int s0, double* __restrict__ partials) {
    __shared__ double sh[2][8];
    const int i = s0 + (int)(blockIdx.x / kSegBlocks), part = (int)(blockIdx.x % kSegBlocks);
    const int64_t b0 = base[i], n = base[i + 1] - b0;
    const int64_t chunk = (n + kSegBlocks - 1) / kSegBlocks;
    const int64_t lo = b0 + part * chunk;
    const int64_t hi = lo + chunk < b0 + n ? lo + chunk : b0 + n;
    double acc = 0.0, aab = 0.0;
    for (int64_t j = lo + threadIdx.x; j < hi; j += blockDim.x) {
        const double v = c[j];
        acc += v;
        aab += fabs(v);
    }
    for (int off = 16; off > 0; off >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, off);
        aab += __shfl_xor_sync(0xffffffffu, aab, off);
    }
    if ((threadIdx.x & 31) == 0) { sh[0][threadIdx.x >> 5] = acc; sh[1][threadIdx.x >> 5] = aab; }
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? sh[0][threadIdx.x] : 0.0;
        double w = threadIdx.x < (blockDim.x >> 5) ? sh[1][threadIdx.x] : 0.0;
        for (int off = 16; off > 0; off >>= 1) {
            v += __shfl_xor_sync(0xffffffffu, v, off);
            w += __shfl_xor_sync(0xffffffffu, w, off);
        }
        if (threadIdx.x == 0) { partials[2 * blockIdx.x] = v; partials[2 * blockIdx.x + 1] = w; }
    }
}

// One warp per structure i in [s0, s0 + nseg): target == true stores its total in fix[2 i]; otherwise
// fix[2 i + 1] = (fix[2 i] - S_i) / A_i (0 when A_i = 0).
__global__ void seg_fix_kernel(const double* __restrict__ partials, int s0, int nseg, double* __restrict__ fix,
                               bool target) {
    const int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (w >= nseg) return;
    static_assert(kSegBlocks == 32, "one part per lane");
    double S = partials[2 * (w * kSegBlocks + lane)], A = partials[2 * (w * kSegBlocks + lane) + 1];
    for (int off = 16; off > 0; off >>= 1) {
        S += __shfl_xor_sync(0xffffffffu, S, off);
        A += __shfl_xor_sync(0xffffffffu, A, off);
    }
    const int i = s0 + w;
    if (lane == 0) {
        if (target) fix[2 * i] = S;
        else fix[2 * i + 1] = A > 0.0 ? (fix[2 * i] - S) / A : 0.0;
    }
}

__global__ void __launch_bounds__(256) seg_apply_kernel(double* __restrict__ c, const int64_t* __restrict__ base, int s0,
                                                        const double* __restrict__ fix) {
    const int i = s0 + (int)(blockIdx.x / kSegBlocks), part = (int)(blockIdx.x % kSegBlocks);
    const int64_t b0 = base[i], n = base[i + 1] - b0;
    const int64_t chunk = (n + kSegBlocks - 1) / kSegBlocks;
    const int64_t lo = b0 + part * chunk;
    const int64_t hi = lo + chunk < b0 + n ? lo + chunk : b0 + n;
    const double f = fix[2 * i + 1];
    for (int64_t j = lo + threadIdx.x; j < hi; j += blockDim.x) c[j] = fma(f, fabs(c[j]), c[j]);
}

template <typename ST>
__global__ void read_kernels_kernel(const ST* __restrict__ Q, const double* __restrict__ sigma, Grid g, int R,
                                    const int64_t* __restrict__ sources, int64_t n_src, double* __restrict__ out) {
    const int W1 = 2 * R + 1;
    const int64_t W = (int64_t)W1 * W1 * W1;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_src * W; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = t / W;
        const int o = (int)(t % W);
        const int64_t s = sources[q];
        const int ox = o % W1 - R, oy = (o / W1) % W1 - R, oz = o / (W1 * W1) - R;
        const int sx = (int)(s % g.nx);
        const int64_t r = s / g.nx;
        const int sy = (int)(r % g.ny), sz = (int)(r / g.ny);
        const int x = sx + ox, y = sy + oy, z = sz + oz;
        double v = 0.0;
        if (x >= 0 && x < g.nx && y >= 0 && y < g.ny && z >= 0 && z < g.nz) {
            const int64_t i = (int64_t)x + (int64_t)g.nx * y + (int64_t)g.nx * g.ny * z;
            v = (double)widen(Q[(int64_t)o * g.n + i]) * sigma[s];
        }
        out[t] = v;
    }
}
template <>
__global__ void read_kernels_kernel<double>(const double* __restrict__ Q, const double* __restrict__ sigma, Grid g,
                                            int R, const int64_t* __restrict__ sources, int64_t n_src,
                                            double* __restrict__ out) {
    const int W1 = 2 * R + 1;
    const int64_t W = (int64_t)W1 * W1 * W1;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_src * W; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = t / W;
        const int o = (int)(t % W);
        const int64_t s = sources[q];
        const int ox = o % W1 - R, oy = (o / W1) % W1 - R, oz = o / (W1 * W1) - R;
        const int sx = (int)(s % g.nx);
        const int64_t r = s / g.nx;
        const int sy = (int)(r % g.ny), sz = (int)(r / g.ny);
        const int x = sx + ox, y = sy + oy, z = sz + oz;
        double v = 0.0;
        if (x >= 0 && x < g.nx && y >= 0 && y < g.ny && z >= 0 && z < g.nz) {
            const int64_t i = (int64_t)x + (int64_t)g.nx * y + (int64_t)g.nx * g.ny * z;
            v = Q[(int64_t)o * g.n + i] * sigma[s];
        }
        out[t] = v;
    }
}

int blocks_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    return (int)(b < 1 ? 1 : b);
}

// Destination planes [z0, z0 + zn) of the launch and the column offset of its cache (a slab of a
// streamed uniform cache); {0, nz, 0} for a whole grid.
struct Slab {
    int z0, zn;
    int64_t qoff;
};

template <typename ST, int R>
cudaError_t gather_ff_r(const void* Q, const void* chat, Grid g, Pad p, int64_t qs, bool acc_in, double* out,
                        cudaStream_t st, Slab sl) {
    constexpr int VX = 16 / sizeof(ST);
    const int64_t nt = (int64_t)(g.nx / VX) * g.ny * sl.zn;
    if (nt <= 0) return cudaSuccess;
    gather_ff_kernel<ST, R><<<blocks_for(nt, 256), 256, 0, st>>>(reinterpret_cast<const ST*>(Q),
                                                                   reinterpret_cast<const float2*>(chat), g, p, qs,
                                                                   acc_in, out, sl.z0, sl.zn, sl.qoff);
    return cudaGetLastError();
}

template <typename ST>
cudaError_t gather_ff(const void* Q, const void* chat, Grid g, int R, Pad p, int64_t qs, bool acc_in, double* out,
                      cudaStream_t st, Slab sl) {
    switch (R) {
        case 1: return gather_ff_r<ST, 1>(Q, chat, g, p, qs, acc_in, out, st, sl);
        case 2: return gather_ff_r<ST, 2>(Q, chat, g, p, qs, acc_in, out, st, sl);
        case 3: return gather_ff_r<ST, 3>(Q, chat, g, p, qs, acc_in, out, st, sl);
        case 4: return gather_ff_r<ST, 4>(Q, chat, g, p, qs, acc_in, out, st, sl);
        case 5: return gather_ff_r<ST, 5>(Q, chat, g, p, qs, acc_in, out, st, sl);
        case 6: return gather_ff_r<ST, 6>(Q, chat, g, p, qs, acc_in, out, st, sl);
        case 7: return gather_ff_r<ST, 7>(Q, chat, g, p, qs, acc_in, out, st, sl);
        case 8: return gather_ff_r<ST, 8>(Q, chat, g, p, qs, acc_in, out, st, sl);
        case 9: return gather_ff_r<ST, 9>(Q, chat, g, p, qs, acc_in, out, st, sl);
        case 10: return gather_ff_r<ST, 10>(Q, chat, g, p, qs, acc_in, out, st, sl);
        default: return cudaErrorInvalidValue;
    }
}

template <int R>
cudaError_t gather_f64_r(const void* Q, const void* chat, Grid g, Pad p, int64_t qs, double* out, cudaStream_t st,
                         Slab sl) {
    const int64_t nt = (int64_t)(g.nx / 2) * g.ny * sl.zn;
    if (nt <= 0) return cudaSuccess;
    gather_f64_kernel<R><<<blocks_for(nt, 256), 256, 0, st>>>(reinterpret_cast<const double*>(Q),
                                                               reinterpret_cast<const double*>(chat), g, p, out, qs,
                                                               sl.z0, sl.zn, sl.qoff);
    return cudaGetLastError();
}

cudaError_t gather_f64(const void* Q, const void* chat, Grid g, int R, Pad p, int64_t qs, double* out,
                       cudaStream_t st, Slab sl) {
    switch (R) {
        case 1: return gather_f64_r<1>(Q, chat, g, p, qs, out, st, sl);
        case 2: return gather_f64_r<2>(Q, chat, g, p, qs, out, st, sl);
        case 3: return gather_f64_r<3>(Q, chat, g, p, qs, out, st, sl);
        case 4: return gather_f64_r<4>(Q, chat, g, p, qs, out, st, sl);
        case 5: return gather_f64_r<5>(Q, chat, g, p, qs, out, st, sl);
        case 6: return gather_f64_r<6>(Q, chat, g, p, qs, out, st, sl);
        case 7: return gather_f64_r<7>(Q, chat, g, p, qs, out, st, sl);
        case 8: return gather_f64_r<8>(Q, chat, g, p, qs, out, st, sl);
        default: return cudaErrorInvalidValue;
    }
}

template <typename ST, int R>
cudaError_t gather_fp32_r(const void* Q, const float* chat, Grid g, Pad p, int64_t qs, bool acc_in, double* out,
                          cudaStream_t st, Slab sl) {
    constexpr int VX = 16 / sizeof(ST);
    const int64_t nt = (int64_t)(g.nx / VX) * g.ny * sl.zn;
    if (nt <= 0) return cudaSuccess;
    gather_fp32_kernel<ST, R><<<blocks_for(nt, 256), 256, 0, st>>>(reinterpret_cast<const ST*>(Q), chat, g, p, qs,
                                                                     acc_in, out, sl.z0, sl.zn, sl.qoff);
    return cudaGetLastError();
}

template <typename ST>
cudaError_t gather_fp32_st(const void* Q, const float* chat, Grid g, int R, Pad p, int64_t qs, bool acc_in,
                           double* out, cudaStream_t st, Slab sl) {
    switch (R) {
        case 1: return gather_fp32_r<ST, 1>(Q, chat, g, p, qs, acc_in, out, st, sl);
        case 2: return gather_fp32_r<ST, 2>(Q, chat, g, p, qs, acc_in, out, st, sl);
        case 3: return gather_fp32_r<ST, 3>(Q, chat, g, p, qs, acc_in, out, st, sl);
        case 4: return gather_fp32_r<ST, 4>(Q, chat, g, p, qs, acc_in, out, st, sl);
        case 5: return gather_fp32_r<ST, 5>(Q, chat, g, p, qs, acc_in, out, st, sl);
        case 6: return gather_fp32_r<ST, 6>(Q, chat, g, p, qs, acc_in, out, st, sl);
        case 7: return gather_fp32_r<ST, 7>(Q, chat, g, p, qs, acc_in, out, st, sl);
        case 8: return gather_fp32_r<ST, 8>(Q, chat, g, p, qs, acc_in, out, st, sl);
        case 9: return gather_fp32_r<ST, 9>(Q, chat, g, p, qs, acc_in, out, st, sl);
        case 10: return gather_fp32_r<ST, 10>(Q, chat, g, p, qs, acc_in, out, st, sl);
        default: return cudaErrorInvalidValue;
    }
}

// Scalar fallback of both accumulations and the FP64 path (any nx): MODE 0 FP64, 1 float-float, 2 FP32.
template <int MODE>
cudaError_t gather_scalar(const void* Q, Store store, const void* ch, Grid g, Pad p, int R, int64_t qs, bool acc,
                          double* out, cudaStream_t st, Slab sl) {
    const int64_t n = (int64_t)g.nx * g.ny * sl.zn;
    if (n <= 0) return cudaSuccess;
    const int b = blocks_for(n, 256);
    switch (store) {
        case Store::F64:
            if (MODE != 0) return cudaErrorInvalidValue;
            gather_scalar_kernel<double, MODE><<<b, 256, 0, st>>>(reinterpret_cast<const double*>(Q), ch, g, p, R,
                                                                  qs, acc, out, sl.z0, sl.zn, sl.qoff);
            break;
        case Store::F32:
            if (MODE == 0) return cudaErrorInvalidValue;
            gather_scalar_kernel<float, MODE><<<b, 256, 0, st>>>(reinterpret_cast<const float*>(Q), ch, g, p, R, qs,
                                                                 acc, out, sl.z0, sl.zn, sl.qoff);
            break;
        case Store::F16:
            if (MODE == 0) return cudaErrorInvalidValue;
            gather_scalar_kernel<__half, MODE><<<b, 256, 0, st>>>(reinterpret_cast<const __half*>(Q), ch, g, p, R,
                                                                  qs, acc, out, sl.z0, sl.zn, sl.qoff);
            break;
        case Store::BF16:
            if (MODE == 0) return cudaErrorInvalidValue;
            gather_scalar_kernel<__nv_bfloat16, MODE><<<b, 256, 0, st>>>(reinterpret_cast<const __nv_bfloat16*>(Q),
                                                                         ch, g, p, R, qs, acc, out, sl.z0, sl.zn,
                                                                         sl.qoff);
            break;
    }
    return cudaGetLastError();
}

// Float-float (FP32 storage types) or FP64 gather of one part (radius R, chat with a halo of Rp).
cudaError_t gather_part(const void* Q, Store store, int64_t qs, const void* chat, int Rp, Grid g, int R,
                        bool accumulate, double* c_out, cudaStream_t st, Slab sl) {
    if (R < 1 || R > Rp) return cudaErrorInvalidValue;
    const Pad p = make_pad(g, Rp);
    // The kernels index chat as if its halo were R: move the base by (Rp - R) on every axis.
    const int64_t shift = ((int64_t)(Rp - R) * p.py + (Rp - R)) * p.px + (Rp - R);
    const void* ch = static_cast<const char*>(chat) + shift * 8;   // chat element: double or float2, 8 bytes
    const int vx = 16 / store_bytes(store);
    const bool aligned = (reinterpret_cast<uintptr_t>(Q) % 16) == 0 && (qs * store_bytes(store)) % 16 == 0 &&
                         (sl.qoff * store_bytes(store)) % 16 == 0;
    if (store == Store::F64 && accumulate) return cudaErrorInvalidValue;   // uniform FP64 contexts only
    if (R <= (store == Store::F64 ? kMaxR64 : kMaxR) && g.nx % vx == 0 && aligned) {
        switch (store) {
            case Store::F64: return gather_f64(Q, ch, g, R, p, qs, c_out, st, sl);
            case Store::F32: return gather_ff<float>(Q, ch, g, R, p, qs, accumulate, c_out, st, sl);
            case Store::F16: return gather_ff<__half>(Q, ch, g, R, p, qs, accumulate, c_out, st, sl);
            case Store::BF16: return gather_ff<__nv_bfloat16>(Q, ch, g, R, p, qs, accumulate, c_out, st, sl);
        }
        return cudaErrorInvalidValue;
    }
    return store == Store::F64 ? gather_scalar<0>(Q, store, ch, g, p, R, qs, accumulate, c_out, st, sl)
                               : gather_scalar<1>(Q, store, ch, g, p, R, qs, accumulate, c_out, st, sl);
}

// FDIRW_ACCUM_FP32 gather of one part (FP32 chat with a halo of Rp).
cudaError_t gather_part_fp32(const void* Q, Store store, int64_t qs, const float* chat, int Rp, Grid g, int R,
                             bool accumulate, double* c_out, cudaStream_t st, Slab sl) {
    if (R < 1 || R > Rp || R > kMaxR || store == Store::F64) return cudaErrorInvalidValue;
    const Pad p = make_pad(g, Rp);
    const float* ch = chat + ((int64_t)(Rp - R) * p.py + (Rp - R)) * p.px + (Rp - R);
    const int vx = 16 / store_bytes(store);
    const bool aligned = (reinterpret_cast<uintptr_t>(Q) % 16) == 0 && (qs * store_bytes(store)) % 16 == 0 &&
                         (sl.qoff * store_bytes(store)) % 16 == 0;
    if (g.nx % vx == 0 && aligned) {
        switch (store) {
            case Store::F32: return gather_fp32_st<float>(Q, ch, g, R, p, qs, accumulate, c_out, st, sl);
            case Store::F16: return gather_fp32_st<__half>(Q, ch, g, R, p, qs, accumulate, c_out, st, sl);
            case Store::BF16: return gather_fp32_st<__nv_bfloat16>(Q, ch, g, R, p, qs, accumulate, c_out, st, sl);
            default: return cudaErrorInvalidValue;
        }
    }
    return gather_scalar<2>(Q, store, ch, g, p, R, qs, accumulate, c_out, st, sl);
}

}  // namespace

cudaError_t launch_scale(const double* c, const double* sigma, Grid g, int R, void* chat, int mode,
                         cudaStream_t st, int z0, int zn) {
    const Pad p = make_pad(g, R);
    const int64_t nxy = (int64_t)g.nx * g.ny;
    const int64_t i0 = (int64_t)z0 * nxy, i1 = zn < 0 ? g.n : (int64_t)(z0 + zn) * nxy;
    if (i1 <= i0) return cudaSuccess;
    int b = blocks_for(i1 - i0, 256);
    if (b > 152 * 16) b = 152 * 16;
    scale_kernel<<<b, 256, 0, st>>>(c, sigma, g, R, p, chat, mode, i0, i1);
    return cudaGetLastError();
}

cudaError_t launch_gather_part(const void* Q, Store store, int64_t qs, const void* chat, int Rp, Grid g, int R,
                               bool accumulate, double* c_out, cudaStream_t st) {
    return gather_part(Q, store, qs, chat, Rp, g, R, accumulate, c_out, st, Slab{0, g.nz, 0});
}

cudaError_t launch_gather_slab(const void* Q, Store store, int64_t qs, int64_t qoff, const void* chat, Grid g, int R,
                               int mode, int z0, int zn, double* c_out, cudaStream_t st) {
    const Slab sl{z0, zn, qoff};
    if (mode == 2)
        return gather_part_fp32(Q, store, qs, reinterpret_cast<const float*>(chat), R, g, R, false, c_out, st, sl);
    return gather_part(Q, store, qs, chat, R, g, R, false, c_out, st, sl);
}

cudaError_t launch_gather(const void* Q, Store store, const void* chat, Grid g, int R, double* c_out,
                          cudaStream_t st) {
    return launch_gather_part(Q, store, g.n, chat, R, g, R, false, c_out, st);
}

cudaError_t launch_mass(const double* c, int64_t n, double* partials, double* out, cudaStream_t st) {
    mass_partial_kernel<<<kMassBlocks, 256, 0, st>>>(c, n, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    mass_final_kernel<<<1, kMassBlocks, 0, st>>>(partials, out);
    return cudaGetLastError();
}

cudaError_t launch_seg_target(const double* c, const int64_t* base, int s0, int s1, double* partials, double* fix,
                              cudaStream_t st) {
    const int nseg = s1 - s0;
    if (nseg <= 0) return cudaSuccess;
    seg_sums_kernel<<<nseg * kSegBlocks, 256, 0, st>>>(c, base, s0, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    seg_fix_kernel<<<(nseg * 32 + 255) / 256, 256, 0, st>>>(partials, s0, nseg, fix, true);
    return cudaGetLastError();
}

cudaError_t launch_seg_restore(double* c, const int64_t* base, int s0, int s1, double* partials, double* fix,
                               cudaStream_t st) {
    const int nseg = s1 - s0;
    if (nseg <= 0) return cudaSuccess;
    seg_sums_kernel<<<nseg * kSegBlocks, 256, 0, st>>>(c, base, s0, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    seg_fix_kernel<<<(nseg * 32 + 255) / 256, 256, 0, st>>>(partials, s0, nseg, fix, false);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    seg_apply_kernel<<<nseg * kSegBlocks, 256, 0, st>>>(c, base, s0, fix);
    return cudaGetLastError();
}

cudaError_t launch_restore_mass(double* c, int64_t n, double* partials, double* fix, cudaStream_t st) {
    mass_abs_partial_kernel<<<kMassBlocks, 256, 0, st>>>(c, n, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    mass_fix_kernel<<<1, kMassBlocks, 0, st>>>(partials, fix);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int b = blocks_for(n, 256);
    if (b > 152 * 16) b = 152 * 16;
    mass_apply_kernel<<<b, 256, 0, st>>>(c, n, fix);
    return cudaGetLastError();
}

cudaError_t launch_gather_part_fp32(const void* Q, Store store, int64_t qs, const float* chat, int Rp, Grid g, int R,
                                    bool accumulate, double* c_out, cudaStream_t st) {
    return gather_part_fp32(Q, store, qs, chat, Rp, g, R, accumulate, c_out, st, Slab{0, g.nz, 0});
}

cudaError_t launch_gather_fp32(const void* Q, Store store, const float* chat, Grid g, int R, double* c_out,
                               cudaStream_t st) {
    return launch_gather_part_fp32(Q, store, g.n, chat, R, g, R, false, c_out, st);
}

cudaError_t launch_read_kernels(const void* Q, Store store, const double* sigma, Grid g, int R,
                                const int64_t* sources, int64_t n_src, double* out, cudaStream_t st) {
    const int64_t W = (int64_t)(2 * R + 1) * (2 * R + 1) * (2 * R + 1);
    int b = blocks_for(n_src * W, 256);
    if (b > 152 * 16) b = 152 * 16;
    switch (store) {
        case Store::F64:
            read_kernels_kernel<double><<<b, 256, 0, st>>>(reinterpret_cast<const double*>(Q), sigma, g, R, sources, n_src, out);
            break;
        case Store::F32:
            read_kernels_kernel<float><<<b, 256, 0, st>>>(reinterpret_cast<const float*>(Q), sigma, g, R, sources, n_src, out);
            break;
        case Store::F16:
            read_kernels_kernel<__half><<<b, 256, 0, st>>>(reinterpret_cast<const __half*>(Q), sigma, g, R, sources, n_src, out);
            break;
        case Store::BF16:
            read_kernels_kernel<__nv_bfloat16><<<b, 256, 0, st>>>(reinterpret_cast<const __nv_bfloat16*>(Q), sigma, g, R,
                                                                   sources, n_src, out);
            break;
    }
    return cudaGetLastError();
}

}  // namespace fdirw
