// Batched FDiRW with per-source window radii: many independent structures in one context, each source
// marched on a window whose radius follows its local diffusivity (Eq. 8 per structure; the paper has one
// domain and no window, so both the batch and the radius rule are extensions of Sec. 3.1).
//
//   radius     R(s) = clamp(ceil(2 sqrt(2 D(s) dt_macro) / h), R_min, R_max)   (FP64, this order)
//   buckets    the sources of each radius r, in global cell order; code(s) = (r << 28) | position of s
//              in its bucket
//   kernels    per radius r, one of two layouts (planes = offsets of the (2r+1)^3 window):
//              * destination-indexed, Q_r[plane][x] as in a uniform context (zero where the source x - o
//                has another radius), for radii held by at least kDestFraction of the cells: the gather
//                streams it with vector loads and needs no lookup;
//              * source-indexed, K_r[plane][j], j = the source's position in the chunk's part of bucket
//                r, for rare radii: only real kernel values are stored, and the gather finds j(x - o)
//                through the bucket code of the source.
//   gather     c'(x) = the source-indexed radii (ascending) in one pass, then each destination-indexed
//              radius (ascending) accumulated on top; within a radius the rows (o_z, o_y) ascend and each
//              row is a float-float sum added to the FP64 total, the arithmetic of the uniform gather.
//   chunks     structures are independent, so when the kernels of all of them do not fit the memory
//              budget they are processed in chunks of consecutive structures: build the chunk's kernels,
//              run all requested macro steps on its cells, move on.
//   graph      each fdirw_step call's device work (per chunk: the march launches of the radii present,
//              then scale + gather per macro step) is captured once into a CUDA graph and replayed.
#include "fdirw.h"
#include "fdirw_internal.h"
#include "ctx.h"
#include "ff.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

using namespace fdirw::host;

namespace fdirw {

namespace {

constexpr int kCodeShift = 28;
constexpr uint32_t kCodeMask = (1u << kCodeShift) - 1u;
constexpr int64_t kMaxBatchCells = (int64_t)1 << kCodeShift;   // bucket positions fit 28 bits
constexpr int kTileX = 32, kTileY = 8;                           // gather block: 32 x 8 destinations
constexpr double kDestFraction = 0.2;          // radii on at least this share of the cells: destination-indexed

inline int64_t wcells(int r) { return (int64_t)(2 * r + 1) * (2 * r + 1) * (2 * r + 1); }
inline uint64_t align256(uint64_t v) { return (v + 255u) & ~(uint64_t)255u; }

struct Chunk {
    int s0 = 0, s1 = 0;                          // structures [s0, s1)
    int64_t c0 = 0, c1 = 0;                      // their global cells
    int64_t qn = 0;                              // columns of a destination-indexed plane (16-aligned slots)
    int64_t seg_begin[kMaxR + 1] = {}, seg_end[kMaxR + 1] = {};   // positions in each bucket list
    uint64_t k_off[kMaxR + 1] = {};              // byte offset of the radius-r kernels in the arena
    uint64_t k_bytes = 0;
};

}  // namespace

constexpr int kAux = 8;                          // parallel branches for per-structure gathers

struct Batch {
    int n = 0;
    std::vector<Grid> grids;
    std::vector<double> hs, lams;
    std::vector<int64_t> base;                   // n + 1: first global cell of each structure
    std::vector<int64_t> blk;                    // n + 1: first gather block of each structure
    int64_t* d_base = nullptr;
    int4* d_dims = nullptr;
    int64_t* d_blk = nullptr;
    int Rmin = 0, Rmax = 0;
    std::vector<int> radii;                      // radii present, ascending
    int64_t count[kMaxR + 1] = {};
    std::vector<int64_t> before[kMaxR + 1];      // n + 1: bucket-r sources in structures < i
    int64_t* d_list[kMaxR + 1] = {};
    uint32_t* d_code = nullptr;
    uint32_t dest_mask = 0;                      // bit r: radius r uses the destination-indexed layout
    std::vector<int64_t> qbase;                  // n: first cache column of each structure within its chunk
    int64_t* d_qbase = nullptr;
    std::vector<int64_t> pbase;                  // n + 1: first element of each structure's padded chat
    float2* chat_pad = nullptr;                  // sigma * c with a halo of R_max (destination-indexed radii)
    double* seg_part = nullptr;                  // FDIRW_ACCUM_FP32: 2 * kSegBlocks partial sums per structure
    double* seg_fix = nullptr;                   // FDIRW_ACCUM_FP32: [target total, factor] per structure
    std::vector<Chunk> chunks;
    void* arena = nullptr;
    uint64_t arena_bytes = 0;
    int resident = -1;                           // chunk whose kernels the arena holds
    int parts[kMaxR + 1] = {};                   // march mapping per radius (0 = not chosen yet)
    float2* chat = nullptr;
    cudaStream_t gs = nullptr;                   // capture stream
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaStream_t aux[kAux] = {};                 // branches of the captured graph: per-structure gathers
    cudaEvent_t afork = nullptr, ajoin[kAux] = {};
    std::vector<cudaEvent_t> ev;                 // 4 per chunk: march begin/end, last gather begin/end
    std::vector<char> built, stepped;            // per chunk, in the last call
    cudaGraphExec_t exec = nullptr;
    const double* g_src = nullptr;
    double* g_dst = nullptr;
    int g_steps = -1;
    bool g_build = false;
    int graph_launches = 0;
};

namespace {

// ------------------------------------------------------------------------------------------ kernels

__global__ void radius_kernel(const double* __restrict__ D, int64_t n, double dt_macro, double h, int Rmin, int Rmax,
                              int8_t* __restrict__ R) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double t = __dmul_rn(2.0, D[i]);
        t = __dmul_rn(t, dt_macro);
        double r = __dsqrt_rn(t);
        r = __dmul_rn(2.0, r);
        r = __ddiv_rn(r, h);
        const double c = ceil(r);
        int v = c > (double)Rmax ? Rmax : (int)c;
        R[i] = (int8_t)(v < Rmin ? Rmin : v);
    }
}

__global__ void fill_kernel(double* __restrict__ p, int64_t n, double v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}

// chat = sigma * c over global cells [c0, c1), split into (hi, lo) FP32 halves.
__global__ void scale_flat_kernel(const double* __restrict__ c, const double* __restrict__ sigma, int64_t c0,
                                  int64_t c1, float2* __restrict__ chat) {
    for (int64_t i = c0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < c1; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = sigma[i] * c[i];
        const float hi = (float)v;
        chat[i] = make_float2(hi, (float)(v - (double)hi));
    }
}

struct VarArgs {
    const float2* chat;
    const uint32_t* code;
    double* out;
    const int64_t* s_base;
    const int4* s_dims;
    const int64_t* blk;
    int s0, s1;
    uint32_t rmask;                              // bit r set: radius r summed by gather_var_kernel
    uint32_t dmask;                              // bit r set: radius r is destination-indexed
    bool acc_in;                                 // add to out instead of overwriting it
    const int64_t* qbase;
    const void* K[kMaxR + 1];
    int64_t jbase[kMaxR + 1];
    int64_t ncol[kMaxR + 1];
};

// Contribution of the radius-R sources around destination (x, y, z) of a structure of dimensions d whose
// first global cell is base.
template <typename ST, int R>
__device__ __forceinline__ void acc_radius(const VarArgs& a, int4 d, int64_t base, int x, int y, int z, float& A,
                                           float& B) {
    constexpr int W1 = 2 * R + 1;
    const ST* __restrict__ K = reinterpret_cast<const ST*>(a.K[R]);
    const int64_t jb = a.jbase[R], nc = a.ncol[R];
    const uint32_t tag = (uint32_t)R << kCodeShift;
    for (int oz = -R; oz <= R; oz++) {
        const int sz = z - oz;
        if (sz < 0 || sz >= d.z) continue;
        for (int oy = -R; oy <= R; oy++) {
            const int sy = y - oy;
            if (sy < 0 || sy >= d.y) continue;
            const int64_t row = base + (int64_t)d.x * (sy + (int64_t)d.y * sz);
            const int64_t plane0 = (int64_t)((oz + R) * W1 + (oy + R)) * W1;
            float s = 0.f, c = 0.f;
#pragma unroll
            for (int ox = -R; ox <= R; ox++) {
                const int sx = x - ox;
                if (sx >= 0 && sx < d.x) {
                    const uint32_t code = __ldg(a.code + row + sx);
                    if ((code & ~kCodeMask) == tag) {
                        const float q = widen(K[(plane0 + (ox + R)) * nc + ((int64_t)(code & kCodeMask) - jb)]);
                        ff_madd(s, c, q, __ldg(a.chat + row + sx));
                    }
                }
            }
            ff_add(A, B, s, c);
        }
    }
}

template <typename ST>
__global__ void __launch_bounds__(kTileX * kTileY) gather_var_kernel(VarArgs a) {
    const int64_t gb = __ldg(a.blk + a.s0) + blockIdx.x;
    int lo = a.s0, hi = a.s1 - 1;                    // structure of this block
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(a.blk + mid) <= gb) lo = mid; else hi = mid - 1;
    }
    const int4 d = __ldg(a.s_dims + lo);
    const int64_t base = __ldg(a.s_base + lo);
    const int64_t t = gb - __ldg(a.blk + lo);
    const int ntx = (d.x + kTileX - 1) / kTileX, nty = (d.y + kTileY - 1) / kTileY;
    const int x = (int)(t % ntx) * kTileX + (threadIdx.x & (kTileX - 1));
    const int y = (int)((t / ntx) % nty) * kTileY + (threadIdx.x / kTileX);
    const int z = (int)(t / ((int64_t)ntx * nty));
    if (x >= d.x || y >= d.y) return;
    const int64_t i = base + x + (int64_t)d.x * (y + (int64_t)d.y * z);
    float A = 0.f, B = 0.f;                       // running double-float sum of the destination
    const uint32_t m = a.rmask;                   // radii summed here, in ascending order
    if (m & 1u) {                                 // radius 0: identity kernel, sigma = 1
        if ((__ldg(a.code + i) >> kCodeShift) == 0u) {
            const float2 ch = __ldg(a.chat + i);
            ff_add(A, B, ch.x, ch.y);
        }
    }
    if (m & (1u << 1)) acc_radius<ST, 1>(a, d, base, x, y, z, A, B);
    if (m & (1u << 2)) acc_radius<ST, 2>(a, d, base, x, y, z, A, B);
    if (m & (1u << 3)) acc_radius<ST, 3>(a, d, base, x, y, z, A, B);
    if (m & (1u << 4)) acc_radius<ST, 4>(a, d, base, x, y, z, A, B);
    if (m & (1u << 5)) acc_radius<ST, 5>(a, d, base, x, y, z, A, B);
    if (m & (1u << 6)) acc_radius<ST, 6>(a, d, base, x, y, z, A, B);
    if (m & (1u << 7)) acc_radius<ST, 7>(a, d, base, x, y, z, A, B);
    if (m & (1u << 8)) acc_radius<ST, 8>(a, d, base, x, y, z, A, B);
    if (m & (1u << 9)) acc_radius<ST, 9>(a, d, base, x, y, z, A, B);
    if (m & (1u << 10)) acc_radius<ST, 10>(a, d, base, x, y, z, A, B);
    a.out[i] = (a.acc_in ? a.out[i] : 0.0) + ((double)A + (double)B);
}

// Renormalised kernels of listed global sources on the (2 R_max + 1)^3 offset layout (zero outside the
// source's own window and structure).
template <typename ST>
__global__ void read_var_kernel(VarArgs a, const double* __restrict__ sigma, int n_struct, int Rm,
                                const int64_t* __restrict__ sources, int64_t n_src, double* __restrict__ out) {
    const int Wm = 2 * Rm + 1;
    const int64_t W = (int64_t)Wm * Wm * Wm;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_src * W; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = t / W;
        const int o = (int)(t % W);
        const int64_t s = sources[q];
        int lo = 0, hi = n_struct - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.s_base[mid] <= s) lo = mid; else hi = mid - 1;
        }
        const int4 d = a.s_dims[lo];
        const int64_t ls = s - a.s_base[lo];
        const int sx = (int)(ls % d.x), sy = (int)((ls / d.x) % d.y), sz = (int)(ls / ((int64_t)d.x * d.y));
        const int ox = o % Wm - Rm, oy = (o / Wm) % Wm - Rm, oz = o / (Wm * Wm) - Rm;
        const uint32_t code = a.code[s];
        const int r = (int)(code >> kCodeShift);
        const int x = sx + ox, y = sy + oy, z = sz + oz;
        double v = 0.0;
        if (abs(ox) <= r && abs(oy) <= r && abs(oz) <= r && x >= 0 && x < d.x && y >= 0 && y < d.y && z >= 0 &&
            z < d.z) {
            if (r == 0) {
                v = sigma[s];
            } else {
                const int W1 = 2 * r + 1;
                const int64_t plane = (ox + r) + (int64_t)W1 * ((oy + r) + (int64_t)W1 * (oz + r));
                const ST* K = reinterpret_cast<const ST*>(a.K[r]);
                const int64_t col = (a.dmask >> r) & 1u ? a.qbase[lo] + x + (int64_t)d.x * (y + (int64_t)d.y * z)
                                                        : (int64_t)(code & kCodeMask) - a.jbase[r];
                v = (double)widen(K[plane * a.ncol[r] + col]) * sigma[s];
            }
        }
        out[t] = v;
    }
}

int grid_blocks(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b > 152 * 16) b = 152 * 16;
    return (int)(b < 1 ? 1 : b);
}

// ------------------------------------------------------------------------------------------ host

VarArgs var_args(const fdirw_ctx* c, const Chunk& ch, double* out) {
    const Batch& b = *c->batch;
    VarArgs a{};
    a.chat = b.chat;
    a.code = b.d_code;
    a.out = out;
    a.s_base = b.d_base;
    a.s_dims = b.d_dims;
    a.blk = b.d_blk;
    a.s0 = ch.s0;
    a.s1 = ch.s1;
    a.rmask = 0;
    a.dmask = b.dest_mask;
    a.acc_in = false;
    a.qbase = b.d_qbase;
    for (int r : b.radii) {
        const bool dest = (b.dest_mask >> r) & 1u;
        if (!dest) a.rmask |= 1u << r;
        a.K[r] = static_cast<const char*>(b.arena) + ch.k_off[r];
        a.jbase[r] = dest ? 0 : ch.seg_begin[r];
        a.ncol[r] = dest ? ch.qn : ch.seg_end[r] - ch.seg_begin[r];
    }
    return a;
}

MarchArgs march_args(const fdirw_ctx* c, const Chunk& ch, int r) {
    const Batch& b = *c->batch;
    MarchArgs a{};
    a.g = b.grids[ch.s0];
    a.R = r;
    a.Rq = r;
    a.n_sub = c->n_sub;
    a.ax = reinterpret_cast<const float*>(c->coef[0]);
    a.ay = reinterpret_cast<const float*>(c->coef[1]);
    a.az = reinterpret_cast<const float*>(c->coef[2]);
    a.Q = static_cast<char*>(b.arena) + ch.k_off[r];
    a.store = c->store;
    a.sigma = c->sigma;
    if (c->flow) {                                    // convection: direction-dependent faces (mapping 5)
        a.bx = reinterpret_cast<const float*>(c->coefb[0]);
        a.by = reinterpret_cast<const float*>(c->coefb[1]);
        a.bz = reinterpret_cast<const float*>(c->coefb[2]);
    }
    a.src_begin = ch.seg_begin[r];
    a.src_end = ch.seg_end[r];
    a.list = b.d_list[r];
    a.nstruct = b.n;
    a.s_base = b.d_base;
    a.s_dims = b.d_dims;
    if ((b.dest_mask >> r) & 1u) {
        a.s_qbase = b.d_qbase;
        a.q_stride = ch.qn;
        a.src_major = 0;
    } else {
        a.q_stride = ch.seg_end[r] - ch.seg_begin[r];
        a.src_major = 1;
    }
    return a;
}

int ensure_arena(fdirw_ctx* c) {
    Batch& b = *c->batch;
    if (b.arena) return FDIRW_OK;
    uint64_t need = 0;
    for (const Chunk& ch : b.chunks) need = std::max(need, ch.k_bytes);
    if (need == 0) need = 256;
    const int rc = dalloc(c, &b.arena, need, "kernel cache");
    if (rc != FDIRW_OK) return rc;
    b.arena_bytes = need;
    c->q_bytes = need;
    return FDIRW_OK;
}

// Chooses the march mapping of every radius present (timing candidates on the first chunk holding that
// radius when autotuning); any kernels in the arena are invalid afterwards.
int ensure_parts(fdirw_ctx* c) {
    Batch& b = *c->batch;
    bool tuned = false;
    for (int r : b.radii) {
        if (r == 0 || b.parts[r] != 0) continue;
        for (const Chunk& ch : b.chunks) {
            if (ch.seg_end[r] == ch.seg_begin[r]) continue;
            FDIRW_CUDA(c, tune_march(march_args(c, ch, r), c->num_sms, c->parts_req, c->stream, &b.parts[r]));
            tuned = true;
            break;
        }
    }
    if (tuned) b.resident = -1;
    return FDIRW_OK;
}

// Timing events: inside a stream capture they must be external event nodes to be queryable after a
// graph launch; outside a capture that flag is not accepted.
cudaError_t record(cudaEvent_t ev, cudaStream_t st, bool captured) {
    return captured ? cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal) : cudaEventRecord(ev, st);
}

cudaError_t build_chunk(fdirw_ctx* c, int ci, cudaStream_t st, bool captured) {
    Batch& b = *c->batch;
    const Chunk& ch = b.chunks[ci];
    cudaError_t e = record(b.ev[4 * ci], st, captured);
    for (int r : b.radii) {                     // destination-indexed planes: zero where another radius owns the source
        if (e != cudaSuccess || r == 0 || !((b.dest_mask >> r) & 1u)) continue;
        e = cudaMemsetAsync(static_cast<char*>(b.arena) + ch.k_off[r], 0,
                            (size_t)wcells(r) * ch.qn * store_bytes(c->store), st);
    }
    for (int r : b.radii) {
        if (e != cudaSuccess) break;
        if (r == 0 || ch.seg_end[r] == ch.seg_begin[r]) continue;
        int used = 0;
        e = launch_march(march_args(c, ch, r), c->num_sms, b.parts[r], st, &used);
        c->parts_used = used;
    }
    if (e == cudaSuccess) e = record(b.ev[4 * ci + 1], st, captured);
    return e;
}

cudaError_t step_chunk(fdirw_ctx* c, int ci, const double* src, double* dst, int n_steps, cudaStream_t st,
                       bool captured) {
    Batch& b = *c->batch;
    const Chunk& ch = b.chunks[ci];
    VarArgs a = var_args(c, ch, dst);
    const int64_t nblk = b.blk[ch.s1] - b.blk[ch.s0];
    const bool fp32acc = c->accum == FDIRW_ACCUM_FP32;   // destination-indexed radii only; see the header
    const int Rm = c->R;
    cudaError_t e = cudaSuccess;
    const double* cur = src;
    for (int t = 0; t < n_steps && e == cudaSuccess; t++) {
        if (a.rmask) {
            scale_flat_kernel<<<grid_blocks(ch.c1 - ch.c0, 256), 256, 0, st>>>(cur, c->sigma, ch.c0, ch.c1, b.chat);
            e = cudaGetLastError();
        }
        for (int i = ch.s0; i < ch.s1 && e == cudaSuccess && b.dest_mask; i++)
            e = launch_scale(cur + b.base[i], c->sigma + b.base[i], b.grids[i], Rm, b.chat_pad + b.pbase[i],
                             fp32acc ? 2 : 1, st);
        const bool last = t + 1 == n_steps;
        if (e == cudaSuccess && last) e = record(b.ev[4 * ci + 2], st, captured);
        if (e != cudaSuccess) break;
        bool written = false;
        if (a.rmask && nblk > 0) {
            switch (c->store) {
                case Store::F32: gather_var_kernel<float><<<(unsigned)nblk, kTileX * kTileY, 0, st>>>(a); break;
                case Store::F16: gather_var_kernel<__half><<<(unsigned)nblk, kTileX * kTileY, 0, st>>>(a); break;
                default: gather_var_kernel<__nv_bfloat16><<<(unsigned)nblk, kTileX * kTileY, 0, st>>>(a); break;
            }
            e = cudaGetLastError();
            written = true;
        }
        if (e == cudaSuccess && b.dest_mask) {
            // Structures are independent: their destination-indexed gathers run as kAux parallel branches
            // of the graph (one structure alone fills a fraction of the GPU), each structure's radii in
            // ascending order on its branch, so every destination sums in the same order as before.
            const size_t sb = store_bytes(c->store);
            e = cudaEventRecord(b.afork, st);
            for (int k = 0; k < kAux && e == cudaSuccess; k++) e = cudaStreamWaitEvent(b.aux[k], b.afork, 0);
            for (int i = ch.s0; i < ch.s1 && e == cudaSuccess; i++) {
                cudaStream_t sx = b.aux[(i - ch.s0) % kAux];
                bool w = written;
                for (int r : b.radii) {
                    if (r == 0 || !((b.dest_mask >> r) & 1u)) continue;
                    const void* Q = static_cast<const char*>(a.K[r]) + (size_t)b.qbase[i] * sb;
                    e = fp32acc ? launch_gather_part_fp32(Q, c->store, ch.qn,
                                                          reinterpret_cast<const float*>(b.chat_pad + b.pbase[i]), Rm,
                                                          b.grids[i], r, w, dst + b.base[i], sx)
                                : launch_gather_part(Q, c->store, ch.qn, b.chat_pad + b.pbase[i], Rm, b.grids[i], r, w,
                                                     dst + b.base[i], sx);
                    if (e != cudaSuccess) break;
                    w = true;
                }
            }
            for (int k = 0; k < kAux && e == cudaSuccess; k++) {
                e = cudaEventRecord(b.ajoin[k], b.aux[k]);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(st, b.ajoin[k], 0);
            }
            written = true;
        }
        if (e == cudaSuccess && last) e = record(b.ev[4 * ci + 3], st, captured);
        if (e == cudaSuccess && fp32acc) e = launch_seg_restore(dst, b.d_base, ch.s0, ch.s1, b.seg_part, b.seg_fix, st);
        cur = dst;
    }
    return e;
}

// The device work of one fdirw_step call (all chunks), issued on the capture stream.  The timing events
// are recorded as external event nodes so that they can be queried after each graph launch.
cudaError_t issue_all(fdirw_ctx* c, const double* src, double* dst, int n_steps, bool build_single) {
    Batch& b = *c->batch;
    cudaError_t e = cudaSuccess;
    const int nch = (int)b.chunks.size();
    // FDIRW_ACCUM_FP32: every structure's FP64 total of the call's input, the target of its restoration.
    if (c->accum == FDIRW_ACCUM_FP32) e = launch_seg_target(src, b.d_base, 0, b.n, b.seg_part, b.seg_fix, b.gs);
    for (int ci = 0; ci < nch && e == cudaSuccess; ci++) {
        const bool build = nch > 1 || build_single;
        if (build) e = build_chunk(c, ci, b.gs, true);
        if (e == cudaSuccess) e = step_chunk(c, ci, src, dst, n_steps, b.gs, true);
    }
    return e;
}

void drop_graph(Batch& b) {
    if (b.exec) cudaGraphExecDestroy(b.exec);
    b.exec = nullptr;
    b.g_steps = -1;
}

int run_graph(fdirw_ctx* c, const double* src, double* dst, int n_steps) {
    Batch& b = *c->batch;
    const int nch = (int)b.chunks.size();
    const bool build_single = nch == 1 && b.resident != 0;
    if (!(b.exec && b.g_src == src && b.g_dst == dst && b.g_steps == n_steps && b.g_build == build_single)) {
        drop_graph(b);
        FDIRW_CUDA(c, cudaStreamBeginCapture(b.gs, cudaStreamCaptureModeThreadLocal));
        const cudaError_t e = issue_all(c, src, dst, n_steps, build_single);
        cudaGraph_t graph = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(b.gs, &graph);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return fail(c, FDIRW_ERR_CUDA, cuda_msg("capturing the batch step", e != cudaSuccess ? e : e2));
        }
        const cudaError_t e3 = cudaGraphInstantiate(&b.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e3 != cudaSuccess) { b.exec = nullptr; return fail(c, FDIRW_ERR_CUDA, cuda_msg("cudaGraphInstantiate", e3)); }
        b.g_src = src;
        b.g_dst = dst;
        b.g_steps = n_steps;
        b.g_build = build_single;
    }
    FDIRW_CUDA(c, cudaEventRecord(b.fork, c->stream));
    FDIRW_CUDA(c, cudaStreamWaitEvent(b.gs, b.fork, 0));
    FDIRW_CUDA(c, cudaGraphLaunch(b.exec, b.gs));
    FDIRW_CUDA(c, cudaEventRecord(b.join, b.gs));
    FDIRW_CUDA(c, cudaStreamWaitEvent(c->stream, b.join, 0));
    b.graph_launches++;
    for (int ci = 0; ci < nch; ci++) {
        b.built[ci] = (nch > 1 || build_single) ? 1 : 0;
        b.stepped[ci] = 1;
    }
    if (nch > 1 || build_single) b.resident = nch - 1;
    return FDIRW_OK;
}

// Sum over the cells of a structure of their clipped window sizes for the cell's own radius.
double window_cells_of(const Grid& g, const int8_t* R) {
    double s = 0.0;
    for (int z = 0; z < g.nz; z++)
        for (int y = 0; y < g.ny; y++)
            for (int x = 0; x < g.nx; x++) {
                const int r = R[x + (int64_t)g.nx * (y + (int64_t)g.ny * z)];
                auto ext = [r](int v, int n) { return (double)(std::min(v + r, n - 1) - std::max(v - r, 0) + 1); };
                s += ext(x, g.nx) * ext(y, g.ny) * ext(z, g.nz);
            }
    return s;
}

void release_batch(fdirw_ctx* c) {
    Batch* b = c->batch;
    if (!b) return;
    drop_graph(*b);
    void* p;
    p = b->d_base; dfree(p);
    p = b->d_dims; dfree(p);
    p = b->d_blk; dfree(p);
    for (auto& l : b->d_list) { p = l; dfree(p); l = nullptr; }
    p = b->d_code; dfree(p);
    p = b->d_qbase; dfree(p);
    dfree(b->arena);
    p = b->chat; dfree(p);
    p = b->chat_pad; dfree(p);
    p = b->seg_part; dfree(p);
    p = b->seg_fix; dfree(p);
    for (auto& e : b->ev) if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->join) cudaEventDestroy(b->join);
    if (b->gs) cudaStreamDestroy(b->gs);
    if (b->afork) cudaEventDestroy(b->afork);
    for (int k = 0; k < kAux; k++) {
        if (b->aux[k]) cudaStreamDestroy(b->aux[k]);
        if (b->ajoin[k]) cudaEventDestroy(b->ajoin[k]);
    }
    delete b;
    c->batch = nullptr;
}

}  // namespace

// ------------------------------------------------------------------------------------------ entry points

int batch_kernels(fdirw_ctx* c) {
    Batch& b = *c->batch;
    if (c->R == 0 || c->n_sub == 0) { c->kernels_ready = true; return FDIRW_OK; }
    if (b.chunks.size() != 1) return FDIRW_OK;        // built chunk by chunk inside fdirw_step
    int rc = ensure_arena(c);
    if (rc != FDIRW_OK) return rc;
    if ((rc = ensure_parts(c)) != FDIRW_OK) return rc;
    FDIRW_CUDA(c, cudaEventRecord(b.fork, c->stream));
    FDIRW_CUDA(c, cudaStreamWaitEvent(b.gs, b.fork, 0));
    FDIRW_CUDA(c, build_chunk(c, 0, b.gs, false));
    FDIRW_CUDA(c, cudaEventRecord(b.join, b.gs));
    FDIRW_CUDA(c, cudaStreamWaitEvent(c->stream, b.join, 0));
    b.built[0] = 1;
    b.stepped[0] = 0;
    b.resident = 0;
    c->kernels_ready = true;
    return FDIRW_OK;
}

int batch_step(fdirw_ctx* c, const double* c_in, double* c_out, int32_t n_steps, double* mass_out) {
    Batch& b = *c->batch;
    const Kind kin = classify(c_in, c->device), kout = classify(c_out, c->device);
    if (kin == Kind::Foreign || kout == Kind::Foreign)
        return fail(c, FDIRW_ERR_ARG, "c_in/c_out are device memory of another device");
    const size_t bytes = (size_t)c->g.n * 8;
    const double* src = c_in;
    if (kin == Kind::Host) {
        FDIRW_CUDA(c, cudaMemcpyAsync(c->cbuf, c_in, bytes, cudaMemcpyHostToDevice, c->stream));
        src = c->cbuf;
    }
    double* dst = kout == Kind::Device ? c_out : c->cbuf;
    if (mass_out) {
        FDIRW_CUDA(c, launch_mass(src, c->g.n, c->partials, c->dmass, c->stream));
        FDIRW_CUDA(c, cudaMemcpyAsync(&c->mass_in, c->dmass, 8, cudaMemcpyDeviceToHost, c->stream));
    }
    const bool identity = c->R == 0 || c->n_sub == 0 || n_steps == 0;
    if (identity) {
        if (dst != src) FDIRW_CUDA(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, c->stream));
    } else {
        int rc = ensure_arena(c);
        if (rc != FDIRW_OK) return rc;
        if ((rc = ensure_parts(c)) != FDIRW_OK) return rc;
        if ((rc = run_graph(c, src, dst, n_steps)) != FDIRW_OK) return rc;
        c->kernels_ready = b.chunks.size() == 1;
    }
    if (mass_out) {
        FDIRW_CUDA(c, launch_mass(dst, c->g.n, c->partials, c->dmass, c->stream));
        FDIRW_CUDA(c, cudaMemcpyAsync(&c->mass_out, c->dmass, 8, cudaMemcpyDeviceToHost, c->stream));
    }
    if (kout == Kind::Host) FDIRW_CUDA(c, cudaMemcpyAsync(c_out, dst, bytes, cudaMemcpyDeviceToHost, c->stream));
    if (mass_out || kout == Kind::Host) FDIRW_CUDA(c, cudaStreamSynchronize(c->stream));
    if (mass_out) *mass_out = c->mass_out;
    return FDIRW_OK;
}

int batch_read_kernels(fdirw_ctx* c, const int64_t* sources, int64_t n, double* out) {
    Batch& b = *c->batch;
    const int Rm = c->R;
    const int64_t W = wcells(Rm);
    if (c->n_sub == 0 || Rm == 0) {
        // every kernel is the identity
        for (int64_t q = 0; q < n; q++) {
            std::fill(out + q * W, out + (q + 1) * W, 0.0);
            out[q * W + W / 2] = 1.0;
        }
        return FDIRW_OK;
    }
    if (b.chunks.size() != 1 || b.resident != 0)
        return fail(c, FDIRW_ERR_STATE, "kernels of a batch are readable only when they all fit (one chunk) and are built");
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
    const VarArgs a = var_args(c, b.chunks[0], nullptr);
    FDIRW_CUDA(c, cudaMemcpyAsync(c->dsrc, sources, (size_t)n * 8, cudaMemcpyHostToDevice, c->stream));
    const int blocks = grid_blocks(n * W, 256);
    switch (c->store) {
        case Store::F32: read_var_kernel<float><<<blocks, 256, 0, c->stream>>>(a, c->sigma, b.n, Rm, c->dsrc, n, c->dkout); break;
        case Store::F16: read_var_kernel<__half><<<blocks, 256, 0, c->stream>>>(a, c->sigma, b.n, Rm, c->dsrc, n, c->dkout); break;
        default: read_var_kernel<__nv_bfloat16><<<blocks, 256, 0, c->stream>>>(a, c->sigma, b.n, Rm, c->dsrc, n, c->dkout); break;
    }
    FDIRW_CUDA(c, cudaGetLastError());
    FDIRW_CUDA(c, cudaMemcpyAsync(out, c->dkout, (size_t)(n * W) * 8, cudaMemcpyDeviceToHost, c->stream));
    FDIRW_CUDA(c, cudaStreamSynchronize(c->stream));
    return FDIRW_OK;
}

int batch_info(fdirw_ctx* c, fdirw_info* out) {
    Batch& b = *c->batch;
    out->n_structures = b.n;
    out->n_chunks = (int32_t)b.chunks.size();
    out->window_R_min = b.Rmin;
    out->graph_launches = b.graph_launches;
    out->dest_indexed_radii = (int32_t)b.dest_mask;
    float km = 0.f, gm = 0.f;
    bool anyk = false, anyg = false;
    for (size_t ci = 0; ci < b.chunks.size(); ci++) {
        float ms = 0.f;
        if (b.built[ci]) {
            FDIRW_CUDA(c, cudaEventSynchronize(b.ev[4 * ci + 1]));
            FDIRW_CUDA(c, cudaEventElapsedTime(&ms, b.ev[4 * ci], b.ev[4 * ci + 1]));
            km += ms;
            anyk = true;
        }
        if (b.stepped[ci]) {
            FDIRW_CUDA(c, cudaEventSynchronize(b.ev[4 * ci + 3]));
            FDIRW_CUDA(c, cudaEventElapsedTime(&ms, b.ev[4 * ci + 2], b.ev[4 * ci + 3]));
            gm += ms;
            anyg = true;
        }
    }
    out->kernels_ms = anyk ? km : 0.f;
    out->last_gather_ms = anyg ? gm : 0.f;
    return FDIRW_OK;
}

void batch_release(fdirw_ctx* c) { release_batch(c); }

void batch_structures(const fdirw_ctx* c, std::vector<Grid>& grids, std::vector<int64_t>& base,
                      std::vector<double>& lams, std::vector<double>& hs) {
    const Batch& b = *c->batch;
    grids = b.grids;
    base.assign(b.base.begin(), b.base.end() - 1);
    lams = b.lams;
    hs = b.hs;
}

void batch_invalidate(fdirw_ctx* c) {
    Batch& b = *c->batch;
    drop_graph(b);                                    // its launches carry the old march arguments
    b.resident = -1;                                  // no chunk's kernels are current
    for (auto& v : b.built) v = 0;
    c->kernels_ready = false;
}

}  // namespace fdirw

using fdirw::Batch;
using fdirw::Chunk;

extern "C" {

int fdirw_create_batch(int32_t n, const fdirw_grid* grids, const double* const* D_maps, double dt_macro,
                       int32_t R_min, int32_t R_max, int32_t n_sub, const fdirw_opts* opts, fdirw_ctx** out) {
    if (!out) return fail(nullptr, FDIRW_ERR_ARG, "NULL out");
    *out = nullptr;
    if (n < 1 || !grids || !D_maps) return fail(nullptr, FDIRW_ERR_ARG, "need n >= 1 grids and D maps");
    int64_t total = 0;
    for (int i = 0; i < n; i++) {
        if (!grid_ok(&grids[i])) return fail(nullptr, FDIRW_ERR_ARG, "invalid grid of structure " + std::to_string(i));
        if (!D_maps[i]) return fail(nullptr, FDIRW_ERR_ARG, "NULL D map of structure " + std::to_string(i));
        if ((reinterpret_cast<uintptr_t>(D_maps[i]) & 7u) != 0)
            return fail(nullptr, FDIRW_ERR_ARG, "D map of structure " + std::to_string(i) + " is not 8-byte aligned");
        total += (int64_t)grids[i].nx * grids[i].ny * grids[i].nz;
        if (total >= fdirw::kMaxBatchCells)
            return fail(nullptr, FDIRW_ERR_ARG, "a batch holds fewer than 2^28 cells in total");
    }
    if (!(std::isfinite(dt_macro) && dt_macro >= 0.0)) return fail(nullptr, FDIRW_ERR_ARG, "dt_macro must be finite and >= 0");
    if (R_min < 0 || R_max > fdirw::kMaxR || R_min > R_max)
        return fail(nullptr, FDIRW_ERR_ARG, "need 0 <= R_min <= R_max <= " + std::to_string(fdirw::kMaxR));
    if (n_sub < 0) return fail(nullptr, FDIRW_ERR_ARG, "n_sub must be >= 0");
    fdirw_opts o{FDIRW_FP32, -1, nullptr, 0, 0, 0};
    if (opts) o = *opts;
    if (o.prec < FDIRW_FP32 || o.prec > FDIRW_FP32_STORE_BF16)
        return fail(nullptr, FDIRW_ERR_ARG, "a batch needs an FP32-march precision (FP32, FP16 or BF16 storage)");
    if (o.march_parts < 0 || o.march_parts > 7) return fail(nullptr, FDIRW_ERR_ARG, "march_parts must be in [0, 7]");
    if (o.accum != FDIRW_ACCUM_FF && o.accum != FDIRW_ACCUM_FP32) return fail(nullptr, FDIRW_ERR_ARG, "unknown accum");

    DeviceGuard dg(o.device);
    if (!dg.ok) return fail(nullptr, FDIRW_ERR_CUDA, "cannot select CUDA device " + std::to_string(o.device));
    fdirw_ctx* c = new fdirw_ctx();
    cudaGetDevice(&c->device);
    c->batch = new Batch();
    Batch& b = *c->batch;
    c->stream = reinterpret_cast<cudaStream_t>(o.stream);
    c->mem_limit = o.mem_limit;
    c->parts_req = o.march_parts;
    c->accum = o.accum;
    c->g = fdirw::Grid{(int)std::min<int64_t>(total, 0x7fffffff), 1, 1, total};   // flat view for fields
    c->h = grids[0].h;
    c->dt_macro = dt_macro;
    c->R = R_max;
    c->n_sub = n_sub;
    c->prec = o.prec;
    c->store = o.prec == FDIRW_FP32 ? fdirw::Store::F32 : o.prec == FDIRW_FP32_STORE_FP16 ? fdirw::Store::F16
                                                                                          : fdirw::Store::BF16;
    c->dt_sub = n_sub > 0 ? dt_macro / n_sub : 0.0;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    b.n = n;
    b.Rmin = R_min;
    b.Rmax = R_max;

    auto bail = [&](int rc) {
        std::string msg = c->err;
        if (c->stream) cudaStreamSynchronize(c->stream); else cudaDeviceSynchronize();
        fdirw::batch_release(c);
        for (auto& p : c->coef) dfree(p);
        void* p;
        p = c->sigma; dfree(p);
        p = c->cbuf; dfree(p);
        p = c->partials; dfree(p);
        p = c->dmass; dfree(p);
        p = c->Dd; dfree(p);
        for (auto& e : c->ev) if (e) cudaEventDestroy(e);
        delete c;
        return fail(nullptr, rc, msg);
    };
    auto cuda_bail = [&](const char* what, cudaError_t e) {
        c->err = cuda_msg(what, e);
        return bail(FDIRW_ERR_CUDA);
    };

    // Layout of the concatenation.
    b.base.assign(n + 1, 0);
    b.blk.assign(n + 1, 0);
    std::vector<int4> dims(n);
    int64_t maxn = 0;
    for (int i = 0; i < n; i++) {
        const fdirw::Grid g{grids[i].nx, grids[i].ny, grids[i].nz, (int64_t)grids[i].nx * grids[i].ny * grids[i].nz};
        b.grids.push_back(g);
        b.hs.push_back(grids[i].h);
        b.lams.push_back(c->dt_sub / (grids[i].h * grids[i].h));
        b.base[i + 1] = b.base[i] + g.n;
        const int64_t tiles = (int64_t)((g.nx + fdirw::kTileX - 1) / fdirw::kTileX) *
                              ((g.ny + fdirw::kTileY - 1) / fdirw::kTileY) * g.nz;
        b.blk[i + 1] = b.blk[i] + tiles;
        dims[i] = make_int4(g.nx, g.ny, g.nz, 0);
        maxn = std::max(maxn, g.n);
    }
    c->lam = b.lams[0];
    const uint64_t N = (uint64_t)total;
    int rc;
    if ((rc = dalloc(c, reinterpret_cast<void**>(&b.d_base), (n + 1) * 8ull, "structure table")) != FDIRW_OK) return bail(rc);
    if ((rc = dalloc(c, reinterpret_cast<void**>(&b.d_blk), (n + 1) * 8ull, "structure table")) != FDIRW_OK) return bail(rc);
    if ((rc = dalloc(c, reinterpret_cast<void**>(&b.d_dims), n * 16ull, "structure table")) != FDIRW_OK) return bail(rc);
    cudaError_t e = cudaMemcpyAsync(b.d_base, b.base.data(), (n + 1) * 8ull, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.d_blk, b.blk.data(), (n + 1) * 8ull, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.d_dims, dims.data(), n * 16ull, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_bail("copy structure tables", e);

    // D, face coefficients (per structure, with its own lam), radius map.
    if ((rc = dalloc(c, reinterpret_cast<void**>(&c->Dd), N * 8, "D copy")) != FDIRW_OK) return bail(rc);
    for (int a = 0; a < 3; a++)
        if ((rc = dalloc(c, &c->coef[a], N * 4, "coefficients")) != FDIRW_OK) return bail(rc);
    double* g3 = nullptr;
    unsigned long long* flags = nullptr;
    int8_t* dR = nullptr;
    if ((rc = dalloc(c, reinterpret_cast<void**>(&g3), (uint64_t)maxn * 24, "conductance staging")) != FDIRW_OK) return bail(rc);
    auto free_tmp = [&]() {
        void* p = g3; if (p) { dfree(p); c->allocated -= (uint64_t)maxn * 24; } g3 = nullptr;
        p = flags; if (p) { dfree(p); c->allocated -= 16; } flags = nullptr;
        p = dR; if (p) { dfree(p); c->allocated -= N; } dR = nullptr;
    };
    if ((rc = dalloc(c, reinterpret_cast<void**>(&flags), 16, "flags")) != FDIRW_OK) { free_tmp(); return bail(rc); }
    if ((rc = dalloc(c, reinterpret_cast<void**>(&dR), N, "radius map")) != FDIRW_OK) { free_tmp(); return bail(rc); }
    double worst = 0.0;
    for (int i = 0; i < n && e == cudaSuccess; i++) {
        const fdirw::Grid& g = b.grids[i];
        double* Di = c->Dd + b.base[i];
        e = cudaMemcpyAsync(Di, D_maps[i], (size_t)g.n * 8, cudaMemcpyDefault, c->stream);
        unsigned long long h[2] = {0ull, 0ull};
        if (e == cudaSuccess) e = cudaMemsetAsync(flags, 0, 16, c->stream);
        if (e == cudaSuccess) e = fdirw::launch_conductance(Di, g, g3, g3 + maxn, g3 + 2 * maxn, flags, flags + 1, c->stream);
        for (int a = 0; a < 3 && e == cudaSuccess; a++)
            e = fdirw::launch_coef_f32(g3 + a * maxn, b.lams[i], g.n, reinterpret_cast<float*>(c->coef[a]) + b.base[i], c->stream);
        if (e == cudaSuccess) {
            fdirw::radius_kernel<<<fdirw::grid_blocks(g.n, 256), 256, 0, c->stream>>>(Di, g.n, dt_macro, b.hs[i], R_min, R_max,
                                                                             dR + b.base[i]);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(h, flags, 16, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) break;
        if (h[1] != 0ull) {
            free_tmp();
            c->err = "D map of structure " + std::to_string(i) + " holds NaN, infinite or negative values";
            return bail(FDIRW_ERR_ARG);
        }
        double m;
        std::memcpy(&m, &h[0], 8);
        if (b.lams[i] * m > 1.0 + 1e-12) {
            free_tmp();
            char buf[256];
            std::snprintf(buf, sizeof buf, "unstable: structure %d has dt_sub*max(sum g)/h^2 = %.17g > 1", i, b.lams[i] * m);
            c->err = buf;
            return bail(FDIRW_ERR_UNSTABLE);
        }
        if (b.lams[i] * m >= worst) { worst = b.lams[i] * m; c->max_face_sum = m; }
    }
    if (e != cudaSuccess) { free_tmp(); return cuda_bail("batch setup", e); }

    // Buckets (host): code(s) = (R << 28) | position in the radius-R list, lists in global cell order.
    std::vector<int8_t> Rh(N);
    e = cudaMemcpy(Rh.data(), dR, N, cudaMemcpyDeviceToHost);
    free_tmp();
    if (e != cudaSuccess) return cuda_bail("copy radius map", e);
    std::vector<uint32_t> code(N);
    std::vector<int64_t> lists[fdirw::kMaxR + 1];
    for (int r = 0; r <= fdirw::kMaxR; r++) b.before[r].assign(n + 1, 0);
    c->window_cells = 0.0;
    for (int i = 0; i < n; i++) {
        for (int r = 0; r <= fdirw::kMaxR; r++) b.before[r][i] = (int64_t)lists[r].size();
        for (int64_t s = b.base[i]; s < b.base[i + 1]; s++) {
            const int r = Rh[s];
            code[s] = ((uint32_t)r << fdirw::kCodeShift) | (uint32_t)lists[r].size();
            lists[r].push_back(s);
        }
        c->window_cells += fdirw::window_cells_of(b.grids[i], Rh.data() + b.base[i]);
    }
    for (int r = 0; r <= fdirw::kMaxR; r++) {
        b.before[r][n] = (int64_t)lists[r].size();
        b.count[r] = (int64_t)lists[r].size();
        if (b.count[r] > 0) b.radii.push_back(r);
        if (r > 0 && b.count[r] > 0 && (double)b.count[r] >= fdirw::kDestFraction * (double)total)
            b.dest_mask |= 1u << r;
    }
    if ((rc = dalloc(c, reinterpret_cast<void**>(&b.d_code), N * 4, "bucket codes")) != FDIRW_OK) return bail(rc);
    e = cudaMemcpy(b.d_code, code.data(), N * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_bail("copy bucket codes", e);
    for (int r : b.radii) {
        if (r == 0) continue;
        if ((rc = dalloc(c, reinterpret_cast<void**>(&b.d_list[r]), (uint64_t)b.count[r] * 8, "bucket list")) != FDIRW_OK)
            return bail(rc);
        e = cudaMemcpy(b.d_list[r], lists[r].data(), (size_t)b.count[r] * 8, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_bail("copy bucket list", e);
    }

    // Field buffers.
    if ((rc = dalloc(c, reinterpret_cast<void**>(&c->sigma), N * 8, "sigma")) != FDIRW_OK) return bail(rc);
    if ((rc = dalloc(c, reinterpret_cast<void**>(&b.chat), N * 8, "scaled field")) != FDIRW_OK) return bail(rc);
    if ((rc = dalloc(c, reinterpret_cast<void**>(&c->cbuf), N * 8, "field staging")) != FDIRW_OK) return bail(rc);
    if ((rc = dalloc(c, reinterpret_cast<void**>(&c->partials), fdirw::kMassBlocks * 8, "mass partials")) != FDIRW_OK) return bail(rc);
    if ((rc = dalloc(c, reinterpret_cast<void**>(&c->dmass), 8, "mass")) != FDIRW_OK) return bail(rc);
    fdirw::fill_kernel<<<fdirw::grid_blocks((int64_t)N, 256), 256, 0, c->stream>>>(c->sigma, (int64_t)N, 1.0);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_bail("fill sigma", e);
    if (b.dest_mask) {
        // Padded scaled field: each structure with a zero halo of R_max cells (written once, never touched).
        b.pbase.assign(n + 1, 0);
        for (int i = 0; i < n; i++) {
            const fdirw::Pad pd = fdirw::make_pad(b.grids[i], R_max);
            b.pbase[i + 1] = b.pbase[i] + pd.n;
        }
        const uint64_t pbytes = (uint64_t)b.pbase[n] * 8;
        if ((rc = dalloc(c, reinterpret_cast<void**>(&b.chat_pad), pbytes, "padded scaled field")) != FDIRW_OK) return bail(rc);
        if ((e = cudaMemsetAsync(b.chat_pad, 0, pbytes, c->stream)) != cudaSuccess) return cuda_bail("zero padded field", e);
    }
    if ((rc = dalloc(c, reinterpret_cast<void**>(&b.d_qbase), (uint64_t)n * 8, "structure table")) != FDIRW_OK) return bail(rc);
    if (c->accum == FDIRW_ACCUM_FP32) {
        if ((rc = dalloc(c, reinterpret_cast<void**>(&b.seg_part), (uint64_t)n * 2 * fdirw::kSegBlocks * 8,
                         "mass restoration partials")) != FDIRW_OK) return bail(rc);
        if ((rc = dalloc(c, reinterpret_cast<void**>(&b.seg_fix), (uint64_t)n * 2 * 8, "mass restoration")) != FDIRW_OK)
            return bail(rc);
    }

    // Chunks: consecutive structures whose kernels fit the budget together.
    const int sb = fdirw::store_bytes(c->store);
    auto slot = [&](int i) { return (b.grids[i].n + 15) / 16 * 16; };   // 16-aligned destination columns
    auto struct_bytes = [&](int i, int r) -> uint64_t {
        if (r == 0) return 0;
        const int64_t cols = (b.dest_mask >> r) & 1u ? slot(i) : b.before[r][i + 1] - b.before[r][i];
        return (uint64_t)cols * (uint64_t)fdirw::wcells(r) * sb;
    };
    b.qbase.assign(n, 0);
    uint64_t budget;
    if (c->mem_limit) {
        budget = c->mem_limit > c->allocated ? c->mem_limit - c->allocated : 0;
    } else {
        size_t fr = 0, tot = 0;
        if ((e = cudaMemGetInfo(&fr, &tot)) != cudaSuccess) return cuda_bail("cudaMemGetInfo", e);
        const uint64_t reserve = std::max<uint64_t>(1ull << 30, tot / 50);
        budget = fr > reserve ? fr - reserve : 0;
    }
    budget = budget > 256ull * (fdirw::kMaxR + 1) ? budget - 256ull * (fdirw::kMaxR + 1) : 0;
    int i = 0;
    while (i < n) {
        Chunk ch;
        ch.s0 = i;
        uint64_t used = 0;
        while (i < n) {
            uint64_t add = 0;
            for (int r : b.radii) add += struct_bytes(i, r);
            if (used + add > budget && i > ch.s0) break;
            if (used + add > budget) {
                c->err = "the kernels of structure " + std::to_string(i) + " (" + std::to_string(add) +
                         " bytes) do not fit the device memory budget (" + std::to_string(budget) + " bytes)";
                return bail(FDIRW_ERR_NOMEM);
            }
            used += add;
            i++;
        }
        ch.s1 = i;
        ch.c0 = b.base[ch.s0];
        ch.c1 = b.base[ch.s1];
        ch.qn = 0;
        for (int k = ch.s0; k < ch.s1; k++) {
            b.qbase[k] = ch.qn;
            ch.qn += slot(k);
        }
        uint64_t off = 0;
        for (int r : b.radii) {
            ch.seg_begin[r] = b.before[r][ch.s0];
            ch.seg_end[r] = b.before[r][ch.s1];
            ch.k_off[r] = off;
            const int64_t cols = (b.dest_mask >> r) & 1u ? ch.qn : ch.seg_end[r] - ch.seg_begin[r];
            if (r > 0) off += fdirw::align256((uint64_t)cols * fdirw::wcells(r) * sb);
        }
        ch.k_bytes = off;
        b.chunks.push_back(ch);
    }
    if ((e = cudaMemcpyAsync(b.d_qbase, b.qbase.data(), (size_t)n * 8, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess)
        return cuda_bail("copy structure tables", e);
    b.built.assign(b.chunks.size(), 0);
    b.stepped.assign(b.chunks.size(), 0);
    b.ev.assign(4 * b.chunks.size(), nullptr);
    for (auto& ev : b.ev)
        if ((e = cudaEventCreate(&ev)) != cudaSuccess) return cuda_bail("cudaEventCreate", e);
    if ((e = cudaEventCreateWithFlags(&b.fork, cudaEventDisableTiming)) != cudaSuccess) return cuda_bail("cudaEventCreate", e);
    if ((e = cudaEventCreateWithFlags(&b.join, cudaEventDisableTiming)) != cudaSuccess) return cuda_bail("cudaEventCreate", e);
    if ((e = cudaStreamCreateWithFlags(&b.gs, cudaStreamNonBlocking)) != cudaSuccess) return cuda_bail("cudaStreamCreate", e);
    if ((e = cudaEventCreateWithFlags(&b.afork, cudaEventDisableTiming)) != cudaSuccess) return cuda_bail("cudaEventCreate", e);
    for (int k = 0; k < fdirw::kAux; k++) {
        if ((e = cudaStreamCreateWithFlags(&b.aux[k], cudaStreamNonBlocking)) != cudaSuccess) return cuda_bail("cudaStreamCreate", e);
        if ((e = cudaEventCreateWithFlags(&b.ajoin[k], cudaEventDisableTiming)) != cudaSuccess) return cuda_bail("cudaEventCreate", e);
    }
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_bail("batch setup", e);
    *out = c;
    return FDIRW_OK;
}

int fdirw_read_radius(fdirw_ctx* c, int32_t* out) {
    if (!c || !out) return fail(c, FDIRW_ERR_ARG, "NULL context or out");
    if (!c->batch) {
        for (int64_t s = 0; s < c->g.n; s++) out[s] = c->R;
        return FDIRW_OK;
    }
    DeviceGuard dg(c->device);
    std::vector<uint32_t> code((size_t)c->g.n);
    FDIRW_CUDA(c, cudaStreamSynchronize(c->stream));
    FDIRW_CUDA(c, cudaMemcpy(code.data(), c->batch->d_code, (size_t)c->g.n * 4, cudaMemcpyDeviceToHost));
    for (int64_t s = 0; s < c->g.n; s++) out[s] = (int32_t)(code[s] >> fdirw::kCodeShift);
    return FDIRW_OK;
}

}  // extern "C"
