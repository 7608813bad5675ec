// Learned surrogate of the per-source spreading kernel (the network itself has no counterpart in the
// paper; what it predicts is the column of p of Sec. 3.1, and the explicit FD march stays its fallback).
//
// Network (per source s, a 17^3 patch centred on s): features [log10 D / 8 + 1, domain mask, source
// marker, o_x / 8, o_y / 8, o_z / 8, |o|^2 / 256 with o the offset from the source] (16 channels, 9 zero)
// -> 4 x { conv3d 3^3, 16 -> 16 channels, zero padding, + bias } with
// ReLU after layers 1-3 -> head y = exp(z_4[channel 0]) on in-domain cells.  Gate: accept the prediction
// when |sum y - 1| <= 1e-3 (FP64); the stored kernel is then renormalised like the FD kernels.
//
// Tensor-core convolution (conv_kernel): implicit GEMM per 128-voxel tile, M = 128 voxels, N = 16 output
// channels, K = 16 input channels per tap, 27 tcgen05.mma (kind::f16, BF16 in, FP32 accumulate in TMEM)
// per tile.  Activations are kept in a zero-halo 19^3 volume split into two 8-channel halves, so every
// voxel row is 16 bytes and each of the 27 tap-shifted views of a plane ring is a valid K-major,
// no-swizzle operand (LBO = distance between the halves, SBO = 8 rows) -- no im2col copy.  One thread
// issues the MMAs, tcgen05.commit signals an mbarrier, and 4 warps drain the accumulators with
// tcgen05.ld.  The same kernel runs the input gradient (flipped, transposed taps, ReLU mask in the
// epilogue).  The weight and bias gradients (wgrad_kernel) reduce over voxel rows on the tensor cores too:
// the dz-shifted activation rows and a ones group stacked into M, the (dx, dy)-shifted gradient rows into
// N = 144, both MN-major, gathered by tensor copies through overlapping tensor-map views.
#include "ctx.h"
#include "tc.cuh"

#include <cuda.h>   // CUtensorMap and its encoding enums (the encoder is fetched from the driver at run time)
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

using fdirw::Store;

namespace fdirw {
namespace net {

constexpr int SP = 17, SH = 8, PP = 19, PLANE = PP * PP, VOL = PP * PLANE, KV = SP * SP * SP;
constexpr int GUARD = 64, ROWS = GUARD + VOL + GUARD;            // rows per 8-channel half of a patch
constexpr int64_t PATCH = 2 * (int64_t)ROWS * 8;                   // bf16 elements per patch activation
constexpr int NL = 4, C = 16, TAPS = 27;
constexpr int NW = NL * TAPS * C * C;                              // weights [layer][tap][co][ci]
constexpr int NPARAM = NW + NL * C;                                // + biases [layer][co]
constexpr int WCAN = TAPS * C * C;                                 // bf16 per layer, canonical layout
constexpr int MAX_BATCH = 1024;
constexpr uint64_t WAIT_NS = 2000000000ull;                        // default MMA-wait budget: 2 s
constexpr int NTILE = 3;                                           // 128-row tiles per plane (384 >= 361)
constexpr int HALO_ROWS = PP + 1;                                  // rows a tap can reach beyond a tile (dy, dx)
constexpr int TROWS = 128 + 2 * HALO_ROWS;                         // plane rows one tile reads: 168
constexpr int NSLOT = 16;                                          // plane slots of the shared-memory ring
constexpr int RROWS = NSLOT * TROWS;                               // ring rows per 8-channel half
constexpr int NZ = 3;                                              // z taps stacked into one MMA's N
constexpr int N48 = NZ * C;                                        // MMA N: 3 output planes x 16 channels
constexpr int TAPS_XY = 9;                                         // (dy, dx) taps: MMAs per input plane
constexpr int ACC_PLANES = PP;                                     // accumulators of padded planes 0..18
constexpr int EPI_SETS = 2;                                        // epilogue warp sets (alternate output planes)
constexpr int CONV_THREADS = 64 + EPI_SETS * 128;                  // producer, MMA and the epilogue warps
constexpr int NBAR = 2 * NSLOT + 2 * SP + 1;                       // ring full/empty, plane acc full/empty, drain
constexpr size_t CONV_SMEM_USED = (size_t)2 * RROWS * 16 + (size_t)WCAN * 2 + NBAR * 8 + 16;
// One CTA per SM (it allocates all 512 TMEM columns): the shared-memory request keeps a second one off.
constexpr size_t CONV_SMEM = CONV_SMEM_USED > 120 * 1024 ? CONV_SMEM_USED : 120 * 1024;
constexpr double GATE_TOL = 1e-3;

enum Mode { FWD_RELU = 0, FWD_HEAD = 1, DGRAD = 2 };

struct ConvArgs {
    const __nv_bfloat16* in;        // [batch][PATCH]
    __nv_bfloat16* out;             // [batch][PATCH] (FWD_RELU, DGRAD)
    float* zhead;                   // [batch][KV]    (FWD_HEAD)
    const __nv_bfloat16* mask_act;  // [batch][PATCH] (DGRAD: relu mask = this activation > 0)
    const __nv_bfloat16* w;         // [TAPS][512 B] canonical layout of one layer
    const float* bias;              // [C]
    int batch;
    int mode;
    int* err;                       // 1: a wait gave up with nothing left in flight; 2: MMAs may still run
    uint64_t wait_ns;               // budget of each wait on the MMAs
    int hold;                       // test hook: issue no MMA and no commit, so the first wait runs out
};

__device__ __forceinline__ uint4 pack8(const float* v) {
    uint4 r;
    __nv_bfloat162 h[4];
#pragma unroll
    for (int i = 0; i < 4; i++) h[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    memcpy(&r, h, 16);
    return r;
}

// Warp-specialised convolution, one work unit = one 128-row tile of one patch (every plane's rows
// 128 t .. 128 t + 127 of the 19 x 19 padded plane).  An input plane q feeds output planes q + 1, q and
// q - 1 through the z taps dz = -1, 0, +1, so each (dy, dx) tap is ONE MMA with N = 48 = 3 x 16: its A
// operand (the plane's rows shifted by dx + 19 dy) is read once for all three z taps, and its D columns
// are the accumulators of output planes q + 1, q, q - 1, which TMEM holds side by side (plane z at column
// 16 (18 - z); planes 0 and 18 only collect halo terms and are never read).  The first MMA that reaches an
// accumulator in a unit overwrites it: at input plane 1 the first tap's N = 48 MMA (planes 2, 1, 0), at
// input plane q >= 2 the first tap split into an N = 16 MMA that overwrites plane q + 1 and an N = 32 MMA
// that accumulates into planes q and q - 1; every other MMA accumulates.
//   warp 0 (one thread): streams input planes 1..17 of the unit (the 168 rows the tile reaches, both
//     8-channel halves) into a ring of NSLOT slots with cp.async.bulk ("full" mbarrier per slot), refilling
//     a slot once its "empty" barrier says the 9 MMAs that read it have completed;
//   warp 1 (one thread): per input plane, the 9 MMAs into accumulators q + 1, q, q - 1 (every fourth
//     plane, after the epilogue has released the next four planes of the previous unit), then commits to
//     the slot's "empty" barrier
//     and, for the output plane now complete (q - 1; plane 17 too after plane 17), to its "acc full";
//   warps 2..: EPI_SETS sets of 4 warps, set s taking the output planes z with z mod EPI_SETS = s: drain
//     the plane's 16 columns with tcgen05.ld (warp w reads TMEM lanes 32 (w mod 4)..), arrive on its
//     "acc empty", apply bias / relu / mask and write the rows.
// Every wait is bounded by a.wait_ns.  A role whose wait runs out stops; the others then run out too.
// Before the TMEM is freed, the MMA thread waits (bounded) for every MMA it issued and the producer for
// every copy it issued; if either is still outstanding the kernel reports err 2.
__global__ void __launch_bounds__(CONV_THREADS) conv_kernel(ConvArgs a) {
    extern __shared__ __align__(128) uint8_t sm[];
    uint8_t* ring0 = sm;
    uint8_t* ring1 = sm + (size_t)RROWS * 16;
    uint8_t* wsm = ring1 + (size_t)RROWS * 16;
    uint64_t* bars = reinterpret_cast<uint64_t*>(wsm + (size_t)WCAN * 2);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + NBAR);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    // barriers: FULL + slot, EMPTY + slot, AFULL + z - 1, AEMPTY + z - 1 (output planes z = 1..17), DRAIN
    constexpr int FULL = 0, EMPTY = NSLOT, AFULL = 2 * NSLOT, AEMPTY = 2 * NSLOT + SP, DRAIN = 2 * NSLOT + 2 * SP;
    const uint32_t bar0 = tc::smem_u32(bars);
    auto bar = [&](int i) { return bar0 + 8u * (uint32_t)i; };
    const int units = a.batch * NTILE;

    if (warp == 1) tc::tmem_alloc(tslot, 512);
    if (t == 0) {
        for (int i = 0; i < NSLOT; i++) {
            tc::mbar_init(bar(FULL + i), 1);
            tc::mbar_init(bar(EMPTY + i), 1);
        }
        for (int i = 0; i < SP; i++) {
            tc::mbar_init(bar(AFULL + i), 1);
            tc::mbar_init(bar(AEMPTY + i), 4);
        }
        tc::mbar_init(bar(DRAIN), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const uint4* wsrc = reinterpret_cast<const uint4*>(a.w);
    for (int i = t; i < WCAN * 2 / 16; i += CONV_THREADS) reinterpret_cast<uint4*>(wsm)[i] = wsrc[i];
    const uint4 z4 = make_uint4(0, 0, 0, 0);
    for (int i = t; i < 2 * RROWS; i += CONV_THREADS) reinterpret_cast<uint4*>(ring0)[i] = z4;   // both halves
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    int err = 0;

    if (warp == 0) {
        if (lane == 0) {                                  // producer
            uint32_t q = 0;
            bool alive = true;
            for (int u = blockIdx.x; u < units && alive; u += gridDim.x) {
                const int p = u / NTILE, tile = u % NTILE;
                const int r_lo = tile * 128 - HALO_ROWS;                      // plane row of slot row 0
                const int r0 = r_lo > 0 ? r_lo : 0, r1 = r_lo + TROWS < PLANE ? r_lo + TROWS : PLANE;
                const uint32_t bytes = (uint32_t)(r1 - r0) * 16;
                const uint8_t* h0 = reinterpret_cast<const uint8_t*>(a.in + (int64_t)p * PATCH);
                const uint8_t* h1 = h0 + (size_t)ROWS * 16;
                for (int zz = 1; zz <= SP; zz++, q++) {
                    const uint32_t slot = q % NSLOT, use = q / NSLOT;
                    if (use > 0 && !tc::mbar_wait(bar(EMPTY + (int)slot), (use - 1) & 1u, a.wait_ns)) { alive = false; break; }
                    const size_t off = (size_t)(GUARD + zz * PLANE + r0) * 16;
                    const uint32_t dst = (uint32_t)(slot * TROWS + (r0 - r_lo)) * 16;
                    tc::mbar_arrive_expect_tx(bar(FULL + (int)slot), 2 * bytes);
                    tc::bulk_g2s(tc::smem_u32(ring0) + dst, h0 + off, bytes, bar(FULL + (int)slot));
                    tc::bulk_g2s(tc::smem_u32(ring1) + dst, h1 + off, bytes, bar(FULL + (int)slot));
                }
            }
            for (uint32_t sl = 0; sl < NSLOT && sl < q; sl++) {     // the last copy into every used slot has landed
                const uint32_t last = (q - 1 - sl) / NSLOT;
                if (!tc::mbar_wait(bar(FULL + (int)sl), last & 1u, a.wait_ns)) err = 2;
            }
            if (!alive && err == 0) err = 1;
        }
    } else if (warp == 1) {
        if (lane == 0) {                                  // MMA issuer
            constexpr uint32_t IDESC = tc::idesc_bf16_f32(128, N48);
            constexpr uint32_t IDESC16 = tc::idesc_bf16_f32(128, C), IDESC32 = tc::idesc_bf16_f32(128, 2 * C);
            // K-major no-swizzle operands; a descriptor's start-address field counts 16-byte rows, so row and
            // tap offsets are added to the base descriptors directly.  B per (dy, dx) tap: [2 K chunks]
            // [6 groups of 8 N rows][8 x 8], 1536 B.
            const uint64_t adesc0 = tc::smem_desc(tc::smem_u32(ring0), RROWS * 16, 128);
            const uint64_t bdesc0 = tc::smem_desc(tc::smem_u32(wsm), (N48 / 8) * 128, 128);
            uint32_t q = 0, unit = 0;
            bool alive = true, issued = false;
            for (int u = blockIdx.x; u < units && alive; u += gridDim.x, unit++) {
                for (int zz = 1; zz <= SP; zz++, q++) {
                    const uint32_t slot = q % NSLOT;
                    alive = tc::mbar_wait(bar(FULL + (int)slot), (q / NSLOT) & 1u, a.wait_ns);
                    // accumulators first written at input planes zz .. zz + 3: planes zz + 1 .. zz + 4 (and plane
                    // 1 at zz = 1).  Each epilogue set drains the planes of one parity in order, so the release
                    // of the highest plane of each parity covers the lower ones: two waits per four planes.
                    static_assert(EPI_SETS == 2, "one epilogue set per plane parity");
                    if (alive && unit > 0 && (zz & 3) == 1 && zz + 1 <= SP) {
                        const int hi = zz + 4 < SP ? zz + 4 : SP;
                        alive = tc::mbar_wait(bar(AEMPTY + hi - 1), (unit - 1) & 1u, a.wait_ns);
                        if (alive) alive = tc::mbar_wait(bar(AEMPTY + hi - 2), (unit - 1) & 1u, a.wait_ns);
                    }
                    if (!alive) break;
                    tc::fence_after_sync();
                    if (!a.hold) {
                        const uint32_t dst = tmem + (uint32_t)(16 * (SP - zz));     // planes zz + 1, zz, zz - 1
                        const uint32_t base = slot * TROWS + HALO_ROWS;
#pragma unroll
                        for (int txy = 0; txy < TAPS_XY; txy++) {
                            const int dy = txy / 3 - 1, dx = txy % 3 - 1;
                            const uint64_t ad = adesc0 + (base + (uint32_t)(dx + PP * dy));
                            const uint64_t bd = bdesc0 + (uint64_t)(txy * (N48 * C * 2 / 16));
                            if (txy > 0) {
                                tc::mma_bf16(dst, ad, bd, IDESC, 1u);
                            } else if (zz == 1) {
                                tc::mma_bf16(dst, ad, bd, IDESC, 0u);                          // planes 2, 1, 0 fresh
                            } else {
                                tc::mma_bf16(dst, ad, bd, IDESC16, 0u);                        // plane zz + 1 fresh
                                tc::mma_bf16(dst + 16, ad, bd + (2 * 128 / 16), IDESC32, 1u);  // planes zz, zz - 1
                            }
                        }
                        issued = true;
                        tc::mma_commit(bar(EMPTY + (int)slot));                       // input plane zz is done
                        if (zz >= 2) tc::mma_commit(bar(AFULL + (zz - 2)));          // output plane zz - 1
                        if (zz == SP) tc::mma_commit(bar(AFULL + (SP - 1)));         // output plane 17
                    }
                }
            }
            if (issued) {                                 // every MMA issued has completed
                tc::mma_commit(bar(DRAIN));
                if (!tc::mbar_wait(bar(DRAIN), 0, a.wait_ns)) err = 2;
            }
            if (!alive && err == 0) err = 1;
        }
    } else {                                              // epilogue warp sets
        const int quarter = warp & 3, set = (warp - 2) / 4;
        const uint32_t lanes = (uint32_t)(32 * quarter) << 16;
        uint32_t unit = 0;
        bool alive = true;
        for (int u = blockIdx.x; u < units && alive; u += gridDim.x, unit++) {
            const int p = u / NTILE, tile = u % NTILE;
            const int r = tile * 128 + 32 * quarter + lane;
            const int x = r % PP, y = r / PP;
            const bool interior = r < PLANE && x >= 1 && x <= SP && y >= 1 && y <= SP;
            for (int z = 1 + set; z <= SP; z += EPI_SETS) {
                alive = __all_sync(0xffffffffu, tc::mbar_wait(bar(AFULL + z - 1), unit & 1u, a.wait_ns) ? 1 : 0) != 0;
                if (!alive) break;
                tc::fence_after_sync();
                const uint32_t col = tmem + lanes + (uint32_t)(16 * (ACC_PLANES - 1 - z));
                float v[16];
                tc::tmem_ld16_wait(col, v);
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(bar(AEMPTY + z - 1));
                if (r >= PLANE) continue;
                const int64_t row = GUARD + (int64_t)z * PLANE + r;
                if (a.mode == FWD_HEAD) {
                    if (interior) a.zhead[(int64_t)p * KV + ((z - 1) * SP + (y - 1)) * SP + (x - 1)] = v[0] + a.bias[0];
                    continue;
                }
                float o[16];
                if (a.mode == FWD_RELU) {
#pragma unroll
                    for (int c = 0; c < 16; c++) o[c] = interior ? fmaxf(v[c] + a.bias[c], 0.f) : 0.f;
                } else {
                    const uint4* m = reinterpret_cast<const uint4*>(a.mask_act + (int64_t)p * PATCH);
                    uint4 mv[2] = {m[row], m[ROWS + row]};
                    const __nv_bfloat16* mb16 = reinterpret_cast<const __nv_bfloat16*>(mv);
#pragma unroll
                    for (int c = 0; c < 16; c++) o[c] = (interior && __bfloat162float(mb16[c]) > 0.f) ? v[c] : 0.f;
                }
                uint4* dst = reinterpret_cast<uint4*>(a.out + (int64_t)p * PATCH);
                dst[row] = pack8(o);
                dst[ROWS + row] = pack8(o + 8);
            }
        }
        if (!alive && lane == 0) err = 1;
    }
    if (err) atomicMax(a.err, err);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 1) tc::tmem_dealloc(tmem, 512);
}

// Row of padded voxel (i, j, k) of the 17^3 patch (0-based interior coordinates).
__device__ __forceinline__ int prow(int i, int j, int k) { return GUARD + (i + 1) + PP * ((j + 1) + PP * (k + 1)); }

struct PatchPos {
    int sx, sy, sz;
};
__device__ __forceinline__ PatchPos pos_of(int64_t s, const Grid& g) {
    PatchPos q;
    q.sx = (int)(s % g.nx);
    const int64_t r = s / g.nx;
    q.sy = (int)(r % g.ny);
    q.sz = (int)(r / g.ny);
    return q;
}
__device__ __forceinline__ bool in_domain(const PatchPos& q, int i, int j, int k, const Grid& g, int64_t* gi) {
    const int x = q.sx - SH + i, y = q.sy - SH + j, z = q.sz - SH + k;
    if (x < 0 || x >= g.nx || y < 0 || y >= g.ny || z < 0 || z >= g.nz) return false;
    *gi = (int64_t)x + (int64_t)g.nx * y + (int64_t)g.nx * g.ny * z;
    return true;
}

// Feature channel 0 per grid cell, once per context: log10 D / 8 + 1 clamped to [-0.5, 1.5] (FP64, -0.5
// where D <= 0), rounded to BF16 (bits).
__global__ void feat0_kernel(const double* __restrict__ D, int64_t n, uint16_t* __restrict__ f0) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double d = D[i];
        double f = d > 0.0 ? log10(d) / 8.0 + 1.0 : -0.5;
        f = f < -0.5 ? -0.5 : (f > 1.5 ? 1.5 : f);
        f0[i] = __bfloat16_as_ushort(__float2bfloat16_rn((float)f));
    }
}

// Feature patches: channels 0-7 of every voxel in one 16-byte store (channels 7-15 are zero; the halo and
// guard rows stay zero from a prior memset).
__global__ void features_kernel(const uint16_t* __restrict__ f0, Grid g, const int64_t* __restrict__ src, int n,
                                __nv_bfloat16* __restrict__ act) {
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)n * KV;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(idx / KV), v = (int)(idx % KV);
        const int i = v % SP, j = (v / SP) % SP, k = v / (SP * SP);
        const PatchPos q = pos_of(src[b], g);
        int64_t gi;
        float h[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        uint4 row;
        if (in_domain(q, i, j, k, g, &gi)) {
            h[0] = __bfloat162float(__ushort_as_bfloat16(f0[gi]));    // exact: already BF16
            h[1] = 1.f;
        }
        if (i == SH && j == SH && k == SH) h[2] = 1.f;
        const int ox = i - SH, oy = j - SH, oz = k - SH;     // offsets from the source: exact in BF16
        h[3] = (float)ox * 0.125f;
        h[4] = (float)oy * 0.125f;
        h[5] = (float)oz * 0.125f;
        h[6] = (float)(ox * ox + oy * oy + oz * oz) * (1.f / 256.f);
        row = pack8(h);
        *reinterpret_cast<uint4*>(act + (int64_t)b * PATCH + (int64_t)prow(i, j, k) * 8) = row;
    }
}

// Head for prediction: y = exp(z) in the domain, FP64 mass, gate; kernels_out [n][KV] (nullable).
__global__ void __launch_bounds__(256) head_predict_kernel(const float* __restrict__ zhead, Grid g,
                                                           const int64_t* __restrict__ src, double* __restrict__ kout,
                                                           double* __restrict__ mass, int* __restrict__ accept) {
    __shared__ double sh[8];
    const int b = blockIdx.x;
    const PatchPos q = pos_of(src[b], g);
    double acc = 0.0;
    for (int v = threadIdx.x; v < KV; v += blockDim.x) {
        const int i = v % SP, j = (v / SP) % SP, k = v / (SP * SP);
        int64_t gi;
        const double y = in_domain(q, i, j, k, g, &gi) ? (double)expf(zhead[(int64_t)b * KV + v]) : 0.0;
        if (kout) kout[(int64_t)b * KV + v] = y;
        acc += y;
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double w = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        for (int off = 16; off > 0; off >>= 1) w += __shfl_xor_sync(0xffffffffu, w, off);
        if (threadIdx.x == 0) {
            mass[b] = w;
            accept[b] = fabs(w - 1.0) <= GATE_TOL ? 1 : 0;
        }
    }
}

// Head for training: the generalised Kullback-Leibler divergence sum_v (y - k z + k ln k - k), y = exp(z),
// over in-domain cells (0 ln 0 = 0) and its gradient y - k with respect to z (channel 0); the gradient
// penalises predicted mass wherever the target kernel has less, which is what the mass gate checks.
__global__ void __launch_bounds__(256) head_train_kernel(const float* __restrict__ zhead, Grid g,
                                                         const int64_t* __restrict__ src, const double* __restrict__ tgt,
                                                         __nv_bfloat16* __restrict__ grad, double* __restrict__ loss) {
    __shared__ double sh[8];
    const int b = blockIdx.x;
    const PatchPos q = pos_of(src[b], g);
    double acc = 0.0;
    for (int v = threadIdx.x; v < KV; v += blockDim.x) {
        const int i = v % SP, j = (v / SP) % SP, k = v / (SP * SP);
        int64_t gi;
        const bool ind = in_domain(q, i, j, k, g, &gi);
        double gz = 0.0;
        if (ind) {
            const double kk = tgt[(int64_t)b * KV + v];
            const double z = (double)zhead[(int64_t)b * KV + v];
            const double y = exp(z);
            acc += y - kk * z + (kk > 0.0 ? kk * log(kk) : 0.0) - kk;
            gz = y - kk;
        }
        grad[(int64_t)b * PATCH + (int64_t)prow(i, j, k) * 8] = __float2bfloat16_rn((float)gz);
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double w = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        for (int off = 16; off > 0; off >>= 1) w += __shfl_xor_sync(0xffffffffu, w, off);
        if (threadIdx.x == 0) loss[b] = w;
    }
}

// Head for the kernel cache: accepted predictions are rounded to the storage type and written into
// Q[o][s + o]; sigma_s = 1 / FP64 sum of the stored values (the march's renormalisation).
__global__ void __launch_bounds__(256) head_store_kernel(const float* __restrict__ zhead, Grid g,
                                                         const int64_t* __restrict__ src, const int* __restrict__ accept,
                                                         void* Q, Store st, double* __restrict__ sigma) {
    __shared__ double sh[8];
    const int b = blockIdx.x;
    if (!accept[b]) return;
    const int64_t s = src[b];
    const PatchPos q = pos_of(s, g);
    double acc = 0.0;
    for (int v = threadIdx.x; v < KV; v += blockDim.x) {
        const int i = v % SP, j = (v / SP) % SP, k = v / (SP * SP);
        int64_t gi;
        if (!in_domain(q, i, j, k, g, &gi)) continue;
        const float y = expf(zhead[(int64_t)b * KV + v]);
        const int64_t idx = (int64_t)v * g.n + gi;       // offset o = (i-8, j-8, k-8), destination gi
        float stored;
        if (st == Store::F32) { reinterpret_cast<float*>(Q)[idx] = y; stored = y; }
        else if (st == Store::F16) { const __half h = __float2half_rn(y); reinterpret_cast<__half*>(Q)[idx] = h; stored = __half2float(h); }
        else { const __nv_bfloat16 h = __float2bfloat16_rn(y); reinterpret_cast<__nv_bfloat16*>(Q)[idx] = h; stored = __bfloat162float(h); }
        acc += (double)stored;
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double w = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        for (int off = 16; off > 0; off >>= 1) w += __shfl_xor_sync(0xffffffffu, w, off);
        if (threadIdx.x == 0) sigma[s] = w > 0.0 ? 1.0 / w : 0.0;
    }
}

// Weight and bias gradients of one layer on the tensor cores.  dW[tap][co][ci] = sum over rows r' of
// act[r' + off(tap)][ci] grad[r'][co] and db[co] = sum over r' of grad[r'][co], r' over the interior rows
// (grad is zero on halo rows), off(tap) = dx + 19 dy + 361 dz.  The reduction runs over rows, so both
// operands are MN-major (channels contiguous within a 16-byte row), and the taps are split between them:
// with r = r' - dx - 19 dy, the term is act[r + 361 dz][ci] grad[r + dx' + 19 dy'][co], dx' = -dx, dy' = -dy.
// Per 32-row unit (rows r of padded planes 1..17, which the +-20-row in-plane shifts cannot push past the
// plane halo):
//   A (M = 128): groups g = 3 h + dz_i (g < 6) hold channels 8h.. of act rows r + 361 (dz_i - 1); group 6
//     holds ones (its D rows are db); groups 7..15 are never read back;
//   B (N = 144): groups 9 h + 3 dy_i + dx_i hold channels 8h.. of grad rows r + (dx_i - 1) + 19 (dy_i - 1);
// so ONE MMA (K = 16 rows) yields every (tap, ci, co) pair (an N = 144 MMA takes 72 clocks at the tensor
// rate, four N = 16 ones at least 4 x 45).  In the no-swizzle MN-major layout a core matrix is 8 rows x 16
// bytes; a group of a unit is 512 contiguous bytes, core matrices of consecutive rows 128 B apart (the K
// stride), groups 512 B apart (the M / N stride).
//   Both operands arrive as one tiled tensor copy each: the activation buffer is described to the TMA unit
//   as an overlapping 3-D view (rows x channels flattened: the unit's 256 elements, dz: 361 rows, half), the
//   gradient buffer as a 4-D one (elements, dx: 16 B, dy: 19 rows, half); each box lands in shared memory in
//   the group order above.
//   warp 0 (one thread): copies WG_SUB units per stage into a ring of WG_NST stages (full / empty mbarriers);
//   warp 1 (one thread): 2 MMAs (M = 128, N = 144, K = 16) per unit into one of two TMEM accumulators,
//     switching accumulator every WG_GST stages (a group) and committing the finished one ("acc full");
//   warps 2..5: add each finished group's accumulator (warp w: TMEM lanes 32 (w mod 4)..) into FP32 register
//     sums, release it ("acc empty"), and at the end write the sums to partial[part][slot][co][ci].
// The tensor core's FP32 accumulation is not round-to-nearest (a chain of ~160 MMAs per CTA showed errors
// of one sign, 10x those of FP32 FMAs), and Adam integrates a one-sided error in a near-cancelling
// gradient; short TMEM chains (16 MMAs) summed round-to-nearest in registers keep it at FP32-FMA level.
// Fixed partition into WG_PARTS ranges and a fixed-order sum over them (wgrad_reduce_kernel): the result
// depends on the batch only.  Waits are bounded like the convolution's (err 1, or 2 if MMAs or copies may
// still be in flight).
constexpr int WG_ROWS = 32;                                        // rows (the K extent) per unit
constexpr int WG_UNITS = (SP * PLANE + WG_ROWS - 1) / WG_ROWS;    // units per patch: 192
constexpr int WG_SLOTS = 32;                                       // partial slots: 27 taps, the bias, 4 unused
constexpr int WG_GROUP = WG_ROWS * 16;                             // bytes per 8-channel group of a unit: 512
constexpr int WG_NA = 6, WG_NB = 18;                               // copied groups of A and of B
constexpr int WG_ONES = WG_NA * WG_GROUP;                          // A group 6
constexpr int WG_B = 8 * WG_GROUP;                                 // B (A's unread groups 8..15 overlay it)
constexpr int WG_UNIT = WG_B + WG_NB * WG_GROUP;                   // shared bytes per unit: 13312
constexpr int WG_N = WG_NB * 8;                                    // MMA N: 144
constexpr int WG_SUB = 4;                                          // units per ring stage
constexpr int WG_NST = 3;                                          // ring stages
constexpr int WG_PARTS = 152;                                      // CTAs, each a contiguous range of units
constexpr int WG_GST = 2;                                          // stages per accumulator group (8 units)
constexpr int WG_THREADS = 192;                                    // producer, MMA, four drain warps
constexpr uint32_t WG_TX = (WG_NA + WG_NB) * WG_GROUP;            // bytes copied per unit
constexpr int WG_NBAR = 2 * WG_NST + 4;                            // ring full / empty, accumulator full / empty
constexpr size_t WG_SMEM = (size_t)WG_NST * WG_SUB * WG_UNIT + WG_NBAR * 8 + 16;
static_assert(WG_ROWS * 8 == 256, "one box row is 256 BF16 elements");
static_assert(16 * WG_GROUP <= WG_UNIT, "A's 16 groups stay inside the unit's shared bytes");
// The first unit's rows start at plane 1; the last unit ends 7 rows into plane 18.  A reaches one plane
// either way, B 20 rows either way: inside the guard rows of the patch's half, and B inside the volume.
static_assert(GUARD + PLANE - PLANE >= 0, "A rows below the first unit leave the patch");
static_assert(GUARD + PLANE + WG_UNITS * WG_ROWS + PLANE <= ROWS, "A rows past the last unit leave the patch");
static_assert(PLANE + WG_UNITS * WG_ROWS + PP + 1 <= VOL, "B rows past the last unit leave the volume");

struct WgradArgs {
    float* partial;                 // [WG_PARTS][WG_SLOTS][C co][C ci]
    int batch;
    int* err;
    uint64_t wait_ns;
    int hold;                       // test hook: issue no MMA and no commit, so the drain warps' wait runs out
};

// tm_act: the layer's input [batch][PATCH] as the view (elements, dz, half), box (256, 3, 2); tm_grad: the
// gradient of its output as (elements, dx, dy, half), box (256, 3, 3, 2).
__global__ void __launch_bounds__(WG_THREADS) wgrad_kernel(const __grid_constant__ CUtensorMap tm_act,
                                                           const __grid_constant__ CUtensorMap tm_grad, WgradArgs a) {
    extern __shared__ __align__(128) uint8_t sm[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + (size_t)WG_NST * WG_SUB * WG_UNIT);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + WG_NBAR);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    constexpr int FULL = 0, EMPTY = WG_NST, AFULL = 2 * WG_NST, AEMPTY = 2 * WG_NST + 2;
    const uint32_t sbase = tc::smem_u32(sm), bar0 = tc::smem_u32(bars);
    auto bar = [&](int i) { return bar0 + 8u * (uint32_t)i; };
    const int64_t units = (int64_t)a.batch * WG_UNITS;
    const int64_t u_lo = units * blockIdx.x / WG_PARTS, u_hi = units * (blockIdx.x + 1) / WG_PARTS;
    const int nstage = (int)((u_hi - u_lo + WG_SUB - 1) / WG_SUB);
    const int ngroup = (nstage + WG_GST - 1) / WG_GST;

    if (warp == 1) tc::tmem_alloc(tslot, 512);           // accumulators at columns 0 and 256
    if (t == 0) {
        for (int i = 0; i < WG_NST; i++) {
            tc::mbar_init(bar(FULL + i), 1);
            tc::mbar_init(bar(EMPTY + i), 1);
        }
        for (int i = 0; i < 2; i++) {
            tc::mbar_init(bar(AFULL + i), 1);
            tc::mbar_init(bar(AEMPTY + i), 4);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // A group 6 of every unit slot: ones (BF16 1.0 = 0x3F80); the copies never write it
    constexpr int ONE_WORDS = WG_GROUP / 4;
    for (int i = t; i < WG_NST * WG_SUB * ONE_WORDS; i += WG_THREADS)
        reinterpret_cast<uint32_t*>(sm + (size_t)(i / ONE_WORDS) * WG_UNIT + WG_ONES)[i % ONE_WORDS] = 0x3F803F80u;
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    int err = 0;

    if (warp == 0) {
        if (lane == 0) {                                  // producer
            bool alive = true;
            int q = 0;
            for (; q < nstage; q++) {
                const uint32_t s = (uint32_t)q % WG_NST, use = (uint32_t)q / WG_NST;
                if (use > 0 && !tc::mbar_wait(bar(EMPTY + (int)s), (use - 1) & 1u, a.wait_ns)) { alive = false; break; }
                const int64_t u0 = u_lo + (int64_t)q * WG_SUB;
                const int cnt = u_hi - u0 < WG_SUB ? (int)(u_hi - u0) : WG_SUB;
                tc::mbar_arrive_expect_tx(bar(FULL + (int)s), (uint32_t)cnt * WG_TX);
                for (int j = 0; j < cnt; j++) {
                    const int64_t u = u0 + j;
                    // buffer row of the unit's first row r (patch-major, half 0)
                    const int64_t row = (u / WG_UNITS) * 2 * ROWS + GUARD + PLANE + (u % WG_UNITS) * WG_ROWS;
                    const uint32_t dst = sbase + (s * WG_SUB + (uint32_t)j) * WG_UNIT;
                    tc::tma_load_3d(dst, &tm_act, (int)((row - PLANE) * 8), 0, 0, bar(FULL + (int)s));
                    tc::tma_load_4d(dst + WG_B, &tm_grad, (int)((row - PP - 1) * 8), 0, 0, 0, bar(FULL + (int)s));
                }
            }
            for (int sl = 0; sl < WG_NST && sl < q; sl++) {   // the last copies into every used stage have landed
                const uint32_t last = (uint32_t)(q - 1 - sl) / WG_NST;
                if (!tc::mbar_wait(bar(FULL + sl), last & 1u, a.wait_ns)) err = 2;
            }
            if (!alive && err == 0) err = 1;
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {                                  // MMA issuer
            // A and B MN-major (instruction descriptor bits 15 and 16); descriptors: K stride 128 B (8 rows),
            // M / N stride 512 B (one group).  The start-address field counts 16-byte units.
            constexpr uint32_t IDESC = tc::idesc_bf16_f32(128, WG_N) | (1u << 15) | (1u << 16);
            const uint64_t d0 = tc::smem_desc(sbase, 128, WG_GROUP);
            bool alive = true;
            int g = 0, gs = 0;                            // accumulator group, stages issued into it
            for (int q = 0; q < nstage && !a.hold; q++) {
                const uint32_t s = (uint32_t)q % WG_NST, acc = (uint32_t)(g & 1) * 256u;
                // a group's accumulator is reused two groups later, once the drain warps have released it
                if (gs == 0 && g >= 2 &&
                    !tc::mbar_wait(bar(AEMPTY + (g & 1)), (uint32_t)((g >> 1) - 1) & 1u, a.wait_ns)) { alive = false; break; }
                if (!tc::mbar_wait(bar(FULL + (int)s), ((uint32_t)q / WG_NST) & 1u, a.wait_ns)) { alive = false; break; }
                tc::fence_after_sync();
                const int64_t u0 = u_lo + (int64_t)q * WG_SUB;
                const int cnt = u_hi - u0 < WG_SUB ? (int)(u_hi - u0) : WG_SUB;
                for (int j = 0; j < cnt; j++) {
                    const uint32_t ub = (s * WG_SUB + (uint32_t)j) * WG_UNIT;
#pragma unroll
                    for (int k = 0; k < WG_ROWS / 16; k++)
                        tc::mma_bf16(tmem + acc, d0 + (uint64_t)((ub + k * 256) >> 4), d0 + (uint64_t)((ub + WG_B + k * 256) >> 4),
                                     IDESC, (gs > 0 || j > 0 || k > 0) ? 1u : 0u);
                }
                tc::mma_commit(bar(EMPTY + (int)s));
                if (++gs == WG_GST || q == nstage - 1) {  // the group's accumulator is complete
                    tc::mma_commit(bar(AFULL + (g & 1)));
                    g++;
                    gs = 0;
                }
            }
            if (!alive) err = 1;
        }
        __syncwarp();
    } else {                                              // drain warps 2..5
        // D row 8 gA + c (A group gA, channel c), column 8 gB + c' (B group gB, channel c')
        const int quarter = warp & 3, mrow = 32 * quarter + lane, ga = mrow / 8, c8 = mrow % 8;
        const uint32_t lanes = (uint32_t)(32 * quarter) << 16;
        float sum[WG_N];
#pragma unroll
        for (int i = 0; i < WG_N; i++) sum[i] = 0.f;
        bool alive = true;
        for (int g = 0; g < ngroup; g++) {
            alive = __all_sync(0xffffffffu, tc::mbar_wait(bar(AFULL + (g & 1)), (uint32_t)(g >> 1) & 1u, a.wait_ns) ? 1 : 0) != 0;
            if (!alive) break;
            tc::fence_after_sync();
#pragma unroll
            for (int jc = 0; jc < WG_N / 16; jc++) {
                float v[16];
                tc::tmem_ld16_wait(tmem + lanes + (uint32_t)(g & 1) * 256u + (uint32_t)(16 * jc), v);
#pragma unroll
                for (int i = 0; i < 16; i++) sum[16 * jc + i] += v[i];
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(bar(AEMPTY + (g & 1)));
        }
        if (!alive) {
            if (lane == 0) err = a.hold ? 1 : 2;          // MMAs may still be running (none under the hook)
        } else {
            const bool ones = ga == WG_NA && c8 == 0;     // the bias row
            float* part = a.partial + (int64_t)blockIdx.x * WG_SLOTS * C * C;
#pragma unroll
            for (int n = 0; n < WG_N; n++) {
                const int gb = n / 8, co = 8 * (gb / 9) + n % 8, dyi = (gb / 3) % 3, dxi = gb % 3;
                if (ga < WG_NA) {
                    const int tap = (2 - dxi) + 3 * (2 - dyi) + 9 * (ga % 3), ci = 8 * (ga / 3) + c8;
                    part[((int64_t)tap * C + co) * C + ci] = sum[n];
                } else if (ones && dyi == 1 && dxi == 1) {
                    part[((int64_t)TAPS * C + co) * C] = sum[n];
                }
            }
        }
    }
    if (err) atomicMax(a.err, err);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 1) tc::tmem_dealloc(tmem, 512);
}

// dW[tap][co][ci] = sum over the WG_PARTS partials in order; db[co] = the same sum of the ones slot (ci 0).
__global__ void wgrad_reduce_kernel(const float* __restrict__ partial, float* __restrict__ dW, float* __restrict__ db) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= TAPS * C * C + C) return;
    const int64_t idx = e < TAPS * C * C ? e : (int64_t)TAPS * C * C + (int64_t)(e - TAPS * C * C) * C;
    float s = 0.f;
    for (int p = 0; p < WG_PARTS; p++) s += partial[(int64_t)p * WG_SLOTS * C * C + idx];
    if (e < TAPS * C * C) dW[e] = s;
    else db[e - TAPS * C * C] = s;
}

// Canonical UMMA layouts of the BF16 weights for the N = 48 convolution: per (dy, dx) tap txy = (dx+1) +
// 3 (dy+1), a K-major [2 K chunks][6 groups of 8 N rows][8 n][8 k] block (1536 B) whose N row
// n48 = 16 (dz + 1) + n holds z tap dz (so D columns 16 (dz + 1).. belong to output plane q - dz).
// Forward: n = co, k = ci.  Input gradient: tap -> 26 - tap (flip), n = ci, k = co (transpose).
__global__ void canon_kernel(const float* __restrict__ params, __nv_bfloat16* __restrict__ wf,
                             __nv_bfloat16* __restrict__ wd) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NW) return;
    const int l = e / (TAPS * C * C), rem = e % (TAPS * C * C);
    const int tap = rem / (C * C), co = (rem / C) % C, ci = rem % C;
    const __nv_bfloat16 w = __float2bfloat16_rn(params[e]);
    auto cidx = [](int tp, int n, int k) {
        const int txy = tp % 9, dzi = tp / 9, n48 = C * dzi + n;
        return txy * (N48 * C) + (k >> 3) * (N48 * 8) + (n48 >> 3) * 64 + (n48 & 7) * 8 + (k & 7);
    };
    wf[(int64_t)l * WCAN + cidx(tap, co, ci)] = w;
    wd[(int64_t)l * WCAN + cidx(TAPS - 1 - tap, ci, co)] = w;
}

// Adam on the FP32 master parameters (mean gradient over the batch); layer 4 keeps only channel 0.
__global__ void adam_kernel(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ grad, float scale, float lr, float b1t, float b2t) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NPARAM) return;
    bool frozen;
    if (e < NW) frozen = e / (TAPS * C * C) == NL - 1 && ((e % (C * C)) / C) != 0;
    else frozen = (e - NW) / C == NL - 1 && ((e - NW) % C) != 0;
    if (frozen) return;
    const float gr = grad[e] * scale;
    const float mm = 0.9f * m[e] + 0.1f * gr;
    const float vv = 0.999f * v[e] + 0.001f * gr * gr;
    m[e] = mm;
    v[e] = vv;
    p[e] -= lr * (mm / (1.f - b1t)) / (sqrtf(vv / (1.f - b2t)) + 1e-8f);
}

// Unpacks a batch of activation or gradient volumes ([n][2 halves][ROWS][8] BF16, zero halo) into
// [n][C][KV] BF16 bit patterns, voxel v = i + 17 (j + 17 k) of the patch.
__global__ void unpack_kernel(const __nv_bfloat16* __restrict__ src, int n, uint16_t* __restrict__ dst) {
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)n * C * KV;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(idx / (C * KV)), c = (int)((idx / KV) % C), v = (int)(idx % KV);
        const int i = v % SP, j = (v / SP) % SP, k = v / (SP * SP);
        const int64_t half = c < 8 ? 0 : ROWS;
        dst[idx] = __bfloat16_as_ushort(src[(int64_t)b * PATCH + (half + prow(i, j, k)) * 8 + (c & 7)]);
    }
}

}  // namespace net
}  // namespace fdirw

using namespace fdirw::net;
namespace tcx = fdirw::tc;

struct fdirw_net {
    int device = 0;
    float* params = nullptr;   // device FP32 master [NPARAM]
    float* m = nullptr;
    float* v = nullptr;
    int64_t step = 0;
    __nv_bfloat16* wf = nullptr;   // [NL][WCAN]
    __nv_bfloat16* wd = nullptr;
    int cap = 0;
    __nv_bfloat16* act[NL] = {};   // inputs of layers 1..4 (act[0] = features)
    __nv_bfloat16* gbuf[2] = {};
    float* zhead = nullptr;
    int64_t* dsrc = nullptr;
    double* dtgt = nullptr;
    double* dkout = nullptr;
    double* dmass = nullptr;
    int* dacc = nullptr;
    double* dloss = nullptr;
    float* partial = nullptr;
    float* grads = nullptr;
    int* derr = nullptr;
    CUtensorMap tm_act[NL];        // weight-gradient views of act[l] and gbuf[i] (encoded with the buffers)
    CUtensorMap tm_grad[2];
    cudaEvent_t ev[2] = {};        // around the four convolutions of the last forward pass
    bool timed = false;
    uint64_t wait_ns = WAIT_NS;    // budget of each MMA wait (fdirw_net_test_wait)
    int hold = 0;                  // test hook: convolutions and weight gradients withhold their MMAs
    bool failed = false;           // a wait gave up while MMAs may still have been running
    std::string err;
};

namespace {

thread_local std::string g_net_err;

int nfail(fdirw_net* net, int code, const std::string& msg) {
    if (net) net->err = msg; else g_net_err = msg;
    return fdirw::set_thread_error(code, msg);
}

#define NET_CUDA(net, call)                                                                     \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) return nfail((net), FDIRW_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, fetched once through the runtime (no link against the driver library).
EncodeTiledFn encode_tiled() {
    static const EncodeTiledFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// Tensor maps of the weight gradient for buffers of `cap` patches.  Activation view, innermost first: the
// buffer's BF16 elements (box 256 = one unit's 32 rows x 8 channels), dz (one plane, 361 x 16 B), half
// (ROWS x 16 B); box (256, 3, 2).  Gradient view: elements, dx (16 B), dy (one padded row of the plane,
// 19 x 16 B), half; box (256, 3, 3, 2).  The views overlap themselves; each box is a unit's shifted groups.
int encode_maps(fdirw_net* net, int cap) {
    const EncodeTiledFn enc = encode_tiled();
    if (!enc) return nfail(net, FDIRW_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const cuuint64_t elems = (cuuint64_t)cap * PATCH;
    const cuuint64_t dim_a[3] = {elems, 3, 2};
    const cuuint64_t str_a[2] = {PLANE * 16, (cuuint64_t)ROWS * 16};
    const cuuint32_t box_a[3] = {256, 3, 2};
    const cuuint64_t dim_g[4] = {elems, 3, 3, 2};
    const cuuint64_t str_g[3] = {16, PP * 16, (cuuint64_t)ROWS * 16};
    const cuuint32_t box_g[4] = {256, 3, 3, 2};
    const cuuint32_t one[4] = {1, 1, 1, 1};
    for (int i = 0; i < NL + 2; i++) {
        const bool act = i < NL;
        const CUresult r = enc(act ? &net->tm_act[i] : &net->tm_grad[i - NL], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, act ? 3 : 4,
                               act ? (void*)net->act[i] : (void*)net->gbuf[i - NL], act ? dim_a : dim_g, act ? str_a : str_g,
                               act ? box_a : box_g, one, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS)
            return nfail(net, FDIRW_ERR_CUDA, std::string("encoding a weight-gradient tensor map failed (CUresult ") +
                                                  std::to_string((int)r) + ")");
    }
    return FDIRW_OK;
}

int ensure_capacity(fdirw_net* net, int n) {
    if (n <= net->cap) return FDIRW_OK;
    const int cap = n;
    for (auto& p : net->act) { cudaFree(p); p = nullptr; }
    for (auto& p : net->gbuf) { cudaFree(p); p = nullptr; }
    cudaFree(net->zhead); cudaFree(net->dsrc); cudaFree(net->dtgt); cudaFree(net->dkout);
    cudaFree(net->dmass); cudaFree(net->dacc); cudaFree(net->dloss);
    net->cap = 0;
    const size_t ab = (size_t)cap * PATCH * 2;
    for (auto& p : net->act) NET_CUDA(net, cudaMalloc(&p, ab));
    for (auto& p : net->gbuf) NET_CUDA(net, cudaMalloc(&p, ab));
    for (auto& p : net->act) NET_CUDA(net, cudaMemset(p, 0, ab));       // halos stay zero from here on
    for (auto& p : net->gbuf) NET_CUDA(net, cudaMemset(p, 0, ab));
    NET_CUDA(net, cudaMalloc(&net->zhead, (size_t)cap * KV * 4));
    NET_CUDA(net, cudaMalloc(&net->dsrc, (size_t)cap * 8));
    NET_CUDA(net, cudaMalloc(&net->dtgt, (size_t)cap * KV * 8));
    NET_CUDA(net, cudaMalloc(&net->dkout, (size_t)cap * KV * 8));
    NET_CUDA(net, cudaMalloc(&net->dmass, (size_t)cap * 8));
    NET_CUDA(net, cudaMalloc(&net->dacc, (size_t)cap * 4));
    NET_CUDA(net, cudaMalloc(&net->dloss, (size_t)cap * 8));
    if (const int rc = encode_maps(net, cap); rc != FDIRW_OK) return rc;
    net->cap = cap;
    return FDIRW_OK;
}

int launch_conv(fdirw_net* net, cudaStream_t st, int num_sms, const __nv_bfloat16* in, __nv_bfloat16* out,
                float* zhead, const __nv_bfloat16* mask, const __nv_bfloat16* w, const float* bias, int n, int mode) {
    ConvArgs a{in, out, zhead, mask, w, bias, n, mode, net->derr, net->wait_ns, net->hold};
    NET_CUDA(net, cudaFuncSetAttribute(conv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CONV_SMEM));
    int per_sm = 0;
    NET_CUDA(net, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, conv_kernel, CONV_THREADS, CONV_SMEM));
    if (per_sm != 1) return nfail(net, FDIRW_ERR_CUDA, "the convolution needs exactly one CTA per SM (TMEM)");
    const int units = n * NTILE;
    const int grid = units < num_sms ? units : num_sms;
    conv_kernel<<<grid, CONV_THREADS, CONV_SMEM, st>>>(a);
    NET_CUDA(net, cudaGetLastError());
    return FDIRW_OK;
}

// Weight and bias gradients of one layer: the tensor-core partial sums, then their fixed-order reduction.
// Layer l's input is act[l]; the gradient of its output is gbuf[cur].
int launch_wgrad(fdirw_net* net, cudaStream_t st, int l, int cur, int n, float* dW, float* db) {
    WgradArgs a{net->partial, n, net->derr, net->wait_ns, net->hold};
    NET_CUDA(net, cudaFuncSetAttribute(wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)WG_SMEM));
    wgrad_kernel<<<WG_PARTS, WG_THREADS, WG_SMEM, st>>>(net->tm_act[l], net->tm_grad[cur], a);
    NET_CUDA(net, cudaGetLastError());
    wgrad_reduce_kernel<<<(TAPS * C * C + C + 255) / 256, 256, 0, st>>>(net->partial, dW, db);
    NET_CUDA(net, cudaGetLastError());
    return FDIRW_OK;
}

// Features + the 4 convolutions for sources dsrc[0..n) (already on the device).  The first layer's
// input keeps its halo zero; channels 3..15 and the out-of-domain rows are cleared every call.
int forward(fdirw_ctx* c, fdirw_net* net, int n) {
    cudaStream_t st = c->stream;
    NET_CUDA(net, cudaMemsetAsync(net->act[0], 0, (size_t)n * PATCH * 2, st));
    const int64_t work = (int64_t)n * KV;
    const int fb = (int)((work + 255) / 256 < 152 * 16 ? (work + 255) / 256 : 152 * 16);
    if (!c->feat0) {                                      // channel 0 per cell, made once per context
        if (fdirw::host::dalloc(c, reinterpret_cast<void**>(&c->feat0), (uint64_t)c->g.n * 2, "surrogate features") != FDIRW_OK)
            return nfail(net, FDIRW_ERR_NOMEM, "allocating the surrogate's per-cell features");
        feat0_kernel<<<152 * 8, 256, 0, st>>>(c->Dd, c->g.n, c->feat0);
        NET_CUDA(net, cudaGetLastError());
    }
    features_kernel<<<fb, 256, 0, st>>>(c->feat0, c->g, net->dsrc, n, net->act[0]);
    NET_CUDA(net, cudaGetLastError());
    NET_CUDA(net, cudaEventRecord(net->ev[0], st));
    for (int l = 0; l < NL; l++) {
        const bool head = l == NL - 1;
        const int rc = launch_conv(net, st, c->num_sms, net->act[l], head ? nullptr : net->act[l + 1],
                                   head ? net->zhead : nullptr, nullptr, net->wf + (size_t)l * WCAN,
                                   net->params + NW + l * C, n, head ? FWD_HEAD : FWD_RELU);
        if (rc != FDIRW_OK) return rc;
    }
    NET_CUDA(net, cudaEventRecord(net->ev[1], st));
    net->timed = true;
    return FDIRW_OK;
}

int check_err(fdirw_net* net, cudaStream_t st) {
    int h = 0;
    NET_CUDA(net, cudaMemcpyAsync(&h, net->derr, 4, cudaMemcpyDeviceToHost, st));
    NET_CUDA(net, cudaStreamSynchronize(st));
    if (h) {
        cudaMemsetAsync(net->derr, 0, 4, st);
        if (h >= 2) {
            net->failed = true;
            return nfail(net, FDIRW_ERR_TIMEOUT, "a tensor-core kernel (convolution or weight gradient) gave up on MMAs or copies that had not "
                                                 "completed after two waits; the network refuses further calls");
        }
        return nfail(net, FDIRW_ERR_TIMEOUT, "a tensor-core kernel (convolution or weight gradient) timed out waiting for its MMAs");
    }
    return FDIRW_OK;
}

// Calls on a network whose convolution gave up on running MMAs are refused: the tensor memory it
// released may still be written by them.
int usable(fdirw_net* net) {
    if (net && net->failed)
        return nfail(net, FDIRW_ERR_STATE, "this network's convolution gave up on MMAs that may still be running; "
                                           "destroy it (and, to be safe, the CUDA context)");
    return FDIRW_OK;
}

int upload_sources(fdirw_ctx* c, fdirw_net* net, const int64_t* sources, int64_t n) {
    if (n < 0 || n > MAX_BATCH) return nfail(net, FDIRW_ERR_ARG, "batch size must be in [0, 1024]");
    for (int64_t q = 0; q < n; q++)
        if (sources[q] < 0 || sources[q] >= c->g.n) return nfail(net, FDIRW_ERR_ARG, "source index out of range");
    int rc = ensure_capacity(net, (int)(n > 0 ? n : 1));
    if (rc != FDIRW_OK) return rc;
    NET_CUDA(net, cudaMemcpyAsync(net->dsrc, sources, (size_t)n * 8, cudaMemcpyHostToDevice, c->stream));
    return FDIRW_OK;
}

// Receives the gradient with respect to layer l's output (its pre-activation; masked by the relu) before
// layer l's weight gradient is formed.
using GradHook = std::function<int(int, const __nv_bfloat16*)>;

// Backward through the 4 layers into net->grads (sum over the batch); the head gradient is in gbuf[0].
int backward(fdirw_ctx* c, fdirw_net* net, int n, const GradHook* hook = nullptr) {
    cudaStream_t st = c->stream;
    int cur = 0;
    for (int l = NL - 1; l >= 0; l--) {
        if (hook) {
            const int rc = (*hook)(l, net->gbuf[cur]);
            if (rc != FDIRW_OK) return rc;
        }
        const int rw = launch_wgrad(net, st, l, cur, n, net->grads + (size_t)l * TAPS * C * C, net->grads + NW + l * C);
        if (rw != FDIRW_OK) return rw;
        if (l > 0) {
            const int rc = launch_conv(net, st, c->num_sms, net->gbuf[cur], net->gbuf[cur ^ 1], nullptr, net->act[l],
                                       net->wd + (size_t)l * WCAN, nullptr, n, DGRAD);
            if (rc != FDIRW_OK) return rc;
            cur ^= 1;
        }
    }
    return FDIRW_OK;
}

int gradients(fdirw_ctx* c, fdirw_net* net, const int64_t* sources, int64_t n, const double* targets,
              double* loss_out, const GradHook* hook = nullptr) {
    int rc = upload_sources(c, net, sources, n);
    if (rc != FDIRW_OK) return rc;
    NET_CUDA(net, cudaMemcpyAsync(net->dtgt, targets, (size_t)n * KV * 8, cudaMemcpyDefault, c->stream));
    if ((rc = forward(c, net, (int)n)) != FDIRW_OK) return rc;
    NET_CUDA(net, cudaMemsetAsync(net->gbuf[0], 0, (size_t)n * PATCH * 2, c->stream));
    head_train_kernel<<<(int)n, 256, 0, c->stream>>>(net->zhead, c->g, net->dsrc, net->dtgt, net->gbuf[0], net->dloss);
    NET_CUDA(net, cudaGetLastError());
    if ((rc = backward(c, net, (int)n, hook)) != FDIRW_OK) return rc;
    std::vector<double> lv((size_t)n);
    NET_CUDA(net, cudaMemcpyAsync(lv.data(), net->dloss, (size_t)n * 8, cudaMemcpyDeviceToHost, c->stream));
    if ((rc = check_err(net, c->stream)) != FDIRW_OK) return rc;
    double s = 0.0;
    for (double x : lv) s += x;
    if (loss_out) *loss_out = n > 0 ? s / (double)n : 0.0;
    return FDIRW_OK;
}

}  // namespace

extern "C" {

FDIRW_API int fdirw_net_create(const float* params, int32_t device, fdirw_net** out) {
    if (!out || !params) return nfail(nullptr, FDIRW_ERR_ARG, "NULL params or out");
    *out = nullptr;
    int prev = 0;
    cudaGetDevice(&prev);
    if (device >= 0 && cudaSetDevice(device) != cudaSuccess) return nfail(nullptr, FDIRW_ERR_CUDA, "cannot select device");
    fdirw_net* net = new fdirw_net();
    cudaGetDevice(&net->device);
    auto bail = [&](const std::string& m) {
        std::string msg = m;
        fdirw_net_destroy(net);
        if (device >= 0) cudaSetDevice(prev);
        return nfail(nullptr, FDIRW_ERR_CUDA, msg);
    };
    if (cudaMalloc(&net->params, NPARAM * 4) != cudaSuccess || cudaMalloc(&net->m, NPARAM * 4) != cudaSuccess ||
        cudaMalloc(&net->v, NPARAM * 4) != cudaSuccess || cudaMalloc(&net->grads, NPARAM * 4) != cudaSuccess ||
        cudaMalloc(&net->wf, (size_t)NL * WCAN * 2) != cudaSuccess || cudaMalloc(&net->wd, (size_t)NL * WCAN * 2) != cudaSuccess ||
        cudaMalloc(&net->partial, (size_t)WG_PARTS * WG_SLOTS * C * C * 4) != cudaSuccess ||
        cudaMalloc(&net->derr, 4) != cudaSuccess || cudaEventCreate(&net->ev[0]) != cudaSuccess ||
        cudaEventCreate(&net->ev[1]) != cudaSuccess)
        return bail("allocating the network");
    if (cudaMemcpy(net->params, params, NPARAM * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(net->m, 0, NPARAM * 4) != cudaSuccess || cudaMemset(net->v, 0, NPARAM * 4) != cudaSuccess ||
        cudaMemset(net->derr, 0, 4) != cudaSuccess)
        return bail("initialising the network");
    canon_kernel<<<(NW + 255) / 256, 256>>>(net->params, net->wf, net->wd);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return bail("weight layout kernel");
    if (device >= 0) cudaSetDevice(prev);
    *out = net;
    return FDIRW_OK;
}

FDIRW_API int fdirw_net_params(fdirw_net* net, float* params_out) {
    if (!net || !params_out) return nfail(net, FDIRW_ERR_ARG, "NULL net or params_out");
    NET_CUDA(net, cudaMemcpy(params_out, net->params, NPARAM * 4, cudaMemcpyDeviceToHost));
    return FDIRW_OK;
}

FDIRW_API void fdirw_net_destroy(fdirw_net* net) {
    if (!net) return;
    cudaDeviceSynchronize();
    for (auto& p : net->act) cudaFree(p);
    for (auto& p : net->gbuf) cudaFree(p);
    cudaFree(net->params); cudaFree(net->m); cudaFree(net->v); cudaFree(net->wf); cudaFree(net->wd);
    cudaFree(net->zhead); cudaFree(net->dsrc); cudaFree(net->dtgt); cudaFree(net->dkout); cudaFree(net->dmass);
    cudaFree(net->dacc); cudaFree(net->dloss); cudaFree(net->partial); cudaFree(net->grads); cudaFree(net->derr);
    for (auto e : net->ev) if (e) cudaEventDestroy(e);
    delete net;
}

FDIRW_API int fdirw_net_predict(fdirw_ctx* ctx, fdirw_net* net, const int64_t* sources, int64_t n,
                                double* kernels_out, double* mass_out, int32_t* accept_out) {
    if (!ctx || !net || (n > 0 && !sources)) return nfail(net, FDIRW_ERR_ARG, "NULL ctx, net or sources");
    if (ctx->batch || ctx->coarse) return nfail(net, FDIRW_ERR_ARG, "the surrogate serves fdirw_create contexts only");
    if (const int u = usable(net); u != FDIRW_OK) return u;
    if (n == 0) return FDIRW_OK;
    int rc = upload_sources(ctx, net, sources, n);
    if (rc != FDIRW_OK) return rc;
    if ((rc = forward(ctx, net, (int)n)) != FDIRW_OK) return rc;
    head_predict_kernel<<<(int)n, 256, 0, ctx->stream>>>(net->zhead, ctx->g, net->dsrc, net->dkout, net->dmass, net->dacc);
    NET_CUDA(net, cudaGetLastError());
    if (kernels_out) NET_CUDA(net, cudaMemcpyAsync(kernels_out, net->dkout, (size_t)n * KV * 8, cudaMemcpyDefault, ctx->stream));
    if (mass_out) NET_CUDA(net, cudaMemcpyAsync(mass_out, net->dmass, (size_t)n * 8, cudaMemcpyDeviceToHost, ctx->stream));
    if (accept_out) NET_CUDA(net, cudaMemcpyAsync(accept_out, net->dacc, (size_t)n * 4, cudaMemcpyDeviceToHost, ctx->stream));
    return check_err(net, ctx->stream);
}

FDIRW_API int fdirw_net_gradients(fdirw_ctx* ctx, fdirw_net* net, const int64_t* sources, int64_t n,
                                  const double* targets, float* grads_out, double* loss_out) {
    if (!ctx || !net || n <= 0 || !sources || !targets) return nfail(net, FDIRW_ERR_ARG, "bad arguments");
    if (ctx->batch || ctx->coarse) return nfail(net, FDIRW_ERR_ARG, "the surrogate serves fdirw_create contexts only");
    if (const int u = usable(net); u != FDIRW_OK) return u;
    int rc = gradients(ctx, net, sources, n, targets, loss_out);
    if (rc != FDIRW_OK) return rc;
    if (grads_out) NET_CUDA(net, cudaMemcpy(grads_out, net->grads, NPARAM * 4, cudaMemcpyDeviceToHost));
    return FDIRW_OK;
}

FDIRW_API int fdirw_net_train_step(fdirw_ctx* ctx, fdirw_net* net, const int64_t* sources, int64_t n,
                                   const double* targets, float lr, double* loss_out) {
    if (!ctx || !net || n <= 0 || !sources || !targets || !(lr > 0.f)) return nfail(net, FDIRW_ERR_ARG, "bad arguments");
    if (ctx->batch || ctx->coarse) return nfail(net, FDIRW_ERR_ARG, "the surrogate serves fdirw_create contexts only");
    if (const int u = usable(net); u != FDIRW_OK) return u;
    int rc = gradients(ctx, net, sources, n, targets, loss_out);
    if (rc != FDIRW_OK) return rc;
    net->step++;
    const float b1t = (float)std::pow(0.9, (double)net->step), b2t = (float)std::pow(0.999, (double)net->step);
    adam_kernel<<<(NPARAM + 255) / 256, 256, 0, ctx->stream>>>(net->params, net->m, net->v, net->grads,
                                                               1.f / (float)n, lr, b1t, b2t);
    NET_CUDA(net, cudaGetLastError());
    canon_kernel<<<(NW + 255) / 256, 256, 0, ctx->stream>>>(net->params, net->wf, net->wd);
    NET_CUDA(net, cudaGetLastError());
    return FDIRW_OK;
}

FDIRW_API int fdirw_net_timing(fdirw_net* net, float* conv_ms) {
    if (!net || !conv_ms) return nfail(net, FDIRW_ERR_ARG, "NULL net or conv_ms");
    *conv_ms = 0.f;
    if (!net->timed) return FDIRW_OK;
    NET_CUDA(net, cudaEventSynchronize(net->ev[1]));
    NET_CUDA(net, cudaEventElapsedTime(conv_ms, net->ev[0], net->ev[1]));
    return FDIRW_OK;
}

FDIRW_API int fdirw_net_test_wait(fdirw_net* net, uint64_t wait_ns, int32_t withhold_mma) {
    if (!net) return nfail(net, FDIRW_ERR_ARG, "NULL net");
    net->wait_ns = wait_ns ? wait_ns : WAIT_NS;
    net->hold = withhold_mma ? 1 : 0;
    return FDIRW_OK;
}

FDIRW_API int fdirw_net_trace(fdirw_ctx* ctx, fdirw_net* net, const int64_t* sources, int64_t n,
                              const double* targets, uint16_t* acts_out, float* z_out, uint16_t* grads_out,
                              float* grads_param_out, double* loss_out) {
    if (!ctx || !net || n <= 0 || !sources) return nfail(net, FDIRW_ERR_ARG, "bad arguments");
    if (grads_out && !targets) return nfail(net, FDIRW_ERR_ARG, "gradient buffers need targets");
    if (ctx->batch || ctx->coarse) return nfail(net, FDIRW_ERR_ARG, "the surrogate serves fdirw_create contexts only");
    if (const int u = usable(net); u != FDIRW_OK) return u;
    cudaStream_t st = ctx->stream;
    const size_t vol = (size_t)n * C * KV;      // BF16 values of one traced volume set
    uint16_t* stage = nullptr;
    if (acts_out || grads_out) NET_CUDA(net, cudaMalloc(&stage, vol * 2));
    const int ub = (int)std::min<int64_t>(((int64_t)vol + 255) / 256, 152 * 16);
    auto dump = [&](const __nv_bfloat16* src, uint16_t* dst) -> int {
        unpack_kernel<<<ub, 256, 0, st>>>(src, (int)n, stage);
        NET_CUDA(net, cudaGetLastError());
        NET_CUDA(net, cudaMemcpyAsync(dst, stage, vol * 2, cudaMemcpyDefault, st));
        return FDIRW_OK;
    };
    int rc = FDIRW_OK;
    if (targets) {
        GradHook hook = [&](int l, const __nv_bfloat16* g) -> int {
            if (l == NL - 1) {          // the forward pass is complete here
                if (acts_out)
                    for (int a = 0; a < NL; a++)
                        if (const int r = dump(net->act[a], acts_out + (size_t)a * vol); r != FDIRW_OK) return r;
                if (z_out) NET_CUDA(net, cudaMemcpyAsync(z_out, net->zhead, (size_t)n * KV * 4, cudaMemcpyDefault, st));
            }
            return grads_out ? dump(g, grads_out + (size_t)l * vol) : FDIRW_OK;
        };
        rc = gradients(ctx, net, sources, n, targets, loss_out, &hook);
        if (rc == FDIRW_OK && grads_param_out)
            rc = cudaMemcpy(grads_param_out, net->grads, NPARAM * 4, cudaMemcpyDefault) == cudaSuccess
                     ? FDIRW_OK : nfail(net, FDIRW_ERR_CUDA, "copying the parameter gradients");
    } else {
        rc = upload_sources(ctx, net, sources, n);
        if (rc == FDIRW_OK) rc = forward(ctx, net, (int)n);
        if (rc == FDIRW_OK && acts_out)
            for (int a = 0; a < NL && rc == FDIRW_OK; a++) rc = dump(net->act[a], acts_out + (size_t)a * vol);
        if (rc == FDIRW_OK && z_out && cudaMemcpyAsync(z_out, net->zhead, (size_t)n * KV * 4, cudaMemcpyDefault, st) != cudaSuccess)
            rc = nfail(net, FDIRW_ERR_CUDA, "copying the head");
        if (rc == FDIRW_OK) rc = check_err(net, st);
    }
    cudaStreamSynchronize(st);
    cudaFree(stage);
    return rc;
}

FDIRW_API int fdirw_kernels_surrogate(fdirw_ctx* c, fdirw_net* net, int64_t* accepted_out) {
    if (!c || !net) return nfail(net, FDIRW_ERR_ARG, "NULL ctx or net");
    if (c->batch || c->coarse || c->flow) return nfail(net, FDIRW_ERR_ARG, "the surrogate serves diffusion-only fdirw_create contexts");
    if (const int u = usable(net); u != FDIRW_OK) return u;
    if (c->R != SH) return nfail(net, FDIRW_ERR_ARG, "the surrogate predicts 17^3 kernels: window_R must be 8");
    if (c->store == Store::F64) return nfail(net, FDIRW_ERR_ARG, "the surrogate serves the FP32-march precisions only");
    {
        const int rc = fdirw::ensure_cache(c);
        if (rc != FDIRW_OK) return nfail(net, rc, fdirw_last_error(c));
        if (c->slab_T) return nfail(net, FDIRW_ERR_STATE, "the surrogate needs a resident kernel cache (this one is streamed)");
    }
    const int64_t N = c->g.n;
    std::vector<int64_t> src(MAX_BATCH), rejected;
    std::vector<int32_t> acc(MAX_BATCH);
    rejected.reserve((size_t)(N / 4));
    int64_t accepted = 0;
    int rc = ensure_capacity(net, MAX_BATCH);
    if (rc != FDIRW_OK) return rc;
    for (int64_t b0 = 0; b0 < N; b0 += MAX_BATCH) {
        const int n = (int)(N - b0 < MAX_BATCH ? N - b0 : MAX_BATCH);
        for (int q = 0; q < n; q++) src[q] = b0 + q;
        NET_CUDA(net, cudaMemcpyAsync(net->dsrc, src.data(), (size_t)n * 8, cudaMemcpyHostToDevice, c->stream));
        if ((rc = forward(c, net, n)) != FDIRW_OK) return rc;
        head_predict_kernel<<<n, 256, 0, c->stream>>>(net->zhead, c->g, net->dsrc, nullptr, net->dmass, net->dacc);
        NET_CUDA(net, cudaGetLastError());
        head_store_kernel<<<n, 256, 0, c->stream>>>(net->zhead, c->g, net->dsrc, net->dacc, c->Q, c->store, c->sigma);
        NET_CUDA(net, cudaGetLastError());
        NET_CUDA(net, cudaMemcpyAsync(acc.data(), net->dacc, (size_t)n * 4, cudaMemcpyDeviceToHost, c->stream));
        NET_CUDA(net, cudaStreamSynchronize(c->stream));
        for (int q = 0; q < n; q++) {
            if (acc[q]) accepted++;
            else rejected.push_back(src[q]);
        }
    }
    if ((rc = check_err(net, c->stream)) != FDIRW_OK) return rc;
    if (!rejected.empty()) {
        int64_t* dlist = nullptr;
        NET_CUDA(net, cudaMalloc(&dlist, rejected.size() * 8));
        cudaError_t e = cudaMemcpyAsync(dlist, rejected.data(), rejected.size() * 8, cudaMemcpyHostToDevice, c->stream);
        fdirw::MarchArgs a{};
        a.g = c->g;
        a.R = c->R;
        a.Rq = c->R;
        a.q_stride = c->g.n;
        a.n_sub = c->n_sub;
        a.ax = reinterpret_cast<const float*>(c->coef[0]);
        a.ay = reinterpret_cast<const float*>(c->coef[1]);
        a.az = reinterpret_cast<const float*>(c->coef[2]);
        a.Q = c->Q;
        a.store = c->store;
        a.sigma = c->sigma;
        a.src_begin = 0;
        a.src_end = (int64_t)rejected.size();
        a.list = dlist;
        if (e == cudaSuccess) e = fdirw::launch_march(a, c->num_sms, c->parts_req, c->stream, &c->parts_used);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        cudaFree(dlist);
        if (e != cudaSuccess) return nfail(net, FDIRW_ERR_CUDA, std::string("fallback march: ") + cudaGetErrorString(e));
    }
    c->kernels_ready = true;
    if (accepted_out) *accepted_out = accepted;
    return FDIRW_OK;
}

}  // extern "C"
