// Coarse-mesh FDiRW (Sec. 3.1, Eqs. 10-15, without the boundary term p_BC c_far).
//
//   nodes      the liquid cells of each B x B x B block form one representative node (B odd; blocks
//              clipped by the domain keep their cells); N_I = liquid cells of block I
//   phase      faces with a non-liquid cell on either side carry no flux; non-liquid cells keep c
//   P          column J: the remapped unit of block J (1 on its liquid cells, Eq. 12) marched n_sub
//              explicit substeps on the block's window widened by R cells, then mapped (Eq. 11):
//              P[I][J] = N_J S_I / (m N_I), S_I the marched mass on block I, m the total.  The march is
//              mapping 5 in coarse mode (march.cu); P is stored FP64, destination-indexed over the
//              (2 Rc + 1)^3 block offsets, Rc = ceil(R / B)
//   step       mapping (Eq. 13): C_I = mean of c over the liquid cells of block I, FP64 in cell order;
//              FDiRW calculation (Eq. 14): C'_I = sum_d P[I][I - d] C_{I - d}, FP64, d ascending;
//              re-mapping (Eq. 15): c'_i = C'_I on every liquid cell of block I.
#include "fdirw.h"
#include "fdirw_internal.h"
#include "ctx.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace fdirw::host;

namespace fdirw {

struct Coarse {
    int B = 1, Rc = 0, Rw = 0;                   // block side, band radius, march window radius
    int ncx = 0, ncy = 0, ncz = 0;
    int64_t nc = 0, nodes = 0;                   // blocks, blocks with liquid
    uint8_t* liquid = nullptr;                   // N
    int32_t* count = nullptr;                    // nc
    int64_t* list = nullptr;                     // blocks with liquid, ascending
    double* Qc = nullptr;                        // Wc^3 planes of nc values
    double* C = nullptr;                         // nc
    double* Cn = nullptr;                        // nc
    bool built = false;
    // Far-field boundary (open outer surface): lam * open-face conductance per cell, P_BC per block,
    // device scalars [c_far, mass before, mass after], FP32 ping-pong fields of the P_BC march.
    bool open = false;
    double V_far = 0.0;
    float* abnd = nullptr;
    double* pbc = nullptr;
    double* far = nullptr;
    float* ubuf = nullptr;
    // Coupled macro step: FP64 solid-phase face conductances, a scratch field, phase-mass partials.
    double* gs = nullptr;                        // 3 N: +x/+y/+z solid-solid faces
    double* tmp = nullptr;                       // 2 N
    double* qpart = nullptr;                     // kMassBlocks
    double* qout = nullptr;                      // [Q_L, Q_S] per step, n_steps_cap * 2
    int64_t qcap = 0;
};

namespace {

int grid_blocks(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b > 152 * 16) b = 152 * 16;
    return (int)(b < 1 ? 1 : b);
}

// Zero the coefficient of every face with a non-liquid cell on either side.
__global__ void mask_faces_kernel(Grid g, const uint8_t* __restrict__ liquid, float* __restrict__ ax,
                                  float* __restrict__ ay, float* __restrict__ az) {
    const int64_t nxy = (int64_t)g.nx * g.ny;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % g.nx);
        const int y = (int)((i / g.nx) % g.ny);
        const int z = (int)(i / nxy);
        const bool l = liquid[i] != 0;
        if (!l || x + 1 >= g.nx || !liquid[i + 1]) ax[i] = 0.f;
        if (!l || y + 1 >= g.ny || !liquid[i + g.nx]) ay[i] = 0.f;
        if (!l || z + 1 >= g.nz || !liquid[i + nxy]) az[i] = 0.f;
    }
}

// Liquid cells per block (one thread per block, cells in z, y, x order).
__global__ void count_kernel(Grid g, const uint8_t* __restrict__ liquid, int B, int ncx, int ncy, int64_t nc,
                             int32_t* __restrict__ count) {
    for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < nc; I += (int64_t)gridDim.x * blockDim.x) {
        const int bx = (int)(I % ncx), by = (int)((I / ncx) % ncy), bz = (int)(I / ((int64_t)ncx * ncy));
        int n = 0;
        for (int z = bz * B; z < min(bz * B + B, g.nz); z++)
            for (int y = by * B; y < min(by * B + B, g.ny); y++)
                for (int x = bx * B; x < min(bx * B + B, g.nx); x++)
                    n += liquid[x + (int64_t)g.nx * (y + (int64_t)g.ny * z)] ? 1 : 0;
        count[I] = n;
    }
}

// Eq. 13: C_I = (sum of c over the liquid cells of block I, z, y, x order) / N_I.
__global__ void map_kernel(Grid g, const uint8_t* __restrict__ liquid, int B, int ncx, int ncy, int64_t nc,
                           const int32_t* __restrict__ count, const double* __restrict__ c, double* __restrict__ C) {
    for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < nc; I += (int64_t)gridDim.x * blockDim.x) {
        const int bx = (int)(I % ncx), by = (int)((I / ncx) % ncy), bz = (int)(I / ((int64_t)ncx * ncy));
        double s = 0.0;
        for (int z = bz * B; z < min(bz * B + B, g.nz); z++)
            for (int y = by * B; y < min(by * B + B, g.ny); y++)
                for (int x = bx * B; x < min(bx * B + B, g.nx); x++) {
                    const int64_t i = x + (int64_t)g.nx * (y + (int64_t)g.ny * z);
                    if (liquid[i]) s += c[i];
                }
        C[I] = count[I] > 0 ? s / (double)count[I] : 0.0;
    }
}

// Open faces: gb_i = D_i times the faces of liquid cell i on the grid's outer surface; abnd = fp32(lam gb)
// (one rounding, as the face coefficients); the largest per-cell sum of masked face conductances plus gb
// (bits of a non-negative double, for atomicMax) for the stability check.
__global__ void open_faces_kernel(Grid g, const double* __restrict__ D, const uint8_t* __restrict__ liquid,
                                  double lam, float* __restrict__ abnd, unsigned long long* __restrict__ max_bits) {
    const int64_t nxy = (int64_t)g.nx * g.ny;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % g.nx), y = (int)((i / g.nx) % g.ny), z = (int)(i / nxy);
        double gb = 0.0, sum = 0.0;
        if (liquid[i]) {
            const int faces = (x == 0) + (x == g.nx - 1) + (y == 0) + (y == g.ny - 1) + (z == 0) + (z == g.nz - 1);
            gb = D[i] * (double)faces;
            auto face = [&](int64_t j) {
                const double a = D[i], b = D[j];
                return (liquid[j] && a + b > 0.0) ? 2.0 * a * b / (a + b) : 0.0;
            };
            if (x > 0) sum += face(i - 1);
            if (x + 1 < g.nx) sum += face(i + 1);
            if (y > 0) sum += face(i - g.nx);
            if (y + 1 < g.ny) sum += face(i + g.nx);
            if (z > 0) sum += face(i - nxy);
            if (z + 1 < g.nz) sum += face(i + nxy);
            sum += gb;
        }
        abnd[i] = (float)(lam * gb);
        atomicMax(max_bits, (unsigned long long)__double_as_longlong(sum));
    }
}

// One explicit substep of the liquid phase over the whole grid with every far-field ghost at 1 (the
// P_BC march): u' = u + (am u + sum c u_nb + abnd), am = -(sum of the cell's coefficients + abnd), in the
// FP32 increment form and association of the windowed kernels.
// With convection (bx != NULL) the inflow from the upper neighbour uses B and the diagonal sums the cell's
// outflows (A of its +faces, B of its -faces), as the block-source march.
__global__ void pbc_substep_kernel(Grid g, const float* __restrict__ ax, const float* __restrict__ ay,
                                   const float* __restrict__ az, const float* __restrict__ bx,
                                   const float* __restrict__ by, const float* __restrict__ bz,
                                   const float* __restrict__ abnd, const float* __restrict__ u,
                                   float* __restrict__ un) {
    const int64_t nxy = (int64_t)g.nx * g.ny;
    const float* ux = bx ? bx : ax;                   // coefficient of the upper neighbour in this cell
    const float* uy = bx ? by : ay;
    const float* uz = bx ? bz : az;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % g.nx), y = (int)((i / g.nx) % g.ny), z = (int)(i / nxy);
        const float cxm = x > 0 ? ax[i - 1] : 0.f, cxp = x + 1 < g.nx ? ux[i] : 0.f;
        const float cym = y > 0 ? ay[i - g.nx] : 0.f, cyp = y + 1 < g.ny ? uy[i] : 0.f;
        const float czm = z > 0 ? az[i - nxy] : 0.f, czp = z + 1 < g.nz ? uz[i] : 0.f;
        // outflows: the cell's own +faces (A) and the lower neighbours' B; equal to the inflows without flow
        const float oxm = x > 0 ? ux[i - 1] : 0.f, oxp = x + 1 < g.nx ? ax[i] : 0.f;
        const float oym = y > 0 ? uy[i - g.nx] : 0.f, oyp = y + 1 < g.ny ? ay[i] : 0.f;
        const float ozm = z > 0 ? uz[i - nxy] : 0.f, ozp = z + 1 < g.nz ? az[i] : 0.f;
        const float vb = abnd[i];
        const float cur = u[i];
        const float am = -((((oxm + oxp) + (oym + oyp)) + (ozm + ozp)) + vb);
        float v = am * cur;
        v = fmaf(cxm, x > 0 ? u[i - 1] : 0.f, v);
        v = fmaf(cxp, x + 1 < g.nx ? u[i + 1] : 0.f, v);
        v = fmaf(cym, y > 0 ? u[i - g.nx] : 0.f, v);
        v = fmaf(cyp, y + 1 < g.ny ? u[i + g.nx] : 0.f, v);
        v = fmaf(czm, z > 0 ? u[i - nxy] : 0.f, v);
        v = fmaf(czp, z + 1 < g.nz ? u[i + nxy] : 0.f, v);
        v = __fadd_rn(v, vb);                           // inflow from the ghosts at c_far = 1
        un[i] = __fadd_rn(cur, v);
    }
}

__global__ void widen_kernel(const float* __restrict__ u, int64_t n, double* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (double)u[i];
}

// Interface exchange of Eqs. 4-6 on every liquid/solid face, pre-step values, rate over dt; each cell adds
// its faces' transfers in the order -z, -y, -x, +x, +y, +z (the order in which a raster sweep over the
// lower cell of each face reaches them), f_L and f_S clamped at 0.  FP64 without contraction.
__device__ __forceinline__ double exchange(const double* c, const uint8_t* liquid, int64_t a, int64_t b, double k,
                                           double cS, double cL, double dt) {
    // transfer from the liquid cell to the solid one across face (a, b); 0 unless the phases differ
    if (liquid[a] == liquid[b]) return 0.0;
    const int64_t l = liquid[a] ? a : b, s = liquid[a] ? b : a;
    const double fL = c[l] > cL ? __ddiv_rn(__dadd_rn(c[l], -cL), cL) : 0.0;
    const double fS = c[s] < cS ? __ddiv_rn(__dadd_rn(cS, -c[s]), cS) : 0.0;
    return __dmul_rn(__dmul_rn(__dmul_rn(k, fL), fS), dt);
}

__global__ void absorb_kernel(Grid g, const uint8_t* __restrict__ liquid, double k, double cS, double cL, double dt,
                              const double* __restrict__ c, double* __restrict__ out) {
    const int64_t nxy = (int64_t)g.nx * g.ny;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % g.nx), y = (int)((i / g.nx) % g.ny), z = (int)(i / nxy);
        const double sgn = liquid[i] ? -1.0 : 1.0;       // the liquid side loses, the solid side gains
        double v = c[i];
        if (z > 0) v = __dadd_rn(v, sgn * exchange(c, liquid, i - nxy, i, k, cS, cL, dt));
        if (y > 0) v = __dadd_rn(v, sgn * exchange(c, liquid, i - g.nx, i, k, cS, cL, dt));
        if (x > 0) v = __dadd_rn(v, sgn * exchange(c, liquid, i - 1, i, k, cS, cL, dt));
        if (x + 1 < g.nx) v = __dadd_rn(v, sgn * exchange(c, liquid, i, i + 1, k, cS, cL, dt));
        if (y + 1 < g.ny) v = __dadd_rn(v, sgn * exchange(c, liquid, i, i + g.nx, k, cS, cL, dt));
        if (z + 1 < g.nz) v = __dadd_rn(v, sgn * exchange(c, liquid, i, i + nxy, k, cS, cL, dt));
        out[i] = v;
    }
}

// FP64 harmonic conductances of the faces between two solid cells (+x, +y, +z of each cell).
__global__ void solid_faces_kernel(Grid g, const double* __restrict__ D, const uint8_t* __restrict__ liquid,
                                   double* __restrict__ gx, double* __restrict__ gy, double* __restrict__ gz) {
    const int64_t nxy = (int64_t)g.nx * g.ny;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % g.nx), y = (int)((i / g.nx) % g.ny), z = (int)(i / nxy);
        auto h = [&](int64_t j) {
            const double a = D[i], b = D[j];
            return (!liquid[i] && !liquid[j] && __dadd_rn(a, b) > 0.0)
                       ? __ddiv_rn(__dmul_rn(__dmul_rn(2.0, a), b), __dadd_rn(a, b)) : 0.0;
        };
        gx[i] = x + 1 < g.nx ? h(i + 1) : 0.0;
        gy[i] = y + 1 < g.ny ? h(i + g.nx) : 0.0;
        gz[i] = z + 1 < g.nz ? h(i + nxy) : 0.0;
    }
}

// One flux-form substep of the solid phase, FP64, faces in the order -x, +x, -y, +y, -z, +z.
__global__ void solid_substep_kernel(Grid g, const double* __restrict__ gx, const double* __restrict__ gy,
                                     const double* __restrict__ gz, double lam, const double* __restrict__ u,
                                     double* __restrict__ un) {
    const int64_t nxy = (int64_t)g.nx * g.ny;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % g.nx), y = (int)((i / g.nx) % g.ny), z = (int)(i / nxy);
        const double ui = u[i];
        double acc = 0.0;
        if (x > 0) acc = __dadd_rn(acc, __dmul_rn(gx[i - 1], __dadd_rn(u[i - 1], -ui)));
        if (x + 1 < g.nx) acc = __dadd_rn(acc, __dmul_rn(gx[i], __dadd_rn(u[i + 1], -ui)));
        if (y > 0) acc = __dadd_rn(acc, __dmul_rn(gy[i - g.nx], __dadd_rn(u[i - g.nx], -ui)));
        if (y + 1 < g.ny) acc = __dadd_rn(acc, __dmul_rn(gy[i], __dadd_rn(u[i + g.nx], -ui)));
        if (z > 0) acc = __dadd_rn(acc, __dmul_rn(gz[i - nxy], __dadd_rn(u[i - nxy], -ui)));
        if (z + 1 < g.nz) acc = __dadd_rn(acc, __dmul_rn(gz[i], __dadd_rn(u[i + nxy], -ui)));
        un[i] = __dadd_rn(ui, __dmul_rn(lam, acc));
    }
}

// Fixed-order FP64 total of the cells of one phase: block b sums chunk b, then one block sums the partials.
__global__ void __launch_bounds__(256) phase_partial_kernel(const double* __restrict__ c, const uint8_t* __restrict__ liquid,
                                                            int want_liquid, int64_t n, double* __restrict__ partials) {
    __shared__ double sh[8];
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t lo = blockIdx.x * chunk;
    const int64_t hi = lo + chunk < n ? lo + chunk : n;
    double acc = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x)
        if ((liquid[i] != 0) == (want_liquid != 0)) acc += c[i];
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (threadIdx.x == 0) partials[blockIdx.x] = v;
    }
}

__global__ void __launch_bounds__(kMassBlocks) phase_final_kernel(const double* __restrict__ partials, double* __restrict__ out) {
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

// Eq. 7 for the step just taken: c_far = (m_in + V_far c_far - m_out) / V_far.
__global__ void far_update_kernel(double* far, double V_far) {
    far[0] = ((far[1] + V_far * far[0]) - far[2]) / V_far;
}

// Eq. 14: C'_I = sum over block offsets d (ascending) of P[I][I - d] C_{I - d}, FP64, plus P_BC[I] c_far
// when the outer surface is open.
__global__ void coarse_gather_kernel(int ncx, int ncy, int ncz, int Rc, const double* __restrict__ Qc,
                                     const double* __restrict__ C, const double* __restrict__ pbc,
                                     const double* __restrict__ far, double* __restrict__ Cn) {
    const int64_t nc = (int64_t)ncx * ncy * ncz;
    const int Wc = 2 * Rc + 1;
    for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < nc; I += (int64_t)gridDim.x * blockDim.x) {
        const int bx = (int)(I % ncx), by = (int)((I / ncx) % ncy), bz = (int)(I / ((int64_t)ncx * ncy));
        double acc = 0.0;
        int d = 0;
        for (int dz = -Rc; dz <= Rc; dz++)
            for (int dy = -Rc; dy <= Rc; dy++)
                for (int dx = -Rc; dx <= Rc; dx++, d++) {
                    const int jx = bx - dx, jy = by - dy, jz = bz - dz;
                    if (jx < 0 || jx >= ncx || jy < 0 || jy >= ncy || jz < 0 || jz >= ncz) continue;
                    const int64_t J = jx + (int64_t)ncx * (jy + (int64_t)ncy * jz);
                    acc = fma(Qc[(int64_t)d * nc + I], C[J], acc);
                }
        if (pbc) acc = __dadd_rn(acc, __dmul_rn(pbc[I], far[0]));
        Cn[I] = acc;
        (void)Wc;
    }
}

// Eq. 15: c'_i = C'_I on liquid cells, c'_i = c_i elsewhere (in place allowed: each cell reads itself).
__global__ void remap_kernel(Grid g, const uint8_t* __restrict__ liquid, int B, int ncx, int ncy,
                             const double* __restrict__ Cn, const double* c_in, double* c_out) {
    const int64_t nxy = (int64_t)g.nx * g.ny;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % g.nx), y = (int)((i / g.nx) % g.ny), z = (int)(i / nxy);
        c_out[i] = liquid[i] ? Cn[(x / B) + (int64_t)ncx * ((y / B) + (int64_t)ncy * (z / B))] : c_in[i];
    }
}

// Columns of P for listed blocks on the source-major band layout [n][Wc^3] (offset d = I - J).
__global__ void read_coarse_kernel(const double* __restrict__ Qc, int ncx, int ncy, int ncz, int Rc,
                                   const int64_t* __restrict__ blocks, int64_t n, double* __restrict__ out) {
    const int Wc = 2 * Rc + 1;
    const int64_t W3 = (int64_t)Wc * Wc * Wc, nc = (int64_t)ncx * ncy * ncz;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * W3; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = t / W3;
        const int d = (int)(t % W3);
        const int64_t J = blocks[q];
        const int bx = (int)(J % ncx), by = (int)((J / ncx) % ncy), bz = (int)(J / ((int64_t)ncx * ncy));
        const int cx = bx + d % Wc - Rc, cy = by + (d / Wc) % Wc - Rc, cz = bz + d / (Wc * Wc) - Rc;
        double v = 0.0;
        if (cx >= 0 && cx < ncx && cy >= 0 && cy < ncy && cz >= 0 && cz < ncz)
            v = Qc[(int64_t)d * nc + cx + (int64_t)ncx * (cy + (int64_t)ncy * cz)];
        out[t] = v;
    }
}

}  // namespace

int coarse_kernels(fdirw_ctx* c) {
    Coarse& k = *c->coarse;
    if (k.built) return FDIRW_OK;
    const uint64_t W3 = (uint64_t)(2 * k.Rc + 1) * (2 * k.Rc + 1) * (2 * k.Rc + 1);
    FDIRW_CUDA(c, cudaMemsetAsync(k.Qc, 0, W3 * (uint64_t)k.nc * 8, c->stream));
    MarchArgs a{};
    a.g = c->g;
    a.R = k.Rw;
    a.Rq = k.Rw;
    a.n_sub = c->n_sub;
    a.ax = reinterpret_cast<const float*>(c->coef[0]);
    a.ay = reinterpret_cast<const float*>(c->coef[1]);
    a.az = reinterpret_cast<const float*>(c->coef[2]);
    a.src_begin = 0;
    a.src_end = k.nodes;
    a.list = k.list;
    a.coarse_B = k.B;
    a.coarse_Rc = k.Rc;
    a.ncx = k.ncx;
    a.ncy = k.ncy;
    a.ncz = k.ncz;
    a.coarse_n = k.nc;
    a.liquid = k.liquid;
    a.ccount = k.count;
    a.Qc = k.Qc;
    a.abnd = k.open ? k.abnd : nullptr;
    if (c->flow) {                                     // convection: direction-dependent faces
        a.bx = reinterpret_cast<const float*>(c->coefb[0]);
        a.by = reinterpret_cast<const float*>(c->coefb[1]);
        a.bz = reinterpret_cast<const float*>(c->coefb[2]);
    }
    FDIRW_CUDA(c, cudaEventRecord(c->ev[0], c->stream));
    if (k.nodes > 0 && c->n_sub >= 0) FDIRW_CUDA(c, launch_march_coarse(a, k.Rw, c->num_sms, c->stream));
    FDIRW_CUDA(c, cudaEventRecord(c->ev[1], c->stream));
    if (k.open) {
        // P_BC: the liquid from 0 with every ghost at 1, n_sub substeps over the whole grid, then Eq. 11.
        float* u0 = k.ubuf;
        float* u1 = k.ubuf + c->g.n;
        FDIRW_CUDA(c, cudaMemsetAsync(u0, 0, (size_t)c->g.n * 4, c->stream));
        for (int t = 0; t < c->n_sub; t++) {
            pbc_substep_kernel<<<grid_blocks(c->g.n, 256), 256, 0, c->stream>>>(
                c->g, a.ax, a.ay, a.az, a.bx, a.by, a.bz, k.abnd, u0, u1);
            FDIRW_CUDA(c, cudaGetLastError());
            std::swap(u0, u1);
        }
        widen_kernel<<<grid_blocks(c->g.n, 256), 256, 0, c->stream>>>(u0, c->g.n, c->cbuf);
        map_kernel<<<grid_blocks(k.nc, 128), 128, 0, c->stream>>>(c->g, k.liquid, k.B, k.ncx, k.ncy, k.nc, k.count,
                                                                  c->cbuf, k.pbc);
        FDIRW_CUDA(c, cudaGetLastError());
    }
    c->kernels_timed = true;
    c->parts_used = 5;
    k.built = true;
    c->kernels_ready = true;
    return FDIRW_OK;
}

int coarse_step(fdirw_ctx* c, const double* c_in, double* c_out, int32_t n_steps, double* mass_out) {
    Coarse& k = *c->coarse;
    const Kind kin = classify(c_in, c->device), kout = classify(c_out, c->device);
    if (kin == Kind::Foreign || kout == Kind::Foreign)
        return fail(c, FDIRW_ERR_ARG, "c_in/c_out are device memory of another device");
    if (!k.built) {
        const int rc = coarse_kernels(c);
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
        FDIRW_CUDA(c, launch_mass(src, c->g.n, c->partials, c->dmass, c->stream));
        FDIRW_CUDA(c, cudaMemcpyAsync(&c->mass_in, c->dmass, 8, cudaMemcpyDeviceToHost, c->stream));
    }
    if (n_steps == 0) {
        if (dst != src) FDIRW_CUDA(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, c->stream));
    } else {
        const double* cur = src;
        for (int t = 0; t < n_steps; t++) {
            map_kernel<<<grid_blocks(k.nc, 128), 128, 0, c->stream>>>(c->g, k.liquid, k.B, k.ncx, k.ncy, k.nc, k.count, cur, k.C);
            FDIRW_CUDA(c, cudaGetLastError());
            const bool last = t + 1 == n_steps;
            if (last) FDIRW_CUDA(c, cudaEventRecord(c->ev[2], c->stream));
            if (k.open) FDIRW_CUDA(c, launch_mass(cur, c->g.n, c->partials, k.far + 1, c->stream));
            coarse_gather_kernel<<<grid_blocks(k.nc, 128), 128, 0, c->stream>>>(k.ncx, k.ncy, k.ncz, k.Rc, k.Qc, k.C,
                                                                                k.open ? k.pbc : nullptr, k.far, k.Cn);
            FDIRW_CUDA(c, cudaGetLastError());
            if (last) FDIRW_CUDA(c, cudaEventRecord(c->ev[3], c->stream));
            remap_kernel<<<grid_blocks(c->g.n, 256), 256, 0, c->stream>>>(c->g, k.liquid, k.B, k.ncx, k.ncy, k.Cn, cur, dst);
            FDIRW_CUDA(c, cudaGetLastError());
            if (k.open) {
                FDIRW_CUDA(c, launch_mass(dst, c->g.n, c->partials, k.far + 2, c->stream));
                far_update_kernel<<<1, 1, 0, c->stream>>>(k.far, k.V_far);
                FDIRW_CUDA(c, cudaGetLastError());
            }
            cur = dst;
        }
        c->gather_timed = true;
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

int coarse_info(fdirw_ctx* c, fdirw_info* out) {
    out->coarse_block = c->coarse->B;
    out->coarse_nodes = c->coarse->nodes;
    out->cache_bytes = (uint64_t)(2 * c->coarse->Rc + 1) * (2 * c->coarse->Rc + 1) * (2 * c->coarse->Rc + 1) *
                       (uint64_t)c->coarse->nc * 8;
    return FDIRW_OK;
}

const uint8_t* coarse_liquid(fdirw_ctx* c) { return c->coarse ? c->coarse->liquid : nullptr; }

const float* coarse_open_faces(fdirw_ctx* c) { return (c->coarse && c->coarse->open) ? c->coarse->abnd : nullptr; }

void coarse_invalidate(fdirw_ctx* c) {
    if (c->coarse) c->coarse->built = false;
}

void coarse_release(fdirw_ctx* c) {
    Coarse* k = c->coarse;
    if (!k) return;
    void* p;
    p = k->liquid; dfree(p);
    p = k->count; dfree(p);
    p = k->list; dfree(p);
    p = k->Qc; dfree(p);
    p = k->C; dfree(p);
    p = k->Cn; dfree(p);
    p = k->abnd; dfree(p);
    p = k->pbc; dfree(p);
    p = k->far; dfree(p);
    p = k->ubuf; dfree(p);
    p = k->gs; dfree(p);
    p = k->tmp; dfree(p);
    p = k->qpart; dfree(p);
    p = k->qout; dfree(p);
    delete k;
    c->coarse = nullptr;
}

}  // namespace fdirw

extern "C" {

int fdirw_create_coarse(const fdirw_grid* grid, const double* D_map, const uint8_t* liquid, int32_t block,
                        double dt_macro, int32_t window_R, int32_t n_sub, const fdirw_opts* opts, fdirw_ctx** out) {
    if (!out) return fail(nullptr, FDIRW_ERR_ARG, "NULL out");
    *out = nullptr;
    if (!grid_ok(grid)) return fail(nullptr, FDIRW_ERR_ARG, "invalid grid (dimensions >= 1, finite h > 0)");
    if (!D_map) return fail(nullptr, FDIRW_ERR_ARG, "NULL D_map");
    if (block < 1 || block % 2 == 0) return fail(nullptr, FDIRW_ERR_ARG, "block must be odd and >= 1");
    if (window_R < 0 || window_R + (block - 1) / 2 > fdirw::kMaxR)
        return fail(nullptr, FDIRW_ERR_ARG, "need 0 <= window_R and window_R + (block - 1) / 2 <= " + std::to_string(fdirw::kMaxR));
    if (window_R + (block - 1) / 2 < 1) return fail(nullptr, FDIRW_ERR_ARG, "window_R + (block - 1) / 2 must be >= 1");
    fdirw_opts o{FDIRW_FP32, -1, nullptr, 0, 0, 0};
    if (opts) o = *opts;
    if (o.prec < FDIRW_FP32 || o.prec > FDIRW_FP32_STORE_BF16)
        return fail(nullptr, FDIRW_ERR_ARG, "the coarse path marches in FP32 (prec FP32, FP16 or BF16; P is FP64)");
    if (o.accum != FDIRW_ACCUM_FF) return fail(nullptr, FDIRW_ERR_ARG, "coarse contexts take FDIRW_ACCUM_FF only");
    // fdirw_create validates D, dt_macro, n_sub and stability and builds the face coefficients; the
    // coarse path then masks them and replaces the kernel cache with the coarse matrix.
    fdirw_opts o2 = o;
    o2.prec = FDIRW_FP32;
    fdirw_ctx* c = nullptr;
    int rc = fdirw_create(grid, D_map, dt_macro, 0, n_sub, &o2, &c);
    if (rc != FDIRW_OK) return rc;
    DeviceGuard dg(c->device);
    c->coarse = new fdirw::Coarse();
    fdirw::Coarse& k = *c->coarse;
    c->R = window_R;
    c->prec = o.prec;
    k.B = block;
    k.Rc = (window_R + block - 1) / block;
    k.Rw = window_R + (block - 1) / 2;
    k.ncx = (grid->nx + block - 1) / block;
    k.ncy = (grid->ny + block - 1) / block;
    k.ncz = (grid->nz + block - 1) / block;
    k.nc = (int64_t)k.ncx * k.ncy * k.ncz;
    const uint64_t n = (uint64_t)c->g.n;
    auto bail = [&](int code) {
        std::string msg = c->err;
        fdirw_destroy(c);
        return fail(nullptr, code, msg);
    };
    if ((rc = dalloc(c, reinterpret_cast<void**>(&k.liquid), n, "liquid mask")) != FDIRW_OK) return bail(rc);
    cudaError_t e = cudaSuccess;
    if (liquid) {
        if (classify(liquid, c->device) == Kind::Foreign) { c->err = "liquid is device memory of another device"; return bail(FDIRW_ERR_ARG); }
        e = cudaMemcpyAsync(k.liquid, liquid, n, cudaMemcpyDefault, c->stream);
    } else {
        e = cudaMemsetAsync(k.liquid, 1, n, c->stream);
    }
    if (e != cudaSuccess) { c->err = cuda_msg("copy liquid mask", e); return bail(FDIRW_ERR_CUDA); }
    if ((rc = dalloc(c, reinterpret_cast<void**>(&k.count), (uint64_t)k.nc * 4, "block counts")) != FDIRW_OK) return bail(rc);
    const uint64_t W3 = (uint64_t)(2 * k.Rc + 1) * (2 * k.Rc + 1) * (2 * k.Rc + 1);
    if ((rc = dalloc(c, reinterpret_cast<void**>(&k.Qc), W3 * (uint64_t)k.nc * 8, "coarse matrix")) != FDIRW_OK) return bail(rc);
    if ((rc = dalloc(c, reinterpret_cast<void**>(&k.C), (uint64_t)k.nc * 8, "coarse field")) != FDIRW_OK) return bail(rc);
    if ((rc = dalloc(c, reinterpret_cast<void**>(&k.Cn), (uint64_t)k.nc * 8, "coarse field")) != FDIRW_OK) return bail(rc);
    fdirw::mask_faces_kernel<<<fdirw::grid_blocks(c->g.n, 256), 256, 0, c->stream>>>(
        c->g, k.liquid, reinterpret_cast<float*>(c->coef[0]), reinterpret_cast<float*>(c->coef[1]),
        reinterpret_cast<float*>(c->coef[2]));
    fdirw::count_kernel<<<fdirw::grid_blocks(k.nc, 128), 128, 0, c->stream>>>(c->g, k.liquid, k.B, k.ncx, k.ncy, k.nc, k.count);
    if ((e = cudaGetLastError()) != cudaSuccess) { c->err = cuda_msg("coarse setup", e); return bail(FDIRW_ERR_CUDA); }
    // Blocks with liquid, ascending (host pass over the counts).
    std::vector<int32_t> cnt((size_t)k.nc);
    if ((e = cudaMemcpyAsync(cnt.data(), k.count, (size_t)k.nc * 4, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(c->stream)) != cudaSuccess) {
        c->err = cuda_msg("coarse setup", e);
        return bail(FDIRW_ERR_CUDA);
    }
    std::vector<int64_t> list;
    for (int64_t I = 0; I < k.nc; I++) if (cnt[(size_t)I] > 0) list.push_back(I);
    k.nodes = (int64_t)list.size();
    if (k.nodes > 0) {
        if ((rc = dalloc(c, reinterpret_cast<void**>(&k.list), (uint64_t)k.nodes * 8, "node list")) != FDIRW_OK) return bail(rc);
        if ((e = cudaMemcpy(k.list, list.data(), (size_t)k.nodes * 8, cudaMemcpyHostToDevice)) != cudaSuccess) {
            c->err = cuda_msg("copy node list", e);
            return bail(FDIRW_ERR_CUDA);
        }
    }
    c->kernels_ready = false;
    // Sum over the nodes of their clipped march windows (cells), for the roofline's work count.
    double wc = 0.0;
    for (int64_t I : list) {
        const int bx = (int)(I % k.ncx), by = (int)((I / k.ncx) % k.ncy), bz = (int)(I / ((int64_t)k.ncx * k.ncy));
        auto ext = [&](int b, int n) {
            return (double)(std::min(b * block + block - 1 + window_R, n - 1) - std::max(b * block - window_R, 0) + 1);
        };
        wc += ext(bx, grid->nx) * ext(by, grid->ny) * ext(bz, grid->nz);
    }
    c->window_cells = wc;
    *out = c;
    return FDIRW_OK;
}

int fdirw_coarse_far_field(fdirw_ctx* c, double V_far, double c_far) {
    if (!c) return fail(nullptr, FDIRW_ERR_ARG, "NULL context");
    if (!c->coarse) return fail(c, FDIRW_ERR_ARG, "not a coarse-mesh context");
    if (!(std::isfinite(V_far) && V_far > 0.0) || !std::isfinite(c_far))
        return fail(c, FDIRW_ERR_ARG, "V_far must be finite and > 0, c_far finite");
    DeviceGuard dg(c->device);
    fdirw::Coarse& k = *c->coarse;
    if (c->flow && !k.abnd)
        return fail(c, FDIRW_ERR_STATE, "open the far field before setting a velocity (its stability check includes the flow)");
    const uint64_t n = (uint64_t)c->g.n;
    int rc;
    if (!k.abnd) {
        if ((rc = dalloc(c, reinterpret_cast<void**>(&k.abnd), n * 4, "open-face coefficients")) != FDIRW_OK) return rc;
        if ((rc = dalloc(c, reinterpret_cast<void**>(&k.pbc), (uint64_t)k.nc * 8, "P_BC")) != FDIRW_OK) return rc;
        if ((rc = dalloc(c, reinterpret_cast<void**>(&k.far), 3 * 8, "far field")) != FDIRW_OK) return rc;
        if ((rc = dalloc(c, reinterpret_cast<void**>(&k.ubuf), 2 * n * 4, "P_BC march")) != FDIRW_OK) return rc;
        unsigned long long* mx = nullptr;
        if ((rc = dalloc(c, reinterpret_cast<void**>(&mx), 8, "flags")) != FDIRW_OK) return rc;
        unsigned long long h = 0;
        cudaError_t e = cudaMemsetAsync(mx, 0, 8, c->stream);
        if (e == cudaSuccess) {
            fdirw::open_faces_kernel<<<fdirw::grid_blocks(c->g.n, 256), 256, 0, c->stream>>>(c->g, c->Dd, k.liquid, c->lam,
                                                                                           k.abnd, mx);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h, mx, 8, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        cudaFree(mx);
        c->allocated -= 8;
        if (e != cudaSuccess) { cudaGetLastError(); return fail(c, FDIRW_ERR_CUDA, cuda_msg("open faces", e)); }
        double m;
        std::memcpy(&m, &h, 8);
        if (c->lam * m > 1.0 + 1e-12) {
            char buf[200];
            std::snprintf(buf, sizeof buf, "unstable with open faces: dt_sub*max(sum g)/h^2 = %.17g > 1", c->lam * m);
            return fail(c, FDIRW_ERR_UNSTABLE, buf);
        }
    }
    const double h3[3] = {c_far, 0.0, 0.0};
    FDIRW_CUDA(c, cudaMemcpyAsync(k.far, h3, 24, cudaMemcpyHostToDevice, c->stream));
    FDIRW_CUDA(c, cudaStreamSynchronize(c->stream));
    k.V_far = V_far;
    if (!k.open) {
        k.open = true;
        k.built = false;                 // the coarse matrix changes with open faces
        c->kernels_ready = false;
    }
    return FDIRW_OK;
}

int fdirw_coarse_get_far_field(fdirw_ctx* c, double* c_far) {
    if (!c || !c_far) return fail(c, FDIRW_ERR_ARG, "NULL context or c_far");
    if (!c->coarse || !c->coarse->open) return fail(c, FDIRW_ERR_STATE, "no far field set (fdirw_coarse_far_field)");
    DeviceGuard dg(c->device);
    FDIRW_CUDA(c, cudaMemcpyAsync(c_far, c->coarse->far, 8, cudaMemcpyDeviceToHost, c->stream));
    FDIRW_CUDA(c, cudaStreamSynchronize(c->stream));
    return FDIRW_OK;
}

int fdirw_read_coarse_pbc(fdirw_ctx* c, double* out) {
    if (!c || !out) return fail(c, FDIRW_ERR_ARG, "NULL context or out");
    if (!c->coarse || !c->coarse->open) return fail(c, FDIRW_ERR_STATE, "no far field set (fdirw_coarse_far_field)");
    if (!c->coarse->built) return fail(c, FDIRW_ERR_STATE, "coarse matrix not built (call fdirw_kernels)");
    DeviceGuard dg(c->device);
    FDIRW_CUDA(c, cudaMemcpyAsync(out, c->coarse->pbc, (size_t)c->coarse->nc * 8, cudaMemcpyDeviceToHost, c->stream));
    FDIRW_CUDA(c, cudaStreamSynchronize(c->stream));
    return FDIRW_OK;
}

int fdirw_coupled_step(fdirw_ctx* c, const fdirw_coupled_params* p, double* field, int32_t n_steps, double* QL,
                       double* QS, double* c_far) {
    if (!c || !p || !field) return fail(c, FDIRW_ERR_ARG, "NULL context, params or field");
    if (!c->coarse || !c->coarse->open)
        return fail(c, FDIRW_ERR_STATE, "the coupled step needs a coarse-mesh context with a far field");
    if (n_steps < 0) return fail(c, FDIRW_ERR_ARG, "n_steps must be >= 0");
    if (!(std::isfinite(p->k) && p->k >= 0.0) || !(std::isfinite(p->cS_eq) && p->cS_eq > 0.0) ||
        !(std::isfinite(p->cL_eq) && p->cL_eq > 0.0) || !(std::isfinite(p->dt) && p->dt >= 0.0) || p->n_sub_solid < 0)
        return fail(c, FDIRW_ERR_ARG, "need k >= 0, cS_eq > 0, cL_eq > 0, dt >= 0, n_sub_solid >= 0");
    if ((reinterpret_cast<uintptr_t>(field) & 7u) != 0) return fail(c, FDIRW_ERR_ARG, "field must be 8-byte aligned");
    DeviceGuard dg(c->device);
    fdirw::Coarse& k = *c->coarse;
    const Kind kf = classify(field, c->device);
    if (kf == Kind::Foreign) return fail(c, FDIRW_ERR_ARG, "field is device memory of another device");
    const uint64_t n = (uint64_t)c->g.n;
    int rc;
    const double lam_s = p->n_sub_solid > 0 ? (p->dt / p->n_sub_solid) / (c->h * c->h) : 0.0;
    if (!k.gs) {
        if ((rc = dalloc(c, reinterpret_cast<void**>(&k.gs), 3 * n * 8, "solid faces")) != FDIRW_OK) return rc;
        if ((rc = dalloc(c, reinterpret_cast<void**>(&k.tmp), 2 * n * 8, "coupled scratch")) != FDIRW_OK) return rc;
        if ((rc = dalloc(c, reinterpret_cast<void**>(&k.qpart), fdirw::kMassBlocks * 8, "phase partials")) != FDIRW_OK) return rc;
        fdirw::solid_faces_kernel<<<fdirw::grid_blocks(c->g.n, 256), 256, 0, c->stream>>>(c->g, c->Dd, k.liquid, k.gs,
                                                                                        k.gs + n, k.gs + 2 * n);
        FDIRW_CUDA(c, cudaGetLastError());
    }
    if (lam_s > 0.0) {
        // stability of the solid march: lam_s * max(sum of solid faces) <= 1, checked on the host once per call
        std::vector<double> gh(3 * n);
        FDIRW_CUDA(c, cudaMemcpyAsync(gh.data(), k.gs, 3 * n * 8, cudaMemcpyDeviceToHost, c->stream));
        FDIRW_CUDA(c, cudaStreamSynchronize(c->stream));
        const int nx = c->g.nx, ny = c->g.ny;
        const int64_t nxy = (int64_t)nx * ny;
        double mx = 0.0;
        for (int64_t i = 0; i < c->g.n; i++) {
            const int x = (int)(i % nx), y = (int)((i / nx) % ny);
            const int64_t z = i / nxy;
            double sum = gh[i] + gh[n + i] + gh[2 * n + i];
            if (x > 0) sum += gh[i - 1];
            if (y > 0) sum += gh[n + i - nx];
            if (z > 0) sum += gh[2 * n + i - nxy];
            mx = std::max(mx, sum);
        }
        if (lam_s * mx > 1.0 + 1e-12) return fail(c, FDIRW_ERR_UNSTABLE, "solid march unstable: raise n_sub_solid");
    }
    if ((QL || QS) && n_steps > k.qcap) {
        void* q = k.qout; dfree(q); k.qout = nullptr;
        c->allocated -= (uint64_t)k.qcap * 16;
        k.qcap = 0;
        if ((rc = dalloc(c, reinterpret_cast<void**>(&k.qout), (uint64_t)n_steps * 16, "phase masses")) != FDIRW_OK) return rc;
        k.qcap = n_steps;
    }
    if (!k.built) {
        if ((rc = fdirw::coarse_kernels(c)) != FDIRW_OK) return rc;
    }
    double* cur = field;
    if (kf == Kind::Host) {
        FDIRW_CUDA(c, cudaMemcpyAsync(c->cbuf, field, n * 8, cudaMemcpyHostToDevice, c->stream));
        cur = c->cbuf;
    }
    const int gb = fdirw::grid_blocks(c->g.n, 256);
    for (int t = 0; t < n_steps; t++) {
        fdirw::absorb_kernel<<<gb, 256, 0, c->stream>>>(c->g, k.liquid, p->k, p->cS_eq, p->cL_eq, p->dt, cur, k.tmp);
        FDIRW_CUDA(c, cudaGetLastError());
        double* a = k.tmp;
        double* b = k.tmp + n;
        for (int s = 0; s < p->n_sub_solid; s++) {
            fdirw::solid_substep_kernel<<<gb, 256, 0, c->stream>>>(c->g, k.gs, k.gs + n, k.gs + 2 * n, lam_s, a, b);
            FDIRW_CUDA(c, cudaGetLastError());
            std::swap(a, b);
        }
        if ((rc = fdirw::coarse_step(c, a, cur, 1, nullptr)) != FDIRW_OK) return rc;
        if (QL || QS) {
            for (int ph = 0; ph < 2; ph++) {
                fdirw::phase_partial_kernel<<<fdirw::kMassBlocks, 256, 0, c->stream>>>(cur, k.liquid, ph == 0, c->g.n, k.qpart);
                fdirw::phase_final_kernel<<<1, fdirw::kMassBlocks, 0, c->stream>>>(k.qpart, k.qout + 2 * t + ph);
                FDIRW_CUDA(c, cudaGetLastError());
            }
        }
    }
    if (kf == Kind::Host) FDIRW_CUDA(c, cudaMemcpyAsync(field, cur, n * 8, cudaMemcpyDeviceToHost, c->stream));
    if ((QL || QS) && n_steps > 0) {
        std::vector<double> q((size_t)n_steps * 2);
        FDIRW_CUDA(c, cudaMemcpyAsync(q.data(), k.qout, (size_t)n_steps * 16, cudaMemcpyDeviceToHost, c->stream));
        FDIRW_CUDA(c, cudaStreamSynchronize(c->stream));
        for (int t = 0; t < n_steps; t++) {
            if (QL) QL[t] = q[2 * t];
            if (QS) QS[t] = q[2 * t + 1];
        }
    }
    if (c_far) FDIRW_CUDA(c, cudaMemcpyAsync(c_far, k.far, 8, cudaMemcpyDeviceToHost, c->stream));
    if (c_far || kf == Kind::Host) FDIRW_CUDA(c, cudaStreamSynchronize(c->stream));
    return FDIRW_OK;
}

int fdirw_read_coarse(fdirw_ctx* c, const int64_t* blocks, int64_t n, double* out) {
    if (!c) return fail(nullptr, FDIRW_ERR_ARG, "NULL context");
    if (!c->coarse) return fail(c, FDIRW_ERR_ARG, "not a coarse-mesh context");
    if (n < 0 || (n > 0 && (!blocks || !out))) return fail(c, FDIRW_ERR_ARG, "bad blocks/out");
    fdirw::Coarse& k = *c->coarse;
    for (int64_t q = 0; q < n; q++)
        if (blocks[q] < 0 || blocks[q] >= k.nc) return fail(c, FDIRW_ERR_ARG, "block index out of range");
    if (!k.built) return fail(c, FDIRW_ERR_STATE, "coarse matrix not built (call fdirw_kernels)");
    if (n == 0) return FDIRW_OK;
    DeviceGuard dg(c->device);
    const int64_t W3 = (int64_t)(2 * k.Rc + 1) * (2 * k.Rc + 1) * (2 * k.Rc + 1);
    int64_t* db = nullptr;
    double* dout = nullptr;
    int rc = dalloc(c, reinterpret_cast<void**>(&db), (uint64_t)n * 8, "block list");
    if (rc != FDIRW_OK) return rc;
    rc = dalloc(c, reinterpret_cast<void**>(&dout), (uint64_t)(n * W3) * 8, "coarse readback");
    if (rc != FDIRW_OK) { cudaFree(db); c->allocated -= (uint64_t)n * 8; return rc; }
    cudaError_t e = cudaMemcpyAsync(db, blocks, (size_t)n * 8, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) {
        fdirw::read_coarse_kernel<<<fdirw::grid_blocks(n * W3, 256), 256, 0, c->stream>>>(k.Qc, k.ncx, k.ncy, k.ncz, k.Rc,
                                                                                         db, n, dout);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, (size_t)(n * W3) * 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(db);
    cudaFree(dout);
    c->allocated -= (uint64_t)n * 8 + (uint64_t)(n * W3) * 8;
    if (e != cudaSuccess) { cudaGetLastError(); return fail(c, FDIRW_ERR_CUDA, cuda_msg("read coarse matrix", e)); }
    return FDIRW_OK;
}

}  // extern "C"
