// Convection folded into the march (Sec. 5: a steady flow changes only the coefficients of p, not the
// superposition).  Upwind faces: across the +a face of cell i (velocity w, positive toward +a) the lower
// cell i sends lam g + lam_a w+ of its value to the upper cell and receives lam g + lam_a w- of the
// upper cell's, with lam = dt_sub / h^2 and lam_a = dt_sub / h.  The two coefficients replace the
// symmetric lam g of the diffusion-only march: A (lower into upper) in the context's coefficient arrays,
// B (upper into lower) in a second set, and the march runs mapping 5 with direction-dependent faces.
// On a coarse-mesh context the liquid mask closes faces touching non-liquid cells for both fluxes, and
// the block-source march and the P_BC march use the same coefficients; open faces stay diffusive.
#include "fdirw.h"
#include "fdirw_internal.h"
#include "ctx.h"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace fdirw::host;

namespace fdirw {
namespace {

int grid_blocks(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b > 152 * 16) b = 152 * 16;
    return (int)(b < 1 ? 1 : b);
}

__device__ __forceinline__ double harmonic(double a, double b) {
    return (a + b > 0.0) ? 2.0 * a * b / (a + b) : 0.0;
}

// A and B of the +x, +y, +z face of every cell (FP32, one rounding from FP64), 0 on the last plane and,
// with a liquid mask, on faces touching a non-liquid cell; and the largest per-cell sum of outflow
// coefficients, open faces included (bits of a non-negative double, for atomicMax) for the stability
// check, +inf where a velocity that enters the march is NaN or infinite.
__global__ void flow_coef_kernel(Grid g, const double* __restrict__ D, const double* __restrict__ w, int64_t ws,
                                 const uint8_t* __restrict__ liquid, bool open, double lam, double lama,
                                 float* __restrict__ A, float* __restrict__ Bc, int64_t os,
                                 unsigned long long* __restrict__ max_bits) {
    const int64_t nxy = (int64_t)g.nx * g.ny;
    const int64_t stride[3] = {1, g.nx, nxy};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x) {
        const int c3[3] = {(int)(i % g.nx), (int)((i / g.nx) % g.ny), (int)(i / nxy)};
        const int n3[3] = {g.nx, g.ny, g.nz};
        double out = 0.0;
        for (int ax = 0; ax < 3; ax++) {
            // +face of cell i
            double a = 0.0, b = 0.0;
            if (c3[ax] + 1 < n3[ax]) {
                const int64_t j = i + stride[ax];
                const double wv = w[ax * ws + i];
                if (!liquid || (liquid[i] && liquid[j])) {
                    const double gd = lam * harmonic(D[i], D[j]);
                    a = gd + lama * (wv > 0.0 ? wv : 0.0);
                    b = gd + lama * (wv < 0.0 ? -wv : 0.0);
                }
                if (!isfinite(wv)) out = INFINITY;          // reported as invalid input, never installed
            }
            A[ax * os + i] = (float)a;
            Bc[ax * os + i] = (float)b;
            out += a;                                   // outflow from i through its +face
            // -face of cell i: outflow is the lower neighbour's B
            if (c3[ax] > 0) {
                const int64_t j = i - stride[ax];
                if (!liquid || (liquid[i] && liquid[j])) {
                    const double gd = lam * harmonic(D[j], D[i]);
                    const double wv = w[ax * ws + j];
                    out += gd + lama * (wv < 0.0 ? -wv : 0.0);
                }
            }
        }
        if (open && liquid && liquid[i]) {                // open faces (far field): diffusive outflow D_i per face
            const int faces = (c3[0] == 0) + (c3[0] == g.nx - 1) + (c3[1] == 0) + (c3[1] == g.ny - 1) +
                              (c3[2] == 0) + (c3[2] == g.nz - 1);
            out += lam * (D[i] * (double)faces);
        }
        atomicMax(max_bits, (unsigned long long)__double_as_longlong(out));
    }
}

}  // namespace
}  // namespace fdirw

extern "C" {

int fdirw_set_velocity(fdirw_ctx* c, const double* w) {
    if (!c) return fail(nullptr, FDIRW_ERR_ARG, "NULL context");
    if (c->store == fdirw::Store::F64) return fail(c, FDIRW_ERR_ARG, "convection needs an FP32-march precision");
    if (!w) return fail(c, FDIRW_ERR_ARG, "NULL velocity field");
    if ((reinterpret_cast<uintptr_t>(w) & 7u) != 0) return fail(c, FDIRW_ERR_ARG, "w must be 8-byte aligned");
    DeviceGuard dg(c->device);
    if (classify(w, c->device) == Kind::Foreign) return fail(c, FDIRW_ERR_ARG, "w is device memory of another device");
    const uint64_t n = (uint64_t)c->g.n;
    int rc;
    if (!c->coefb[0]) {
        for (int a = 0; a < 3; a++)
            if ((rc = dalloc(c, &c->coefb[a], n * 4, "upwind coefficients")) != FDIRW_OK) return rc;
    }
    double* dw = nullptr;
    unsigned long long* mx = nullptr;
    if ((rc = dalloc(c, reinterpret_cast<void**>(&dw), 3 * n * 8, "velocity staging")) != FDIRW_OK) return rc;
    if ((rc = dalloc(c, reinterpret_cast<void**>(&mx), 8, "flags")) != FDIRW_OK) {
        cudaFree(dw);
        c->allocated -= 3 * n * 8;
        return rc;
    }
    // The coefficient arrays are contiguous per axis in this file's kernel; the context keeps three
    // separate allocations, so stage A and B in one block and copy them out.
    float* AB = nullptr;
    if ((rc = dalloc(c, reinterpret_cast<void**>(&AB), 6 * n * 4, "coefficient staging")) != FDIRW_OK) {
        cudaFree(dw); cudaFree(mx);
        c->allocated -= 3 * n * 8 + 8;
        return rc;
    }
    unsigned long long h = 0;
    cudaError_t e = cudaMemcpyAsync(dw, w, 3 * n * 8, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(mx, 0, 8, c->stream);
    if (e == cudaSuccess) {
        if (c->batch) {
            // Every structure with its own grid, lam and h; w, A and B span the concatenated cells.
            std::vector<fdirw::Grid> grids;
            std::vector<int64_t> base;
            std::vector<double> lams, hs;
            fdirw::batch_structures(c, grids, base, lams, hs);
            for (size_t i = 0; i < grids.size() && e == cudaSuccess; i++) {
                fdirw::flow_coef_kernel<<<fdirw::grid_blocks(grids[i].n, 256), 256, 0, c->stream>>>(
                    grids[i], c->Dd + base[i], dw + base[i], (int64_t)n, nullptr, false, lams[i], lams[i] * hs[i],
                    AB + base[i], AB + 3 * n + base[i], (int64_t)n, mx);
                e = cudaGetLastError();
            }
        } else {
            const uint8_t* liquid = c->coarse ? fdirw::coarse_liquid(c) : nullptr;
            const bool open = c->coarse && fdirw::coarse_open_faces(c) != nullptr;
            fdirw::flow_coef_kernel<<<fdirw::grid_blocks(c->g.n, 256), 256, 0, c->stream>>>(
                c->g, c->Dd, dw, (int64_t)n, liquid, open, c->lam, c->lam * c->h, AB, AB + 3 * n, (int64_t)n, mx);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, mx, 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    double m = 0.0;
    std::memcpy(&m, &h, 8);
    const bool stable = m <= 1.0 + 1e-12;
    // Install the coefficients only when the march stays stable with them.
    for (int a = 0; a < 3 && e == cudaSuccess && stable; a++) {
        e = cudaMemcpyAsync(c->coef[a], AB + a * n, n * 4, cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->coefb[a], AB + (3 + a) * n, n * 4, cudaMemcpyDeviceToDevice, c->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(dw);
    cudaFree(mx);
    cudaFree(AB);
    c->allocated -= 3 * n * 8 + 8 + 6 * n * 4;
    if (e != cudaSuccess) { cudaGetLastError(); return fail(c, FDIRW_ERR_CUDA, cuda_msg("velocity coefficients", e)); }
    if (!std::isfinite(m)) return fail(c, FDIRW_ERR_ARG, "w holds NaN or infinite values");
    if (!stable) {
        char buf[200];
        std::snprintf(buf, sizeof buf, "unstable with convection: largest outflow coefficient sum %.17g > 1", m);
        return fail(c, FDIRW_ERR_UNSTABLE, buf);
    }
    c->kernels_ready = false;
    c->flow = true;
    if (c->coarse) fdirw::coarse_invalidate(c);        // P and P_BC are rebuilt with the flow
    if (c->batch) fdirw::batch_invalidate(c);          // every chunk's kernels, and the captured graph
    return FDIRW_OK;
}

}  // extern "C"
