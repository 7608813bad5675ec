// Face conductances and explicit-march coefficients (Eq. 1 discretised by finite differences).
//
// HBM-bound elementwise work done once per context: reads D (8 B/cell), writes three FP64 face arrays,
// then the lam-scaled coefficient arrays.  Not on the per-step path.
#include "fdirw_internal.h"

#include <cmath>

namespace fdirw {

namespace {

// Harmonic-mean conductance of the face between a lower-index cell (a) and a higher-index cell (b).
__device__ __forceinline__ double face_g(double a, double b) {
    return (a + b > 0.0) ? 2.0 * a * b / (a + b) : 0.0;
}

__global__ void conductance_kernel(const double* __restrict__ D, Grid g, double* __restrict__ gx,
                                   double* __restrict__ gy, double* __restrict__ gz,
                                   unsigned long long* max_bits, unsigned long long* bad) {
    const int64_t nxy = (int64_t)g.nx * g.ny;
    unsigned long long local_max = 0ull;
    unsigned long long local_bad = 0ull;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % g.nx);
        const int64_t r = i / g.nx;
        const int y = (int)(r % g.ny);
        const int z = (int)(r / g.ny);
        const double a = D[i];
        if (!(a >= 0.0) || !isfinite(a)) { local_bad++; }
        const double fxp = (x + 1 < g.nx) ? face_g(a, D[i + 1]) : 0.0;
        const double fyp = (y + 1 < g.ny) ? face_g(a, D[i + g.nx]) : 0.0;
        const double fzp = (z + 1 < g.nz) ? face_g(a, D[i + nxy]) : 0.0;
        gx[i] = fxp;
        gy[i] = fyp;
        gz[i] = fzp;
        // Sum of the cell's face conductances, in the order -x, +x, -y, +y, -z, +z.
        double s = 0.0;
        if (x > 0) s += face_g(D[i - 1], a);
        if (x + 1 < g.nx) s += fxp;
        if (y > 0) s += face_g(D[i - g.nx], a);
        if (y + 1 < g.ny) s += fyp;
        if (z > 0) s += face_g(D[i - nxy], a);
        if (z + 1 < g.nz) s += fzp;
        if (s >= 0.0 && isfinite(s)) {
            const unsigned long long b = (unsigned long long)__double_as_longlong(s);
            local_max = b > local_max ? b : local_max;
        }
    }
    // Non-negative doubles order like their bit patterns, so max over bits is max over values.
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, local_max, off);
        local_max = o > local_max ? o : local_max;
        local_bad += __shfl_xor_sync(0xffffffffu, local_bad, off);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(max_bits, local_max);
        if (local_bad) atomicAdd(bad, local_bad);
    }
}

__global__ void coef_f32_kernel(const double* __restrict__ g, double lam, int64_t n, float* __restrict__ c) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        c[i] = (float)(lam * g[i]);
}

__global__ void coef_f64_kernel(double* __restrict__ g, double lam, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        g[i] = lam * g[i];
}

int grid_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b > 152 * 32) b = 152 * 32;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_conductance(const double* D, Grid g, double* gx, double* gy, double* gz,
                               unsigned long long* max_bits, unsigned long long* bad, cudaStream_t st) {
    conductance_kernel<<<grid_for(g.n, 256), 256, 0, st>>>(D, g, gx, gy, gz, max_bits, bad);
    return cudaGetLastError();
}

cudaError_t launch_coef_f32(const double* g, double lam, int64_t n, float* coef, cudaStream_t st) {
    coef_f32_kernel<<<grid_for(n, 256), 256, 0, st>>>(g, lam, n, coef);
    return cudaGetLastError();
}

cudaError_t launch_coef_f64(double* g, double lam, int64_t n, cudaStream_t st) {
    coef_f64_kernel<<<grid_for(n, 256), 256, 0, st>>>(g, lam, n);
    return cudaGetLastError();
}

}  // namespace fdirw
