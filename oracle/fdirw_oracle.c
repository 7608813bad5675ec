/*
 * FDiRW oracle: a plain, slow, FP64 CPU restatement of what the windowed FDiRW hot path computes.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load this library.  It shares no code, header, table or helper with the CUDA path.
 *
 * Method (paper: Mao, Hu, Li, "A GPU accelerated mixed-precision FDiRW solver", Sec. 3.1):
 *   Eq. 8:  c(t + dt) = p(dt) c(t)        (the boundary term p_BC c_far is not part of this path)
 *   Column s of p is the result of an explicit finite-difference march of the diffusion equation
 *   (Eq. 1, pure-diffusion part) from a unit point source at cell s (Sec. 3.1, text after Eq. 9).
 *   Here each source's march runs on its own window: the cube of cells within L-infinity distance R
 *   of s, clipped to the domain, with zero flux through the window faces and the domain faces.
 *
 * Conventions (readings of points the paper leaves open):
 *   - grid nx*ny*nz, cell size h, index i = x + nx*(y + ny*z);
 *   - face conductance between neighbouring cells a, b: harmonic mean 2 D_a D_b / (D_a + D_b)
 *     (0 when D_a + D_b == 0);
 *   - one substep in flux form: u_i <- u_i + lam * sum_{faces f of i inside the window} g_f (u_nb - u_i),
 *     lam = dt_sub / h^2, dt_sub = dt_macro / n_sub;
 *   - a source's kernel is the marched field divided by its total (FP64 renormalisation);
 *   - kernels are reported on the (2R+1)^3 offset layout o = x - s, o_x fastest, zero outside the
 *     domain.
 *
 * Compiled with -ffp-contract=off so that results agree bit for bit across x86-64 and AArch64 hosts.
 * Every sum below is a plain left-to-right FP64 sum in the loop order written.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define IDX(x, y, z, nx, ny) ((int64_t)(x) + (int64_t)(nx) * ((int64_t)(y) + (int64_t)(ny) * (int64_t)(z)))

/* Face conductances (Eq. 1 discretised by finite differences; harmonic-mean face rule).
 * gx[i] is the face between cell i and its +x neighbour (0 on the last x plane); same for gy, gz. */
void fo_face_conductance(int nx, int ny, int nz, const double* D, double* gx, double* gy, double* gz)
{
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                int64_t i = IDX(x, y, z, nx, ny);
                double a = D[i], b;
                gx[i] = 0.0; gy[i] = 0.0; gz[i] = 0.0;
                if (x + 1 < nx) { b = D[i + 1];                       gx[i] = (a + b > 0.0) ? 2.0 * a * b / (a + b) : 0.0; }
                if (y + 1 < ny) { b = D[i + nx];                      gy[i] = (a + b > 0.0) ? 2.0 * a * b / (a + b) : 0.0; }
                if (z + 1 < nz) { b = D[i + (int64_t)nx * ny];        gz[i] = (a + b > 0.0) ? 2.0 * a * b / (a + b) : 0.0; }
            }
}

/* Largest sum of face conductances of one cell over the domain: the explicit march keeps every
 * coefficient non-negative (and is stable) when lam * this <= 1. */
double fo_max_face_sum(int nx, int ny, int nz, const double* gx, const double* gy, const double* gz)
{
    double best = 0.0;
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                int64_t i = IDX(x, y, z, nx, ny);
                double s = 0.0;
                if (x > 0) s += gx[i - 1];
                if (x + 1 < nx) s += gx[i];
                if (y > 0) s += gy[i - nx];
                if (y + 1 < ny) s += gy[i];
                if (z > 0) s += gz[i - (int64_t)nx * ny];
                if (z + 1 < nz) s += gz[i];
                if (s > best) best = s;
            }
    return best;
}

/* One explicit flux-form substep on the box [x0,x0+bx) x [y0,y0+by) x [z0,z0+bz) of the domain.
 * Only faces with both cells inside the box carry flux (zero flux through the box faces). */
static void box_substep(int nx, int ny, const double* gx, const double* gy, const double* gz, double lam,
                        int x0, int y0, int z0, int bx, int by, int bz, const double* u, double* un)
{
    for (int l = 0; l < bz; l++)
        for (int j = 0; j < by; j++)
            for (int i = 0; i < bx; i++) {
                int64_t li = i + (int64_t)bx * (j + (int64_t)by * l);
                int64_t gi = IDX(x0 + i, y0 + j, z0 + l, nx, ny);
                double ui = u[li], acc = 0.0;
                if (i > 0)      acc += gx[gi - 1] * (u[li - 1] - ui);
                if (i + 1 < bx) acc += gx[gi] * (u[li + 1] - ui);
                if (j > 0)      acc += gy[gi - nx] * (u[li - bx] - ui);
                if (j + 1 < by) acc += gy[gi] * (u[li + bx] - ui);
                if (l > 0)      acc += gz[gi - (int64_t)nx * ny] * (u[li - (int64_t)bx * by] - ui);
                if (l + 1 < bz) acc += gz[gi] * (u[li + (int64_t)bx * by] - ui);
                un[li] = ui + lam * acc;
            }
}

/* Spreading kernel of source s (Sec. 3.1: point-source explicit FD march, column s of p in Eq. 8),
 * on the window of radius R clipped to the domain, n_sub substeps.
 * k_out: (2R+1)^3 doubles on the offset layout, the marched field divided by its total.
 * mass_before (nullable): the total before that division (1 up to rounding: the flux form conserves).
 * Returns 0, or -1 on a bad argument or allocation failure. */
int fo_source_kernel(int nx, int ny, int nz, const double* gx, const double* gy, const double* gz,
                     double lam, int R, int n_sub, int64_t s, double* k_out, double* mass_before)
{
    if (R < 0 || n_sub < 0 || s < 0 || s >= (int64_t)nx * ny * nz) return -1;
    int sx = (int)(s % nx), sy = (int)((s / nx) % ny), sz = (int)(s / ((int64_t)nx * ny));
    int x0 = sx - R < 0 ? 0 : sx - R, x1 = sx + R > nx - 1 ? nx - 1 : sx + R;
    int y0 = sy - R < 0 ? 0 : sy - R, y1 = sy + R > ny - 1 ? ny - 1 : sy + R;
    int z0 = sz - R < 0 ? 0 : sz - R, z1 = sz + R > nz - 1 ? nz - 1 : sz + R;
    int bx = x1 - x0 + 1, by = y1 - y0 + 1, bz = z1 - z0 + 1;
    int64_t nb = (int64_t)bx * by * bz;
    double* u = (double*)calloc((size_t)nb, sizeof(double));
    double* un = (double*)calloc((size_t)nb, sizeof(double));
    if (!u || !un) { free(u); free(un); return -1; }
    u[(sx - x0) + (int64_t)bx * ((sy - y0) + (int64_t)by * (sz - z0))] = 1.0;
    for (int k = 0; k < n_sub; k++) {
        box_substep(nx, ny, gx, gy, gz, lam, x0, y0, z0, bx, by, bz, u, un);
        double* t = u; u = un; un = t;
    }
    double m = 0.0;
    for (int64_t q = 0; q < nb; q++) m += u[q];
    if (mass_before) *mass_before = m;
    int W1 = 2 * R + 1;
    memset(k_out, 0, sizeof(double) * (size_t)W1 * W1 * W1);
    for (int l = 0; l < bz; l++)
        for (int j = 0; j < by; j++)
            for (int i = 0; i < bx; i++) {
                int ox = x0 + i - sx, oy = y0 + j - sy, oz = z0 + l - sz;
                k_out[(ox + R) + (int64_t)W1 * ((oy + R) + (int64_t)W1 * (oz + R))] =
                    u[i + (int64_t)bx * (j + (int64_t)by * l)] / m;
            }
    free(u); free(un);
    return 0;
}

/* Kernels of a list of sources (the precomputed coefficient matrix of Sec. 3.1, one column per
 * listed source).  out: n_src * (2R+1)^3 doubles; masses (nullable): n_src totals before renormalising.
 * Sources are independent, so they are spread over OpenMP threads; each writes only its own slice. */
int fo_kernels(int nx, int ny, int nz, const double* gx, const double* gy, const double* gz,
               double lam, int R, int n_sub, const int64_t* sources, int64_t n_src,
               double* out, double* masses)
{
    int64_t W = (int64_t)(2 * R + 1) * (2 * R + 1) * (2 * R + 1);
    int err = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(| : err)
    for (int64_t q = 0; q < n_src; q++) {
        double m = 0.0;
        err |= fo_source_kernel(nx, ny, nz, gx, gy, gz, lam, R, n_sub, sources[q], out + q * W, &m) != 0;
        if (masses) masses[q] = m;
    }
    return err ? -1 : 0;
}

/* One superposition step, Eq. 8 (and Eq. 14 on the full mesh): c_out(x) = sum_s c_in(s) k_s(x).
 * Written as a scatter over sources in index order, each kernel recomputed by its march. */
int fo_superpose(int nx, int ny, int nz, const double* gx, const double* gy, const double* gz,
                 double lam, int R, int n_sub, const double* c_in, double* c_out)
{
    int64_t N = (int64_t)nx * ny * nz;
    int W1 = 2 * R + 1;
    double* k = (double*)malloc(sizeof(double) * (size_t)W1 * W1 * W1);
    if (!k) return -1;
    memset(c_out, 0, sizeof(double) * (size_t)N);
    for (int64_t s = 0; s < N; s++) {
        if (fo_source_kernel(nx, ny, nz, gx, gy, gz, lam, R, n_sub, s, k, NULL) != 0) { free(k); return -1; }
        int sx = (int)(s % nx), sy = (int)((s / nx) % ny), sz = (int)(s / ((int64_t)nx * ny));
        for (int oz = -R; oz <= R; oz++)
            for (int oy = -R; oy <= R; oy++)
                for (int ox = -R; ox <= R; ox++) {
                    int x = sx + ox, y = sy + oy, z = sz + oz;
                    if (x < 0 || x >= nx || y < 0 || y >= ny || z < 0 || z >= nz) continue;
                    c_out[IDX(x, y, z, nx, ny)] += c_in[s] * k[(ox + R) + (int64_t)W1 * ((oy + R) + (int64_t)W1 * (oz + R))];
                }
    }
    free(k);
    return 0;
}

/* Brute-force explicit FD march of a whole field over the full domain (no window), n_sub substeps:
 * the fine-mesh FD solver the paper compares against (Sec. 4.1).  By linearity (Eq. 8) it equals one
 * superposition step whenever every window covers the whole domain. */
/* Per-source window radius from the local diffusivity (not in the paper, which has no window; reading
 * of the batched variant): twice the diffusion length sqrt(2 D dt_macro) of the macro step, in cells,
 * rounded up and clamped:  R(s) = clamp(ceil(2 sqrt(2 D(s) dt_macro) / h), R_min, R_max).
 * Evaluated in FP64 in exactly this order: t = 2 D; t = t dt_macro; r = sqrt(t); r = 2 r; r = r / h. */
void fo_radius_map(int64_t N, const double* D, double dt_macro, double h, int R_min, int R_max, int32_t* Rmap)
{
    for (int64_t s = 0; s < N; s++) {
        double t = 2.0 * D[s];
        t = t * dt_macro;
        double r = sqrt(t);
        r = 2.0 * r;
        r = r / h;
        double c = ceil(r);
        int R = c > (double)R_max ? R_max : (int)c;
        Rmap[s] = R < R_min ? R_min : R;
    }
}

/* Eq. 8 with a radius per source: c_out(x) = sum_s c_in(s) k_s(x), k_s the kernel of s on its own
 * window of radius Rmap[s] (scatter over sources, as fo_superpose). */
int fo_superpose_rmap(int nx, int ny, int nz, const double* gx, const double* gy, const double* gz,
                      double lam, const int32_t* Rmap, int n_sub, const double* c_in, double* c_out)
{
    enum { CHUNK = 256 };
    int64_t N = (int64_t)nx * ny * nz;
    int Rmax = 0;
    for (int64_t s = 0; s < N; s++) {
        if (Rmap[s] < 0) return -1;
        if (Rmap[s] > Rmax) Rmax = Rmap[s];
    }
    int64_t Wm = (int64_t)(2 * Rmax + 1) * (2 * Rmax + 1) * (2 * Rmax + 1);
    double* k = (double*)malloc(sizeof(double) * (size_t)(Wm * CHUNK));
    if (!k) return -1;
    memset(c_out, 0, sizeof(double) * (size_t)N);
    int bad = 0;
    for (int64_t s0 = 0; s0 < N && !bad; s0 += CHUNK) {
        int64_t s1 = s0 + CHUNK < N ? s0 + CHUNK : N;
        /* kernels of a chunk of sources in parallel (independent), then the scatter in source order */
        #pragma omp parallel for schedule(dynamic, 1) reduction(|:bad)
        for (int64_t s = s0; s < s1; s++)
            if (fo_source_kernel(nx, ny, nz, gx, gy, gz, lam, Rmap[s], n_sub, s, k + (s - s0) * Wm, NULL) != 0) bad = 1;
        if (bad) break;
        for (int64_t s = s0; s < s1; s++) {
            const double* ks = k + (s - s0) * Wm;
            int R = Rmap[s], W1 = 2 * R + 1;
            int sx = (int)(s % nx), sy = (int)((s / nx) % ny), sz = (int)(s / ((int64_t)nx * ny));
            for (int oz = -R; oz <= R; oz++)
                for (int oy = -R; oy <= R; oy++)
                    for (int ox = -R; ox <= R; ox++) {
                        int x = sx + ox, y = sy + oy, z = sz + oz;
                        if (x < 0 || x >= nx || y < 0 || y >= ny || z < 0 || z >= nz) continue;
                        c_out[IDX(x, y, z, nx, ny)] += c_in[s] * ks[(ox + R) + (int64_t)W1 * ((oy + R) + (int64_t)W1 * (oz + R))];
                    }
        }
    }
    free(k);
    return bad ? -1 : 0;
}

int fo_full_march(int nx, int ny, int nz, const double* gx, const double* gy, const double* gz,
                  double lam, int n_sub, const double* c_in, double* c_out)
{
    int64_t N = (int64_t)nx * ny * nz;
    double* u = (double*)malloc(sizeof(double) * (size_t)N);
    double* un = (double*)malloc(sizeof(double) * (size_t)N);
    if (!u || !un) { free(u); free(un); return -1; }
    memcpy(u, c_in, sizeof(double) * (size_t)N);
    for (int k = 0; k < n_sub; k++) {
        box_substep(nx, ny, gx, gy, gz, lam, 0, 0, 0, nx, ny, nz, u, un);
        double* t = u; u = un; un = t;
    }
    memcpy(c_out, u, sizeof(double) * (size_t)N);
    free(u); free(un);
    return 0;
}

/* Total mass of a field (Eq. 7: the conserved total; cells have equal volume h^3). */
double fo_mass(const double* c, int64_t n)
{
    double m = 0.0;
    for (int64_t i = 0; i < n; i++) m += c[i];
    return m;
}
