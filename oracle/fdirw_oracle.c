/*
 * FDiRW oracle: a plain, slow, FP64 CPU restatement of what the windowed FDiRW hot path computes.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load this library.  It shares no code, header, table or helper with the CUDA path.
 *
 * Method (paper: Mao, Hu, Li, "A GPU accelerated mixed-precision FDiRW solver", Sec. 3.1):
 *   Eq. 8:  c(t + dt) = p(dt) c(t)        (the boundary term p_BC c_far: the far-field functions below)
 *   Column s of p is the result of an explicit finite-difference march of the diffusion equation
 *   (Eq. 1, pure-diffusion part) from a unit point source at cell s (Sec. 3.1, text after Eq. 9).
 *   Here each source's march runs on its own window: the cube of cells within L-infinity distance R
 *   of s, clipped to the domain, with zero flux through the window faces and the domain faces.
 *   Further down: a window radius per source, the coarse mesh of Eqs. 10-15, the far-field boundary
 *   (Eqs. 7, 10, 14), the coupled macro step (Sec. 2, Eqs. 1-7) and convection (Sec. 5).
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

/* One substep with convection (Sec. 5: a steady flow folded into the computation of p).  Reading:
 * w[a][i] is the velocity through the +a face of cell i (toward +a when positive), the advective flux
 * through a face is upwind, lam_a (w+ u_lower - w- u_upper) from the lower cell to the upper one with
 * lam_a = dt_sub / h, and it adds to the diffusive flux of box_substep.  Faces on a window's or the
 * domain's edge carry neither. */
static void box_substep_adv(int nx, int ny, const double* gx, const double* gy, const double* gz,
                            const double* wx, const double* wy, const double* wz, double lam, double lama,
                            int x0, int y0, int z0, int bx, int by, int bz, const double* u, double* un)
{
    for (int l = 0; l < bz; l++)
        for (int j = 0; j < by; j++)
            for (int i = 0; i < bx; i++) {
                int64_t li = i + (int64_t)bx * (j + (int64_t)by * l);
                int64_t gi = IDX(x0 + i, y0 + j, z0 + l, nx, ny);
                int64_t sy = nx, sz = (int64_t)nx * ny, ly = bx, lz = (int64_t)bx * by;
                double ui = u[li], acc = 0.0, adv = 0.0;
                if (i > 0) {
                    acc += gx[gi - 1] * (u[li - 1] - ui);
                    double w = wx[gi - 1];
                    adv += (w > 0.0 ? w * u[li - 1] : 0.0) - (w < 0.0 ? -w * ui : 0.0);
                }
                if (i + 1 < bx) {
                    acc += gx[gi] * (u[li + 1] - ui);
                    double w = wx[gi];
                    adv -= (w > 0.0 ? w * ui : 0.0) - (w < 0.0 ? -w * u[li + 1] : 0.0);
                }
                if (j > 0) {
                    acc += gy[gi - sy] * (u[li - ly] - ui);
                    double w = wy[gi - sy];
                    adv += (w > 0.0 ? w * u[li - ly] : 0.0) - (w < 0.0 ? -w * ui : 0.0);
                }
                if (j + 1 < by) {
                    acc += gy[gi] * (u[li + ly] - ui);
                    double w = wy[gi];
                    adv -= (w > 0.0 ? w * ui : 0.0) - (w < 0.0 ? -w * u[li + ly] : 0.0);
                }
                if (l > 0) {
                    acc += gz[gi - sz] * (u[li - lz] - ui);
                    double w = wz[gi - sz];
                    adv += (w > 0.0 ? w * u[li - lz] : 0.0) - (w < 0.0 ? -w * ui : 0.0);
                }
                if (l + 1 < bz) {
                    acc += gz[gi] * (u[li + lz] - ui);
                    double w = wz[gi];
                    adv -= (w > 0.0 ? w * ui : 0.0) - (w < 0.0 ? -w * u[li + lz] : 0.0);
                }
                un[li] = ui + lam * acc + lama * adv;
            }
}

/* box_substep, or box_substep_adv when face velocities are given (wx != NULL; Sec. 5 convection). */
static void box_step(int nx, int ny, const double* gx, const double* gy, const double* gz, const double* wx,
                     const double* wy, const double* wz, double lam, double lama, int x0, int y0, int z0, int bx,
                     int by, int bz, const double* u, double* un)
{
    if (wx) box_substep_adv(nx, ny, gx, gy, gz, wx, wy, wz, lam, lama, x0, y0, z0, bx, by, bz, u, un);
    else box_substep(nx, ny, gx, gy, gz, lam, x0, y0, z0, bx, by, bz, u, un);
}

/* Spreading kernel of source s (Sec. 3.1: point-source explicit FD march, column s of p in Eq. 8),
 * on the window of radius R clipped to the domain, n_sub substeps; with face velocities (wx != NULL)
 * every substep also carries the Sec. 5 upwind faces (box_substep_adv).
 * k_out: (2R+1)^3 doubles on the offset layout, the marched field divided by its total.
 * mass_before (nullable): the total before that division (1 up to rounding: the flux form conserves).
 * Returns 0, or -1 on a bad argument or allocation failure. */
static int source_kernel_impl(int nx, int ny, int nz, const double* gx, const double* gy, const double* gz,
                              const double* wx, const double* wy, const double* wz, double lam, double lama,
                              int R, int n_sub, int64_t s, double* k_out, double* mass_before)
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
        box_step(nx, ny, gx, gy, gz, wx, wy, wz, lam, lama, x0, y0, z0, bx, by, bz, u, un);
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

int fo_source_kernel(int nx, int ny, int nz, const double* gx, const double* gy, const double* gz,
                     double lam, int R, int n_sub, int64_t s, double* k_out, double* mass_before)
{
    return source_kernel_impl(nx, ny, nz, gx, gy, gz, NULL, NULL, NULL, lam, 0.0, R, n_sub, s, k_out, mass_before);
}

/* Spreading kernel with convection (Sec. 5): face velocities w, lama = dt_sub / h. */
int fo_source_kernel_adv(int nx, int ny, int nz, const double* gx, const double* gy, const double* gz,
                         const double* wx, const double* wy, const double* wz, double lam, double lama, int R,
                         int n_sub, int64_t s, double* k_out, double* mass_before)
{
    return source_kernel_impl(nx, ny, nz, gx, gy, gz, wx, wy, wz, lam, lama, R, n_sub, s, k_out, mass_before);
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
 * Written as a scatter over sources in index order, each kernel recomputed by its march (with the Sec. 5
 * upwind faces when wx != NULL). */
static int superpose_impl(int nx, int ny, int nz, const double* gx, const double* gy, const double* gz,
                          const double* wx, const double* wy, const double* wz, double lam, double lama, int R,
                          int n_sub, const double* c_in, double* c_out)
{
    int64_t N = (int64_t)nx * ny * nz;
    int W1 = 2 * R + 1;
    double* k = (double*)malloc(sizeof(double) * (size_t)W1 * W1 * W1);
    if (!k) return -1;
    memset(c_out, 0, sizeof(double) * (size_t)N);
    for (int64_t s = 0; s < N; s++) {
        if (source_kernel_impl(nx, ny, nz, gx, gy, gz, wx, wy, wz, lam, lama, R, n_sub, s, k, NULL) != 0) {
            free(k);
            return -1;
        }
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

int fo_superpose(int nx, int ny, int nz, const double* gx, const double* gy, const double* gz,
                 double lam, int R, int n_sub, const double* c_in, double* c_out)
{
    return superpose_impl(nx, ny, nz, gx, gy, gz, NULL, NULL, NULL, lam, 0.0, R, n_sub, c_in, c_out);
}

/* Eq. 8 with convection (Sec. 5): the kernels carry the upwind faces of face velocities w. */
int fo_superpose_adv(int nx, int ny, int nz, const double* gx, const double* gy, const double* gz,
                     const double* wx, const double* wy, const double* wz, double lam, double lama, int R,
                     int n_sub, const double* c_in, double* c_out)
{
    return superpose_impl(nx, ny, nz, gx, gy, gz, wx, wy, wz, lam, lama, R, n_sub, c_in, c_out);
}

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
 * window of radius Rmap[s] (scatter over sources, as fo_superpose); with face velocities (wx != NULL) the
 * kernels carry the Sec. 5 upwind faces. */
static int superpose_rmap_impl(int nx, int ny, int nz, const double* gx, const double* gy, const double* gz,
                               const double* wx, const double* wy, const double* wz, double lama, double lam,
                               const int32_t* Rmap, int n_sub, const double* c_in, double* c_out)
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
            if (source_kernel_impl(nx, ny, nz, gx, gy, gz, wx, wy, wz, lam, lama, Rmap[s], n_sub, s,
                                   k + (s - s0) * Wm, NULL) != 0)
                bad = 1;
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

int fo_superpose_rmap(int nx, int ny, int nz, const double* gx, const double* gy, const double* gz,
                      double lam, const int32_t* Rmap, int n_sub, const double* c_in, double* c_out)
{
    return superpose_rmap_impl(nx, ny, nz, gx, gy, gz, NULL, NULL, NULL, 0.0, lam, Rmap, n_sub, c_in, c_out);
}

int fo_superpose_rmap_adv(int nx, int ny, int nz, const double* gx, const double* gy, const double* gz,
                          const double* wx, const double* wy, const double* wz, double lam, double lama,
                          const int32_t* Rmap, int n_sub, const double* c_in, double* c_out)
{
    return superpose_rmap_impl(nx, ny, nz, gx, gy, gz, wx, wy, wz, lama, lam, Rmap, n_sub, c_in, c_out);
}

/* ---- Coarse mesh (Sec. 3.1, Eqs. 10-15).  The coarsening rule is a reading (the paper takes it from its
 * ref. [12]): the grid is cut into B x B x B blocks (the last ones clipped by the domain), and the
 * liquid cells of block I form representative node I (N_I cells; a block without liquid has no node).
 * Block index I = bx + ncx (by + ncy bz), ncx = ceil(nx / B).  The fast-diffusion phase is the liquid:
 * faces with a non-liquid cell on either side carry no flux, and non-liquid cells keep their value. */

/* Zeroes the face conductances of every face that has a non-liquid cell on either side. */
void fo_mask_faces(int nx, int ny, int nz, const uint8_t* liquid, double* gx, double* gy, double* gz)
{
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                int64_t i = IDX(x, y, z, nx, ny);
                if (!liquid[i] || x + 1 >= nx || !liquid[i + 1]) gx[i] = 0.0;
                if (!liquid[i] || y + 1 >= ny || !liquid[i + nx]) gy[i] = 0.0;
                if (!liquid[i] || z + 1 >= nz || !liquid[i + (int64_t)nx * ny]) gz[i] = 0.0;
            }
}

/* Liquid-cell count of every block: cnt[ncx * ncy * ncz]. */
void fo_coarse_counts(int nx, int ny, int nz, const uint8_t* liquid, int B, int64_t* cnt)
{
    int ncx = (nx + B - 1) / B, ncy = (ny + B - 1) / B, ncz = (nz + B - 1) / B;
    memset(cnt, 0, sizeof(int64_t) * (size_t)ncx * ncy * ncz);
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++)
                if (liquid[IDX(x, y, z, nx, ny)]) cnt[(x / B) + (int64_t)ncx * ((y / B) + (int64_t)ncy * (z / B))]++;
}

/* One flux-form substep as box_substep plus the open faces: u_i += lam gb_i (ghost - u_i). */
static void box_substep_open(int nx, int ny, const double* gx, const double* gy, const double* gz,
                             const double* wxv, const double* wyv, const double* wzv, double lama,
                             const double* gb, double ghost, double lam, int x0, int y0, int z0, int bx, int by,
                             int bz, const double* u, double* un)
{
    box_step(nx, ny, gx, gy, gz, wxv, wyv, wzv, lam, lama, x0, y0, z0, bx, by, bz, u, un);
    for (int l = 0; l < bz; l++)
        for (int j = 0; j < by; j++)
            for (int i = 0; i < bx; i++) {
                int64_t li = i + (int64_t)bx * (j + (int64_t)by * l);
                int64_t gi = IDX(x0 + i, y0 + j, z0 + l, nx, ny);
                un[li] += lam * (gb[gi] * (ghost - u[li]));
            }
}

/* Column J of the coarse matrix for every block J with liquid (Sec. 3.1 for the march, Eqs. 11-12 for
 * the block means): march 1 on J's liquid cells over J's block widened by R cells (box faces closed;
 * with open = 1 the grid's outer faces also exchange with a ghost at 0 through gb), sum the marched
 * field over the liquid cells of every block of the window, and write P[I][J] = N_J S_I / (m N_I)
 * (closed: m the marched total, so each column carries N_J) or S_I / N_I (open: the mass that stays).
 * Face velocities (wxv != NULL) add the Sec. 5 upwind faces to the march. */
static int coarse_kernels_impl(int nx, int ny, int nz, const double* gx, const double* gy, const double* gz,
                               const double* wxv, const double* wyv, const double* wzv, double lama, int open,
                               const double* gb, const uint8_t* liquid, int B, double lam, int R, int n_sub,
                               double* P_band)
{
    if (B < 1 || R < 0 || n_sub < 0) return -1;
    int ncx = (nx + B - 1) / B, ncy = (ny + B - 1) / B, ncz = (nz + B - 1) / B;
    int64_t NC = (int64_t)ncx * ncy * ncz;
    int Rc = (R + B - 1) / B, Wc = 2 * Rc + 1;
    int64_t Wc3 = (int64_t)Wc * Wc * Wc;
    int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * (size_t)NC);
    if (!cnt) return -1;
    fo_coarse_counts(nx, ny, nz, liquid, B, cnt);
    memset(P_band, 0, sizeof(double) * (size_t)(NC * Wc3));
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
    for (int64_t J = 0; J < NC; J++) {
        if (cnt[J] == 0 || err) continue;
        int bx = (int)(J % ncx), by = (int)((J / ncx) % ncy), bz = (int)(J / ((int64_t)ncx * ncy));
        int x0 = bx * B - R < 0 ? 0 : bx * B - R, x1 = bx * B + B - 1 + R > nx - 1 ? nx - 1 : bx * B + B - 1 + R;
        int y0 = by * B - R < 0 ? 0 : by * B - R, y1 = by * B + B - 1 + R > ny - 1 ? ny - 1 : by * B + B - 1 + R;
        int z0 = bz * B - R < 0 ? 0 : bz * B - R, z1 = bz * B + B - 1 + R > nz - 1 ? nz - 1 : bz * B + B - 1 + R;
        int wx = x1 - x0 + 1, wy = y1 - y0 + 1, wz = z1 - z0 + 1;
        int64_t nb = (int64_t)wx * wy * wz;
        double* u = (double*)calloc((size_t)nb, sizeof(double));
        double* un = (double*)calloc((size_t)nb, sizeof(double));
        double* S = (double*)calloc((size_t)Wc3, sizeof(double));
        if (!u || !un || !S) { free(u); free(un); free(S); err = 1; continue; }
        for (int l = 0; l < wz; l++)
            for (int j = 0; j < wy; j++)
                for (int i = 0; i < wx; i++) {
                    int x = x0 + i, y = y0 + j, z = z0 + l;
                    if (x / B == bx && y / B == by && z / B == bz && liquid[IDX(x, y, z, nx, ny)])
                        u[i + (int64_t)wx * (j + (int64_t)wy * l)] = 1.0;
                }
        for (int k = 0; k < n_sub; k++) {
            if (open) box_substep_open(nx, ny, gx, gy, gz, wxv, wyv, wzv, lama, gb, 0.0, lam, x0, y0, z0, wx, wy, wz, u, un);
            else box_step(nx, ny, gx, gy, gz, wxv, wyv, wzv, lam, lama, x0, y0, z0, wx, wy, wz, u, un);
            double* t = u; u = un; un = t;
        }
        double m = 0.0;
        if (!open)
            for (int64_t q = 0; q < nb; q++) m += u[q];
        for (int l = 0; l < wz; l++)
            for (int j = 0; j < wy; j++)
                for (int i = 0; i < wx; i++) {
                    int x = x0 + i, y = y0 + j, z = z0 + l;
                    if (!liquid[IDX(x, y, z, nx, ny)]) continue;
                    int dx = x / B - bx, dy = y / B - by, dz = z / B - bz;
                    S[(dx + Rc) + (int64_t)Wc * ((dy + Rc) + (int64_t)Wc * (dz + Rc))] +=
                        u[i + (int64_t)wx * (j + (int64_t)wy * l)];
                }
        for (int dz = -Rc; dz <= Rc; dz++)
            for (int dy = -Rc; dy <= Rc; dy++)
                for (int dx = -Rc; dx <= Rc; dx++) {
                    int cx = bx + dx, cy = by + dy, cz = bz + dz;
                    if (cx < 0 || cx >= ncx || cy < 0 || cy >= ncy || cz < 0 || cz >= ncz) continue;
                    int64_t I = cx + (int64_t)ncx * (cy + (int64_t)ncy * cz);
                    if (cnt[I] == 0) continue;
                    int64_t o = (dx + Rc) + (int64_t)Wc * ((dy + Rc) + (int64_t)Wc * (dz + Rc));
                    P_band[J * Wc3 + o] = open ? S[o] / (double)cnt[I] : ((double)cnt[J] * S[o]) / (m * (double)cnt[I]);
                }
        free(u); free(un); free(S);
    }
    free(cnt);
    return err ? -1 : 0;
}

/* Column J of the coarse matrix P (Eq. 10) for every block J with liquid cells: the remapped unit
 * C_J = 1 (Eq. 12: 1 on each liquid cell of J) marched n_sub explicit substeps on the window of block J
 * widened by R cells (clipped to the domain; zero flux through its faces and through non-liquid
 * faces, which gx/gy/gz already carry), then mapped (Eq. 11): P[I][J] = N_J S_I / (m N_I), with S_I the
 * marched mass on the liquid cells of block I and m the total (N_J in exact arithmetic, so each column
 * conserves mass).  Stored source-major: P_band[J][d], d = I - J over [-Rc, Rc]^3, Rc = ceil(R / B),
 * offset layout d_x fastest; 0 where block I is outside the grid or has no liquid.  OpenMP over J. */
int fo_coarse_kernels(int nx, int ny, int nz, const double* gx, const double* gy, const double* gz,
                      const uint8_t* liquid, int B, double lam, int R, int n_sub, double* P_band)
{
    return coarse_kernels_impl(nx, ny, nz, gx, gy, gz, NULL, NULL, NULL, 0.0, 0, NULL, liquid, B, lam, R, n_sub,
                               P_band);
}

/* fo_coarse_kernels with the block-source march carrying the upwind faces of face velocities w (Sec. 5),
 * lama = dt_sub / h.  The caller zeroes w on faces that touch a non-liquid cell (no flux there). */
int fo_coarse_kernels_adv(int nx, int ny, int nz, const double* gx, const double* gy, const double* gz,
                          const double* wx, const double* wy, const double* wz, double lama, const uint8_t* liquid,
                          int B, double lam, int R, int n_sub, double* P_band)
{
    return coarse_kernels_impl(nx, ny, nz, gx, gy, gz, wx, wy, wz, lama, 0, NULL, liquid, B, lam, R, n_sub, P_band);
}

/* One coarse FDiRW step, Eqs. 13-15 without the boundary term: 'mapping' C_I = mean of c over the
 * liquid cells of block I (Eq. 13), 'FDiRW calculation' C'_I = sum_J P[I][J] C_J (Eq. 14), 're-mapping'
 * c'_i = C'_I for every liquid cell i of block I (Eq. 15); non-liquid cells keep c. */
int fo_coarse_step(int nx, int ny, int nz, const uint8_t* liquid, int B, int R, const double* P_band,
                   const double* c_in, double* c_out)
{
    int ncx = (nx + B - 1) / B, ncy = (ny + B - 1) / B, ncz = (nz + B - 1) / B;
    int64_t NC = (int64_t)ncx * ncy * ncz;
    int Rc = (R + B - 1) / B, Wc = 2 * Rc + 1;
    int64_t Wc3 = (int64_t)Wc * Wc * Wc;
    int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * (size_t)NC);
    double* C = (double*)calloc((size_t)NC, sizeof(double));
    double* Cn = (double*)calloc((size_t)NC, sizeof(double));
    if (!cnt || !C || !Cn) { free(cnt); free(C); free(Cn); return -1; }
    fo_coarse_counts(nx, ny, nz, liquid, B, cnt);
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                int64_t i = IDX(x, y, z, nx, ny);
                if (liquid[i]) C[(x / B) + (int64_t)ncx * ((y / B) + (int64_t)ncy * (z / B))] += c_in[i];
            }
    for (int64_t I = 0; I < NC; I++) if (cnt[I] > 0) C[I] /= (double)cnt[I];
    for (int64_t J = 0; J < NC; J++) {
        if (cnt[J] == 0) continue;
        int bx = (int)(J % ncx), by = (int)((J / ncx) % ncy), bz = (int)(J / ((int64_t)ncx * ncy));
        for (int dz = -Rc; dz <= Rc; dz++)
            for (int dy = -Rc; dy <= Rc; dy++)
                for (int dx = -Rc; dx <= Rc; dx++) {
                    int cx = bx + dx, cy = by + dy, cz = bz + dz;
                    if (cx < 0 || cx >= ncx || cy < 0 || cy >= ncy || cz < 0 || cz >= ncz) continue;
                    int64_t I = cx + (int64_t)ncx * (cy + (int64_t)ncy * cz);
                    Cn[I] += P_band[J * Wc3 + (dx + Rc) + (int64_t)Wc * ((dy + Rc) + (int64_t)Wc * (dz + Rc))] * C[J];
                }
    }
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                int64_t i = IDX(x, y, z, nx, ny);
                c_out[i] = liquid[i] ? Cn[(x / B) + (int64_t)ncx * ((y / B) + (int64_t)ncy * (z / B))] : c_in[i];
            }
    free(cnt); free(C); free(Cn);
    return 0;
}

/* ---- Far-field boundary (Eq. 7 and the p_BC c_far term of Eqs. 8, 10, 14), coarse path.  Reading: every
 * face of a liquid cell on the outer surface of the grid opens onto the far-field liquid, represented by
 * a ghost cell one cell width outside that holds c_far and has the cell's own diffusivity, so each open
 * face has conductance D_i; gb[i] = D_i times the number of open faces of cell i (0 for non-liquid
 * cells). */
void fo_boundary_conductance(int nx, int ny, int nz, const double* D, const uint8_t* liquid, double* gb)
{
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                int64_t i = IDX(x, y, z, nx, ny);
                int faces = (x == 0) + (x == nx - 1) + (y == 0) + (y == ny - 1) + (z == 0) + (z == nz - 1);
                gb[i] = liquid[i] ? D[i] * (double)faces : 0.0;
            }
}

/* Coarse matrix with open faces: as fo_coarse_kernels, the march also losing mass through the open
 * faces (ghost 0), and no renormalisation: P[I][J] = S_I / N_I (the column carries the mass that stays). */
int fo_coarse_kernels_open(int nx, int ny, int nz, const double* gx, const double* gy, const double* gz,
                           const double* gb, const uint8_t* liquid, int B, double lam, int R, int n_sub,
                           double* P_band)
{
    return coarse_kernels_impl(nx, ny, nz, gx, gy, gz, NULL, NULL, NULL, 0.0, 1, gb, liquid, B, lam, R, n_sub,
                               P_band);
}

/* fo_coarse_kernels_open with upwind faces (Sec. 5); the open faces stay diffusive (no flow leaves the
 * grid), and the caller zeroes w on faces that touch a non-liquid cell. */
int fo_coarse_kernels_open_adv(int nx, int ny, int nz, const double* gx, const double* gy, const double* gz,
                               const double* wx, const double* wy, const double* wz, double lama, const double* gb,
                               const uint8_t* liquid, int B, double lam, int R, int n_sub, double* P_band)
{
    return coarse_kernels_impl(nx, ny, nz, gx, gy, gz, wx, wy, wz, lama, 1, gb, liquid, B, lam, R, n_sub, P_band);
}

/* P_BC of Eq. 10: the liquid phase marched n_sub substeps over the whole grid from 0 with every ghost at
 * c_far = 1, then mapped to the blocks (Eq. 11): PBC[I] = mean over the liquid cells of block I.  With face
 * velocities (wx != NULL) the interior faces carry the upwind advective flux too. */
static int coarse_pbc_impl(int nx, int ny, int nz, const double* gx, const double* gy, const double* gz,
                           const double* wxv, const double* wyv, const double* wzv, double lama, const double* gb,
                           const uint8_t* liquid, int B, double lam, int n_sub, double* PBC)
{
    int64_t N = (int64_t)nx * ny * nz;
    int ncx = (nx + B - 1) / B, ncy = (ny + B - 1) / B, ncz = (nz + B - 1) / B;
    int64_t NC = (int64_t)ncx * ncy * ncz;
    double* u = (double*)calloc((size_t)N, sizeof(double));
    double* un = (double*)calloc((size_t)N, sizeof(double));
    int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * (size_t)NC);
    if (!u || !un || !cnt) { free(u); free(un); free(cnt); return -1; }
    for (int k = 0; k < n_sub; k++) {
        box_substep_open(nx, ny, gx, gy, gz, wxv, wyv, wzv, lama, gb, 1.0, lam, 0, 0, 0, nx, ny, nz, u, un);
        double* t = u; u = un; un = t;
    }
    fo_coarse_counts(nx, ny, nz, liquid, B, cnt);
    memset(PBC, 0, sizeof(double) * (size_t)NC);
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                int64_t i = IDX(x, y, z, nx, ny);
                if (liquid[i]) PBC[(x / B) + (int64_t)ncx * ((y / B) + (int64_t)ncy * (z / B))] += u[i];
            }
    for (int64_t I = 0; I < NC; I++) if (cnt[I] > 0) PBC[I] /= (double)cnt[I];
    free(u); free(un); free(cnt);
    return 0;
}

int fo_coarse_pbc(int nx, int ny, int nz, const double* gx, const double* gy, const double* gz, const double* gb,
                  const uint8_t* liquid, int B, double lam, int n_sub, double* PBC)
{
    return coarse_pbc_impl(nx, ny, nz, gx, gy, gz, NULL, NULL, NULL, 0.0, gb, liquid, B, lam, n_sub, PBC);
}

int fo_coarse_pbc_adv(int nx, int ny, int nz, const double* gx, const double* gy, const double* gz,
                      const double* wx, const double* wy, const double* wz, double lama, const double* gb,
                      const uint8_t* liquid, int B, double lam, int n_sub, double* PBC)
{
    return coarse_pbc_impl(nx, ny, nz, gx, gy, gz, wx, wy, wz, lama, gb, liquid, B, lam, n_sub, PBC);
}

/* One coarse step with the far field (Eqs. 13-15 with the P_BC c_far term of Eq. 14, then Eq. 7):
 * C'_I = sum_J P[I][J] C_J + PBC[I] c_far, re-mapping, and c_far_out = (M0 - sum c_out) / V_far with
 * M0 = sum c_in + V_far c_far (the total, near plus far field, that Eq. 7 conserves). */
int fo_coarse_step_far(int nx, int ny, int nz, const uint8_t* liquid, int B, int R, const double* P_band,
                       const double* PBC, double V_far, double c_far, const double* c_in, double* c_out,
                       double* c_far_out)
{
    int64_t N = (int64_t)nx * ny * nz;
    int ncx = (nx + B - 1) / B, ncy = (ny + B - 1) / B, ncz = (nz + B - 1) / B;
    int64_t NC = (int64_t)ncx * ncy * ncz;
    if (fo_coarse_step(nx, ny, nz, liquid, B, R, P_band, c_in, c_out) != 0) return -1;
    int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * (size_t)NC);
    if (!cnt) return -1;
    fo_coarse_counts(nx, ny, nz, liquid, B, cnt);
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                int64_t i = IDX(x, y, z, nx, ny);
                if (liquid[i]) c_out[i] += PBC[(x / B) + (int64_t)ncx * ((y / B) + (int64_t)ncy * (z / B))] * c_far;
            }
    free(cnt);
    double m_in = 0.0, m_out = 0.0;
    for (int64_t i = 0; i < N; i++) { m_in += c_in[i]; m_out += c_out[i]; }
    *c_far_out = (m_in + V_far * c_far - m_out) / V_far;
    return 0;
}

/* ---- Coupled macro step (Sec. 2, Eqs. 1-7) around the coarse FDiRW.  Readings: the field c holds the
 * liquid concentration on liquid cells and the solid one on the others; D is the effective diffusivity
 * D_m A_m / RT of each cell's phase (Eqs. 1-3: the flux D grad(mu/RT) with mu = A (c - c_eq)); the
 * interface exchange of Eqs. 4-6 acts on every face between a liquid cell and a solid cell, with the
 * pre-step values on both sides and the rate applied over the macro step dt (the reaction runs only
 * while c_L > cL_eq and c_S < cS_eq, as the text after Eq. 6 states, so f_S is clamped at 0 too):
 *   f_L = max(0, (c_L - cL_eq) / cL_eq),  f_S = max(0, (cS_eq - c_S) / cS_eq),  m = k f_L f_S dt,
 *   c_S += m, c_L -= m  (cell volumes equal);
 * the slow solid diffusion is the explicit flux-form march of the solid phase (faces between solid
 * cells only) with n_sub_s substeps of lam_s = (dt / n_sub_s) / h^2; then the fast liquid diffusion is
 * one coarse FDiRW step with the far field (fo_coarse_step_far). */
void fo_absorb(int nx, int ny, int nz, const uint8_t* liquid, double k, double cS_eq, double cL_eq, double dt,
               const double* c_in, double* c_out)
{
    int64_t N = (int64_t)nx * ny * nz;
    memcpy(c_out, c_in, sizeof(double) * (size_t)N);
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                int64_t i = IDX(x, y, z, nx, ny);
                int64_t nb[3];
                int has[3] = {x + 1 < nx, y + 1 < ny, z + 1 < nz};
                nb[0] = i + 1; nb[1] = i + nx; nb[2] = i + (int64_t)nx * ny;
                for (int a = 0; a < 3; a++) {
                    if (!has[a]) continue;
                    int64_t j = nb[a];
                    if (liquid[i] == liquid[j]) continue;
                    int64_t l = liquid[i] ? i : j, sd = liquid[i] ? j : i;
                    double fL = c_in[l] > cL_eq ? (c_in[l] - cL_eq) / cL_eq : 0.0;
                    double fS = c_in[sd] < cS_eq ? (cS_eq - c_in[sd]) / cS_eq : 0.0;
                    double m = k * fL * fS * dt;
                    c_out[sd] += m;
                    c_out[l] -= m;
                }
            }
}

/* Slow solid diffusion: the flux-form march of the solid phase (faces between two solid cells, harmonic
 * mean of D), n_sub substeps of lam. */
int fo_solid_march(int nx, int ny, int nz, const double* D, const uint8_t* liquid, double lam, int n_sub,
                   const double* c_in, double* c_out)
{
    int64_t N = (int64_t)nx * ny * nz;
    double* gx = (double*)malloc(sizeof(double) * (size_t)N);
    double* gy = (double*)malloc(sizeof(double) * (size_t)N);
    double* gz = (double*)malloc(sizeof(double) * (size_t)N);
    double* u = (double*)malloc(sizeof(double) * (size_t)N);
    double* un = (double*)malloc(sizeof(double) * (size_t)N);
    uint8_t* solid = (uint8_t*)malloc((size_t)N);
    if (!gx || !gy || !gz || !u || !un || !solid) {
        free(gx); free(gy); free(gz); free(u); free(un); free(solid);
        return -1;
    }
    for (int64_t i = 0; i < N; i++) solid[i] = liquid[i] ? 0 : 1;
    fo_face_conductance(nx, ny, nz, D, gx, gy, gz);
    fo_mask_faces(nx, ny, nz, solid, gx, gy, gz);
    memcpy(u, c_in, sizeof(double) * (size_t)N);
    for (int k = 0; k < n_sub; k++) {
        box_substep(nx, ny, gx, gy, gz, lam, 0, 0, 0, nx, ny, nz, u, un);
        double* t = u; u = un; un = t;
    }
    memcpy(c_out, u, sizeof(double) * (size_t)N);
    free(gx); free(gy); free(gz); free(u); free(un); free(solid);
    return 0;
}

/* Brute-force explicit FD march of a whole field over the full domain (no window), n_sub substeps:
 * the fine-mesh FD solver the paper compares against (Sec. 4.1).  By linearity (Eq. 8) it equals one
 * superposition step whenever every window covers the whole domain. */
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
