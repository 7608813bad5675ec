/*
 * fdirw.h -- C ABI of the GB300 FDiRW hot path (libfdirw.so).
 *
 * FDiRW (Finite Difference informed Random Walker; Mao, Hu & Li, Sec. 3.1) advances a fast diffusion
 * process over a long macro step dt by superposing precomputed mass proportions:
 *
 *     c(t + dt) = p(dt) c(t)                                            (Eq. 8, without the p_BC term)
 *
 * where column s of p is obtained by an explicit finite-difference march of the diffusion equation
 * (Eq. 1, pure-diffusion part) from a unit point source at cell s (Sec. 3.1, text after Eq. 9).
 * This library computes every column at full grid resolution on a local window: the cube of cells
 * within L-infinity distance R of the source, clipped to the domain, with zero flux through the window
 * faces and the domain faces.  The stored columns form a banded operator (the "kernel cache");
 * one macro step is then a deterministic gather  c'(x) = sum_o K_o(x) * sigma(x-o) * c(x-o).
 *
 * Discretisation (readings of points the paper leaves open):
 *   - grid nx*ny*nz of cubic cells of side h; cell index i = x + nx*(y + ny*z) (x fastest);
 *   - face conductance between neighbouring cells a, b: harmonic mean 2 D_a D_b / (D_a + D_b)
 *     (0 if D_a + D_b == 0);
 *   - substep dt_sub = dt_macro / n_sub, lam = dt_sub / h^2; one substep
 *     u_i <- u_i + lam * sum_{faces f of i inside window and domain} g_f (u_nb - u_i);
 *   - explicit stability (all coefficients >= 0): lam * max_i(sum of the face conductances of i) <= 1;
 *   - each stored column is renormalised to unit total mass in FP64 (sigma, below).
 *
 * Conventions of this API:
 *   - Pointers to fields (D_map, c_in, c_out) may be host or device memory (detected with
 *     cudaPointerGetAttributes); device pointers must live on the context's device.  Arrays are
 *     float64, N = nx*ny*nz elements, x fastest, and are owned by the caller.
 *   - Work is issued on the stream given at creation (NULL = legacy default stream).  A call that
 *     returns data in host memory (mass_out, a host c_out, fdirw_read_kernels, fdirw_stable_dt)
 *     synchronises that stream before returning; otherwise calls return as soon as the work is queued.
 *   - Every int-returning call returns FDIRW_OK (0) or a negative FDIRW_ERR_* code, and then
 *     fdirw_last_error() describes the failure.  No call aborts the process.
 *   - A context is not thread-safe: use one context per host thread or serialise calls.
 */
#ifndef FDIRW_H
#define FDIRW_H

#include <stdint.h>

#if defined(__GNUC__)
#define FDIRW_API __attribute__((visibility("default")))
#else
#define FDIRW_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define FDIRW_OK            0
#define FDIRW_ERR_ARG      -1   /* invalid argument (bad size, NaN/Inf/negative D, bad pointer, ...) */
#define FDIRW_ERR_UNSTABLE -2   /* lam * max face-conductance sum > 1 (explicit march would not be stable) */
#define FDIRW_ERR_NOMEM    -3   /* device allocation failed or would exceed opts.mem_limit */
#define FDIRW_ERR_CUDA     -4   /* a CUDA runtime call failed (message has the CUDA error string) */
#define FDIRW_ERR_TIMEOUT  -5   /* a bounded device-side wait gave up (the surrogate's MMA-completion waits, 2 s each) */
#define FDIRW_ERR_STATE    -6   /* call not valid in the context's current state */

/* Arithmetic of the path (Sec. 3.3: lower precision for the stored proportions, higher precision for
 * accumulation; Table 2 lists the paper's FP64 / FP32 / FP32-FP16 variants). */
typedef enum {
    FDIRW_FP64            = 0,  /* FP64 march, FP64 storage, FP64 gather: the plain FP64 path           */
    FDIRW_FP32            = 1,  /* FP32 march, FP32 storage, FP64 renormalisation, extended accumulation */
    FDIRW_FP32_STORE_FP16 = 2,  /* FP32 march, FP16 storage of the kernel cache, same renorm/accumulation */
    FDIRW_FP32_STORE_BF16 = 3   /* FP32 march, BF16 storage of the kernel cache, same renorm/accumulation */
} fdirw_prec;

/* Accumulation of the superposition for the FP32-march precisions (fdirw_opts.accum; Sec. 3.3: the
 * products in the storage precision, the sums in a higher one).  Both keep the fixed summation order, so
 * results are reproducible bit for bit. */
typedef enum {
    FDIRW_ACCUM_FF   = 0,  /* every row of 2R+1 products summed as an error-free FP32 pair (exact products,
                              TwoSum), the rows of a destination as a double-float pair: within a few 1e-15
                              of FP64 summation; the total mass follows from the per-source renormalisation */
    FDIRW_ACCUM_FP32 = 1   /* FP32 products and FP32 sums along each row (2 operations per term, so the
                              step runs at the HBM rate of the cache stream), the rows as a double-float
                              pair; the rounding of the row sums is not mass-neutral, so after every macro
                              step the field's FP64 total is restored to the total of the call's input:
                              c'(x) += (M_in - S) |c'(x)| / A with S = sum c', A = sum |c'| (FP64,
                              fixed order), a change of the size of the FP32 rounding (~1e-8 relative).
                              Batch contexts restore every structure's total separately, and their rare
                              radii (source-indexed cache) keep the float-float sums */
} fdirw_accum;

typedef struct {
    int32_t nx, ny, nz;   /* cells per axis, each >= 1 */
    double  h;            /* cell size, > 0 */
} fdirw_grid;

typedef struct {
    int32_t  prec;        /* fdirw_prec */
    int32_t  device;      /* CUDA device ordinal; -1 = the calling thread's current device */
    void*    stream;      /* cudaStream_t for all work; NULL = legacy default stream */
    uint64_t mem_limit;   /* cap on the device bytes this context allocates; 0 = no cap */
    int32_t  march_parts; /* FP32 march thread mapping: 1..3 = threads per window column; 4 = one thread
                             per 2x2 block of window columns with the face coefficients in Tensor Memory;
                             5 = one thread per window column with its lateral face coefficients in
                             Tensor Memory; 6 = one thread per window column for a pair of sources,
                             packed f32x2 arithmetic, lateral faces of both in Tensor Memory (R <= 8);
                             7 = one thread per pair of x-adjacent window columns with their lateral faces
                             and diagonals in Tensor Memory;
                             window_R 9 and 10 take 4, 5 or 7 only (another request is autotuned between
                             those three); 0 = autotune (each candidate timed once on the first build for a device, R
                             and storage type, result cached for the process; that build synchronises the
                             stream) */
    int32_t  accum;       /* fdirw_accum; FDIRW_ACCUM_FP32 needs an FP32-march precision and an fdirw_create
                             or batch context (coarse-mesh contexts take FDIRW_ACCUM_FF only) */
} fdirw_opts;

typedef struct {
    int64_t  n_cells;        /* N */
    int32_t  window_R;       /* R */
    int32_t  n_sub;          /* substeps per macro step */
    int32_t  prec;           /* fdirw_prec in use */
    int32_t  kernels_ready;  /* 1 once the kernel cache holds the current kernels */
    double   dt_sub;         /* dt_macro / n_sub */
    double   lam;            /* dt_sub / h^2 */
    double   max_face_sum;   /* max over cells of the sum of its face conductances */
    uint64_t cache_bytes;    /* bytes of the kernel cache (N * (2R+1)^3 * storage size) */
    uint64_t device_bytes;   /* all device bytes held by the context */
    double   window_cells;   /* sum over sources of their clipped window sizes */
    float    kernels_ms;     /* device time of the last kernel-cache build (march kernel only) */
    float    last_gather_ms; /* device time of the last gather launch */
    double   last_mass_in;   /* FP64 total of c_in at the last fdirw_step */
    double   last_mass_out;  /* FP64 total of c_out after the last fdirw_step (if it was computed) */
    int32_t  march_parts;    /* thread mapping of the last kernel-cache build (see fdirw_opts) */
    int32_t  accum;          /* fdirw_accum in use */
    int32_t  n_structures;   /* batch contexts: number of structures (0 for fdirw_create contexts) */
    int32_t  n_chunks;       /* batch contexts: structure chunks whose kernels are built one at a time;
                                fdirw_create contexts: z-slabs of a streamed cache (1 when resident) */
    int32_t  window_R_min;   /* batch contexts: R_min of the radius rule */
    int32_t  graph_launches; /* batch contexts: CUDA graph launches so far (one per fdirw_step call) */
    int32_t  dest_indexed_radii; /* batch contexts: bit r set when radius r's kernels are stored
                                    destination-indexed (radii on >= 20% of the cells), else source-indexed */
    int32_t  coarse_block;   /* coarse-mesh contexts: block side B (0 otherwise) */
    int64_t  coarse_nodes;   /* coarse-mesh contexts: representative nodes (blocks with liquid cells) */
    double   last_restore_drift; /* FDIRW_ACCUM_FP32 on fdirw_create contexts: the largest |M_in - S| / |M_in|
                                    over the macro steps of the last fdirw_step call, S the FP64 total of a
                                    step's FP32-accumulated field before its mass restoration (0 otherwise) */
} fdirw_info;

typedef struct fdirw_ctx fdirw_ctx;

/* Largest stable substep for a diffusivity map: h^2 / max_i(sum of face conductances of cell i),
 * +inf (HUGE_VAL) when every conductance is 0.  D_map: N float64 values (host or device), finite, >= 0.
 * Synchronises.  Errors: FDIRW_ERR_ARG (bad grid, NULL pointer, NaN/Inf/negative D), FDIRW_ERR_CUDA,
 * FDIRW_ERR_NOMEM. */
FDIRW_API int fdirw_stable_dt(const fdirw_grid* grid, const double* D_map, int32_t device, double* dt_sub_max);

/* Create a context for one diffusivity map (Sec. 3.1: p is fixed while the domain is fixed, Sec. 5).
 *   grid       : grid dimensions and cell size
 *   D_map      : N cell diffusivities (host or device), finite and >= 0; copied, not retained
 *   dt_macro   : macro step (>= 0, finite); dt_sub = dt_macro / n_sub
 *   window_R   : window radius, 0 <= R <= 10; <= 8 with FDIRW_FP64 (R = 0 gives the identity operator)
 *   n_sub      : explicit substeps per macro step, >= 0 (0 gives the identity operator)
 *   opts       : NULL for defaults (FDIRW_FP32, current device, default stream, no cap, autotune)
 *   out        : receives the context (set to NULL on failure)
 * Computes the face conductances on the device and checks stability; the kernel cache is built
 * lazily (fdirw_kernels or the first fdirw_step).  Errors: FDIRW_ERR_ARG, FDIRW_ERR_UNSTABLE,
 * FDIRW_ERR_NOMEM, FDIRW_ERR_CUDA. */
FDIRW_API int fdirw_create(const fdirw_grid* grid, const double* D_map, double dt_macro, int32_t window_R,
                 int32_t n_sub, const fdirw_opts* opts, fdirw_ctx** out);

/* Build (or rebuild) the kernel cache: for every source cell s, march a unit mass over its window for
 * n_sub substeps (Sec. 3.1), store the result in the storage precision and sigma_s = 1 / (FP64 sum of
 * the stored values).  Idempotent; asynchronous on the context stream.  When the whole cache
 * (N (2R+1)^3 values) does not fit the device's free memory (less 1 GiB) or mem_limit, the context
 * streams it instead: the cache holds T destination z-planes (as many as fit next to an N-double
 * buffer) and every fdirw_step marches, slab by slab, the sources within R planes of the slab before
 * gathering it (the same results bit for bit, at the cost of a march per step; fdirw_info.n_chunks gives
 * the number of slabs); fdirw_kernels then builds nothing.
 * Errors: FDIRW_ERR_ARG (NULL ctx), FDIRW_ERR_NOMEM (not even one z-plane fits), FDIRW_ERR_CUDA. */
FDIRW_API int fdirw_kernels(fdirw_ctx* ctx);

/* Advance a field n_steps macro steps with the superposition c' = p c (Eq. 8, Eq. 14):
 *   c_in, c_out : N float64 values each (host or device); c_in == c_out is allowed (in place)
 *   n_steps     : >= 0 (0 copies c_in to c_out)
 *   mass_out    : host pointer or NULL; receives the FP64 total of c_out (Eq. 7), computed on the
 *                 device with a fixed reduction order
 * Builds the kernel cache first if needed.  Results are bitwise reproducible for a given context
 * configuration (no atomics in the gather).  Errors: FDIRW_ERR_ARG, FDIRW_ERR_NOMEM, FDIRW_ERR_CUDA. */
FDIRW_API int fdirw_step(fdirw_ctx* ctx, const double* c_in, double* c_out, int32_t n_steps, double* mass_out);

/* FP64 total of a field (host or device, N values) with the library's fixed reduction order.
 * Synchronises.  Errors: FDIRW_ERR_ARG, FDIRW_ERR_CUDA. */
FDIRW_API int fdirw_mass(fdirw_ctx* ctx, const double* c, double* mass_out);

/* Copy renormalised kernels out of the cache: for each of n source indices, (2R+1)^3 float64 values on
 * the offset layout o = x - s (o_x fastest, index (ox+R) + (2R+1)*((oy+R) + (2R+1)*(oz+R))), equal to
 * stored value * sigma_s, and 0 where x is outside the domain.  sources: host int64 array; out: host
 * float64 array of n*(2R+1)^3.  Synchronises.  Errors: FDIRW_ERR_ARG (index out of range),
 * FDIRW_ERR_STATE (cache not built, or streamed by z-slabs), FDIRW_ERR_CUDA, FDIRW_ERR_NOMEM. */
FDIRW_API int fdirw_read_kernels(fdirw_ctx* ctx, const int64_t* sources, int64_t n, double* out);

/* Snapshot of the context's configuration and last timings.  Synchronises on the timing events. */
FDIRW_API int fdirw_get_info(fdirw_ctx* ctx, fdirw_info* out);

/* Release all device memory held by the context.  NULL-safe. */
FDIRW_API void fdirw_destroy(fdirw_ctx* ctx);

/* Create one context for a batch of n independent structures whose sources use per-source window radii
 * (the paper has one domain and no window; Sec. 3.1 and Eq. 8 apply per structure).
 *   n          : number of structures, >= 1; the total cell count must stay below 2^28
 *   grids      : n grids (dimensions, cell size h_i)
 *   D_maps     : n pointers to the structures' cell diffusivities (host or device, each 8-byte aligned,
 *                finite, >= 0); copied, not retained
 *   dt_macro   : macro step shared by all structures (dt_sub = dt_macro / n_sub; each structure is
 *                checked against its own stability limit)
 *   R_min/R_max: clamp of the radius rule R(s) = clamp(ceil(2 sqrt(2 D(s) dt_macro) / h_i), R_min,
 *                R_max), evaluated in FP64 in that order; 0 <= R_min <= R_max <= 10
 *   n_sub      : explicit substeps per macro step, >= 0
 *   opts       : as for fdirw_create; prec must be FDIRW_FP32, FDIRW_FP32_STORE_FP16 or
 *                FDIRW_FP32_STORE_BF16; mem_limit (or, when 0, the free device memory less a reserve)
 *                bounds the kernel cache
 * Fields passed to fdirw_step / fdirw_mass are the concatenation of the structures' fields, structure 0
 * first, each x-fastest.  When the kernels of all structures do not fit the budget, the structures are
 * split into chunks of consecutive structures and each fdirw_step call builds the kernels of one chunk,
 * runs all n_steps macro steps on its cells and moves to the next (so pass all steps in one call); the
 * device work of an fdirw_step call runs as one CUDA graph (captured on first use for the given fields
 * and step count, replayed afterwards).  fdirw_read_kernels (sources as global cell indices, output on
 * the (2 R_max + 1)^3 layout, zero outside a source's own window) needs a single chunk.
 * Errors: FDIRW_ERR_ARG, FDIRW_ERR_UNSTABLE, FDIRW_ERR_NOMEM (a single structure's kernels exceed the
 * budget), FDIRW_ERR_CUDA. */
FDIRW_API int fdirw_create_batch(int32_t n, const fdirw_grid* grids, const double* const* D_maps, double dt_macro,
                                 int32_t R_min, int32_t R_max, int32_t n_sub, const fdirw_opts* opts,
                                 fdirw_ctx** out);

/* Coarse-mesh FDiRW (Sec. 3.1, Eqs. 10-15, without the boundary term p_BC c_far).  The liquid cells of
 * each block x block x block cube of the grid (block odd; cubes clipped by the domain keep their cells)
 * form one representative node I with N_I cells; faces with a non-liquid cell on either side carry no
 * flux and non-liquid cells keep their value (the paper's liquid phase; its coarsening rule is in its
 * ref. [12], this cube grouping is this library's reading).  Column J of the coarse matrix P (Eq. 10) is
 * the remapped unit of node J (1 on its liquid cells, Eq. 12) marched n_sub explicit substeps on the
 * node's cube widened by window_R cells (clipped; zero flux through its faces), then mapped (Eq. 11):
 * P[I][J] = N_J S_I / (m N_I), S_I the marched mass on node I's cells and m the total, in FP64 from the
 * FP32 march.  fdirw_step then applies, per macro step, the mapping C_I = mean of c over node I (Eq. 13),
 * C' = P C (Eq. 14) and the re-mapping c'_i = C'_I on node I's liquid cells (Eq. 15); fdirw_kernels
 * builds P (lazily otherwise), fdirw_mass and fdirw_get_info work as for fdirw_create contexts.
 *   liquid   : N bytes (host or device), nonzero = liquid; NULL = every cell liquid; copied
 *   block    : cube side B, odd, >= 1; window_R + (B - 1) / 2 must lie in [1, 10]
 *   opts.prec: FDIRW_FP32, FDIRW_FP32_STORE_FP16 or FDIRW_FP32_STORE_BF16 (the march is FP32 in every
 *              case and P is stored FP64)
 * Errors: as fdirw_create. */
FDIRW_API int fdirw_create_coarse(const fdirw_grid* grid, const double* D_map, const uint8_t* liquid, int32_t block,
                                  double dt_macro, int32_t window_R, int32_t n_sub, const fdirw_opts* opts,
                                  fdirw_ctx** out);

/* Columns of the coarse matrix for listed nodes (block indices bx + ncx (by + ncy bz), ncx = ceil(nx / B)):
 * out[n][(2 Rc + 1)^3] on the block-offset layout d = I - J (d_x fastest, Rc = ceil(window_R / B)), 0 where
 * block J + d is outside the grid or has no liquid.  Needs the matrix built (FDIRW_ERR_STATE otherwise). */
FDIRW_API int fdirw_read_coarse(fdirw_ctx* ctx, const int64_t* blocks, int64_t n, double* out);

/* Far-field boundary of a coarse-mesh context (the p_BC c_far term of Eqs. 8, 10 and 14, and Eq. 7).
 * Opens every face of a liquid cell on the grid's outer surface onto the far-field liquid, represented
 * by a ghost cell one cell width outside that holds c_far and has the cell's own diffusivity
 * (conductance D_i per open face; this ghost is this library's reading).  The coarse matrix is rebuilt
 * with those faces (its columns then keep the mass that stays, unrenormalised), P_BC is the liquid
 * marched from 0 with every ghost at 1 over the whole grid, mapped to the nodes, and each macro step
 * becomes C' = P C + P_BC c_far followed by the Eq. 7 update c_far <- (m_in + V_far c_far - m_out) /
 * V_far (m = FP64 total of the field before and after the step), so that the near- plus far-field total
 * is conserved.  Calling it again only resets c_far.
 *   V_far : far-field volume in cell volumes (> 0, finite); c_far: its current concentration (finite)
 * Errors: FDIRW_ERR_ARG (not a coarse context, bad values), FDIRW_ERR_UNSTABLE (the open faces push
 * dt_sub * max(sum g) / h^2 above 1), FDIRW_ERR_STATE (the first call after fdirw_set_velocity: open the
 * far field before setting a velocity), FDIRW_ERR_NOMEM, FDIRW_ERR_CUDA. */
FDIRW_API int fdirw_coarse_far_field(fdirw_ctx* ctx, double V_far, double c_far);

/* Current far-field concentration (after the last fdirw_step).  Synchronises the context stream.
 * Errors: FDIRW_ERR_ARG, FDIRW_ERR_STATE (no far field set). */
FDIRW_API int fdirw_coarse_get_far_field(fdirw_ctx* ctx, double* c_far);

/* P_BC of every block (n_blocks doubles, host), once built.  Errors: FDIRW_ERR_ARG, FDIRW_ERR_STATE. */
FDIRW_API int fdirw_read_coarse_pbc(fdirw_ctx* ctx, double* out);

/* Parameters of the coupled macro step (Sec. 2): interface exchange (Eqs. 4-6) and slow solid diffusion
 * around the coarse FDiRW.  k: rate constant; cS_eq, cL_eq: equilibrium concentrations (> 0); dt: the
 * macro step; n_sub_solid: explicit substeps of the solid march within dt (0 = no solid diffusion). */
typedef struct {
    double  k;
    double  cS_eq;
    double  cL_eq;
    double  dt;
    int32_t n_sub_solid;
    int32_t reserved;      /* must be 0 */
} fdirw_coupled_params;

/* n_steps coupled macro steps on a coarse-mesh context with a far field (fdirw_coarse_far_field), in
 * place on field (N float64, host or device; each cell holds the concentration of its own phase: liquid
 * cells the liquid one, the others the solid one).  The context's D map is read as the effective
 * diffusivity D_m A_m / RT of each cell's phase (Eqs. 1-3).  Each step: (1) interface exchange on every
 * liquid/solid face with the pre-step values, m = k f_L f_S dt, f_L = max(0, (c_L - cL_eq) / cL_eq),
 * f_S = max(0, (cS_eq - c_S) / cS_eq) (the reaction runs only while c_L > cL_eq and c_S < cS_eq), the
 * solid cell gaining m and the liquid cell losing it; (2) the solid phase marched n_sub_solid FP64
 * flux-form substeps of lam = (dt / n_sub_solid) / h^2 over solid-solid faces (harmonic mean of D);
 * (3) one coarse FDiRW step of the liquid with the far-field term and the Eq. 7 update.  QL, QS
 * (nullable, host, n_steps each): FP64 totals of the liquid and solid cells after every step; c_far
 * (nullable): the far-field concentration after the last step.  The exchange and the solid march are
 * explicit: parameters that move more than a cell holds within dt are the caller's to avoid.
 * Errors: FDIRW_ERR_ARG, FDIRW_ERR_STATE (not a coarse context with a far field), FDIRW_ERR_UNSTABLE
 * (the solid march), FDIRW_ERR_NOMEM, FDIRW_ERR_CUDA. */
FDIRW_API int fdirw_coupled_step(fdirw_ctx* ctx, const fdirw_coupled_params* params, double* field, int32_t n_steps,
                                 double* QL, double* QS, double* c_far);

/* Convection (Sec. 5, where a steady flow is said to change only the computation of the spreading
 * kernels p, not the superposition of Eq. 8).  w: 3 * n_cells float64 (host or device, 8-byte aligned),
 * w[a * n_cells + i] the velocity through the +a face of cell i (a = 0, 1, 2 for x, y, z; positive toward
 * +a; the value on a cell of the last plane of axis a is ignored).  Every substep of the per-source march
 * then carries, across each interior face, the diffusive flux lam g (u_lower - u_upper) plus the upwind
 * advective flux lam_a (w+ u_lower - w- u_upper), lam = dt_sub / h^2, lam_a = dt_sub / h, w+ = max(w, 0),
 * w- = max(-w, 0); window and domain edges stay closed.  The face coefficients are rounded once to FP32
 * and the march runs mapping 5 (direction-dependent faces); the superposition is unchanged.  On a
 * coarse-mesh context faces touching a non-liquid cell carry neither flux, the block-source march and
 * the P_BC march use the same faces, and the far field's open faces stay diffusive (open the far field
 * first: its stability check then includes the flow).  On a batch context w spans the concatenated cells
 * (structure i at its first global cell) and each structure uses its own lam, h and radius.  A second
 * call replaces the velocity; the kernels
 * (or P and P_BC) are recomputed by the next fdirw_kernels / fdirw_step.  With w = 0 the kernels and
 * steps are bit for bit those without a velocity.  Synchronises the context stream.
 * Errors: FDIRW_ERR_ARG (NULL or misaligned w, NaN or infinite values, FDIRW_FP64 precision),
 * FDIRW_ERR_UNSTABLE (some cell's outflow coefficients sum above 1; the previous velocity, if
 * any, stays in place), FDIRW_ERR_NOMEM, FDIRW_ERR_CUDA. */
FDIRW_API int fdirw_set_velocity(fdirw_ctx* ctx, const double* w);

/* Window radius of every source (n_cells int32 values, host): the radius rule's value for batch
 * contexts, window_R for fdirw_create contexts.  Synchronises the context stream. */
FDIRW_API int fdirw_read_radius(fdirw_ctx* ctx, int32_t* out);

/* Message of the last failed call on ctx, or of the last failed call on this host thread when ctx is
 * NULL (for failures of fdirw_create / fdirw_stable_dt / fdirw_mass_noalloc).  Never NULL; the string
 * stays valid until the next call on the same context / thread. */
FDIRW_API const char* fdirw_last_error(const fdirw_ctx* ctx);

/* ---------------------------------------------------------------------------------------------------
 * Learned surrogate of the spreading kernel (no counterpart in the paper: it predicts the column of p of
 * Sec. 3.1 that the FD march computes, and the march stays its fallback).
 *
 * Network: features of source s on the 17^3 patch centred on s -- clamp(log10 D / 8 + 1, -0.5, 1.5) and a
 * domain mask in the domain (0 outside), a source marker at the centre, and on every voxel its offset o
 * from the source as o_x / 8, o_y / 8, o_z / 8 and |o|^2 / 256 (channels 0-6; 7-15 are 0) -- then 4 convolutions (3^3
 * taps, 16 -> 16 channels, zero padding, bias) with ReLU after the first three, BF16 weights and
 * activations, FP32 accumulation on the tensor cores; head y = exp(z[channel 0]) on in-domain cells.
 * Gate: a prediction is accepted when |sum y - 1| <= 1e-3 (FP64 sum).
 * Parameters (host float arrays of FDIRW_NET_NPARAM values): weights [4][27][16 co][16 ci] (tap index
 * (dx+1) + 3(dy+1) + 9(dz+1)), then biases [4][16].  Only output channel 0 of layer 4 is used (its
 * other weights and biases must be 0 and are kept at 0 by training).
 * Sources are host int64 arrays of cell indices of the context's grid; per call at most 1024 sources.
 * Kernel arrays are n * 17^3 float64 values, offset o = (i-8, j-8, k-8) at index i + 17 (j + 17 k), host or
 * device memory.  The calls run on the context's stream and synchronise it before returning.  The first
 * surrogate call on a context stores feature channel 0 of every cell there (grid cells x 2 bytes, freed
 * with the context); it returns FDIRW_ERR_NOMEM if that exceeds the context's mem_limit. */
#define FDIRW_NET_NPARAM (4 * 27 * 16 * 16 + 4 * 16)
typedef struct fdirw_net fdirw_net;

/* Creates a network from host parameters on `device` (-1 = current).  Errors: FDIRW_ERR_ARG, FDIRW_ERR_CUDA. */
FDIRW_API int fdirw_net_create(const float* params, int32_t device, fdirw_net** out);
/* Copies the current FP32 parameters to host memory. */
FDIRW_API int fdirw_net_params(fdirw_net* net, float* params_out);
FDIRW_API void fdirw_net_destroy(fdirw_net* net);
/* Predicted kernels (unnormalised head output y, nullable), their FP64 masses (host, nullable) and gate
 * decisions (host int32, nullable) for n sources of ctx's domain. */
FDIRW_API int fdirw_net_predict(fdirw_ctx* ctx, fdirw_net* net, const int64_t* sources, int64_t n,
                                double* kernels_out, double* mass_out, int32_t* accept_out);
/* Gradients of the training loss sum_i sum_v (y_iv - k_iv z_iv + k_iv ln k_iv - k_iv) (the generalised
 * Kullback-Leibler divergence; k = targets, z = the head's pre-exponential output, y = exp(z), in-domain
 * cells only, 0 ln 0 = 0; its gradient with respect to z is y - k) with respect to the parameters (host,
 * FDIRW_NET_NPARAM floats, nullable) and the mean loss over the batch (host, nullable). */
FDIRW_API int fdirw_net_gradients(fdirw_ctx* ctx, fdirw_net* net, const int64_t* sources, int64_t n,
                                  const double* targets, float* grads_out, double* loss_out);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8) on the mean of those gradients; loss_out as above. */
FDIRW_API int fdirw_net_train_step(fdirw_ctx* ctx, fdirw_net* net, const int64_t* sources, int64_t n,
                                   const double* targets, float lr, double* loss_out);
/* Builds the kernel cache with the network: every source is predicted, accepted predictions are stored
 * (rounded to the storage type, sigma = 1 / FP64 sum of the stored values), and the rejected sources are
 * marched with the FD march.  Needs window_R = 8 and an FP32-march precision.  accepted_out (host,
 * nullable) receives the number of accepted sources.  Errors: FDIRW_ERR_ARG, FDIRW_ERR_NOMEM,
 * FDIRW_ERR_CUDA, FDIRW_ERR_TIMEOUT (a convolution's bounded wait on its MMAs gave up). */
FDIRW_API int fdirw_kernels_surrogate(fdirw_ctx* ctx, fdirw_net* net, int64_t* accepted_out);
/* Intermediate values of the network for n sources (1..1024), for checking it element by element
 * against a reference implementation.  Volumes are [n][16 channels][17^3] with voxel v = i + 17 (j + 17 k)
 * of the patch (offset (i-8, j-8, k-8)); BF16 values are returned as their 16-bit patterns.  All outputs
 * are nullable and may be host or device memory.
 *   acts_out  : [4][n][16][17^3] BF16: the input of each layer (layer 0's is the feature volume, layers
 *               1..3 the relu outputs of the layer below), as the convolutions read them
 *   z_out     : [n][17^3] float: the head's pre-exponential output z (channel 0 plus its bias)
 *   targets   : nullable; with targets (n * 17^3 float64, host or device) the backward pass runs too:
 *   grads_out : [4][n][16][17^3] BF16: entry l is the gradient of the loss of fdirw_net_gradients with
 *               respect to layer l's output (for l < 3 after the relu mask), as the weight gradient reads it
 *   grads_param_out : FDIRW_NET_NPARAM floats, the parameter gradients summed over the batch
 *   loss_out  : the mean loss over the batch
 * Synchronises the context stream; allocates one staging volume for the BF16 outputs.  Errors:
 * FDIRW_ERR_ARG, FDIRW_ERR_STATE (the network gave up on running MMAs earlier), FDIRW_ERR_NOMEM,
 * FDIRW_ERR_CUDA, FDIRW_ERR_TIMEOUT. */
FDIRW_API int fdirw_net_trace(fdirw_ctx* ctx, fdirw_net* net, const int64_t* sources, int64_t n,
                              const double* targets, uint16_t* acts_out, float* z_out, uint16_t* grads_out,
                              float* grads_param_out, double* loss_out);
/* Device time (ms, host float) of the four tensor-core convolutions of the network's last forward pass
 * (prediction, training step, gradients, trace or gated build batch), from CUDA events recorded on the
 * context stream around them; 0 before the first forward pass.  Errors: FDIRW_ERR_ARG, FDIRW_ERR_CUDA. */
FDIRW_API int fdirw_net_timing(fdirw_net* net, float* conv_ms);
/* Failure-injection hook for tests of the bounded wait.  Every convolution and weight-gradient kernel waits
 * for its copies and MMAs on mbarriers for at most wait_ns nanoseconds of the GPU's global timer (0 restores
 * the default, 2 s).  With withhold_mma != 0 those kernels issue neither their MMAs nor the commits that
 * complete the waits, so the waits run out with nothing in flight: the call returns FDIRW_ERR_TIMEOUT, the
 * kernels have freed their tensor memory, and the network stays usable once the hook is cleared.  A wait that runs out
 * while MMAs were issued is waited once more; if they still have not completed, the call returns
 * FDIRW_ERR_TIMEOUT and every later call on this network returns FDIRW_ERR_STATE (the tensor memory it
 * released may still be written).  Errors: FDIRW_ERR_ARG (NULL net). */
FDIRW_API int fdirw_net_test_wait(fdirw_net* net, uint64_t wait_ns, int32_t withhold_mma);

/* FP64 total of a device field without allocating any memory.  The paper has no counterpart: this is a
 * library service for callers that may not call cudaMalloc when they need the mass budget -- a host
 * framework that owns and pre-partitions all device memory, a real-time loop in which an allocation (and
 * the synchronisation it can imply) is not allowed, or a caller that holds no fdirw context (creating one
 * allocates).  The reduction scratch is a fixed array compiled into the library: 2^14 FP64 partial sums
 * (128 KiB per GPU, held from the library's load until the process exits), one per chunk of 2^16 cells.
 *   c        : n float64 values in device memory of the current device (x fastest; any layout works);
 *              may be NULL when n = 0 (the total written is then 0)
 *   n        : 0 <= n <= 2^30 (larger fields are rejected with FDIRW_ERR_ARG: they need more partials
 *              than the fixed scratch holds)
 *   mass_out : one float64 in device memory of the current device; receives the total
 *   stream   : cudaStream_t to launch on (NULL = legacy default stream); the call is asynchronous
 * The first call on a device looks the scratch address up (cudaGetSymbolAddress) and caches it: make that
 * first call before any stream capture.  All calls share the scratch, so calls whose kernels may overlap
 * on the GPU (unordered streams or host threads) race and can return wrong totals; order them.  Nothing in
 * the scratch needs clearing (each call writes every partial it reads).  The reduction order is fixed,
 * so the result is reproducible; it can differ from fdirw_mass in the last bits (different chunking).
 * Errors: FDIRW_ERR_ARG (n out of range, NULL, misaligned or non-device pointers), FDIRW_ERR_CUDA; the
 * message is available from fdirw_last_error(NULL). */
FDIRW_API int fdirw_mass_noalloc(const double* c, int64_t n, double* mass_out, void* stream);

/* Peaks of a GPU for roofline reports (no counterpart in the paper; a measuring service beside the method).
 *   device           : CUDA device (-1 = current); the current device is restored afterwards
 *   fp32_flops       : host, nullable: FP32 flop/s of a register-only loop of independent FMAs (2 flop
 *                      each) over 4 blocks of 512 threads per SM, best of three timed runs after one warm-up
 *   read_bytes_per_s : host, nullable: bytes/s of a streaming read (16-byte loads, four in flight per
 *                      thread) of a 4 GiB device buffer, larger than L2, best of three after one warm-up
 * Allocates and frees the 4 GiB buffer; synchronises the device.  Errors: FDIRW_ERR_NOMEM, FDIRW_ERR_CUDA;
 * the message is available from fdirw_last_error(NULL). */
FDIRW_API int fdirw_probe_peaks(int32_t device, double* fp32_flops, double* read_bytes_per_s);

#ifdef __cplusplus
}
#endif

#endif /* FDIRW_H */
