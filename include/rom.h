/*
 * rom.h -- C ABI of the GB300 (sm_103a) Random Ordinate Method library.
 *
 * The library solves the steady radiative transport equation
 *     u . grad psi + sigma_T psi = sigma_S fint_S P(u', u) psi(u') du' + q,
 *     psi = psi_Gamma on the inflow boundary (u . n < 0),
 * (Li, Tang & Yang, arXiv 2407.12527, Sec. 1, eq. equ_1 / equ_1_bc) in X-Y
 * geometry, or in 3D (x-y-z) geometry where eq. equ_1 is posed (the paper
 * tests only slab and X-Y), by the Random Ordinate Method (Sec. 3.1): for each of several
 * ordinate sets ("samples") it solves the discrete ordinate system of
 * eq. (equ_random) with inflow eq. (equ_random_bd), discretised in space by
 * diamond difference on a uniform Cartesian grid with cell-centred unknowns
 * (Sec. 2), by classical source iteration (Sec. 3.2, eq. psiexpansion), and
 * averages the scalar fluxes over the samples (Sec. 4.1).  Every step runs in
 * hand-written CUDA kernels; there is no CPU fallback.
 *
 * Conventions shared by every call:
 *   - A context is used by one host thread at a time.  All device work of a
 *     context is issued on its stream (rom_set_stream), in order.
 *   - Cell arrays are [J][I] (2D) or [K][J][I] (3D), x fastest, cell (i, j, k)
 *     centred at (x_L + (i + 1/2) dx, y_B + (j + 1/2) dy, z_B + (k + 1/2) dz),
 *     i = 0..I-1, j = 0..J-1, k = 0..K-1.
 *   - Input buffers are read during the call and never kept: the caller keeps
 *     ownership and may reuse them as soon as the call returns (device inputs
 *     of the *_device calls are copied on the context stream, and the call
 *     waits for that copy).  Output buffers are caller-allocated.
 *   - Every call returns ROM_OK (0) or a negative ROM_ERR_* code; the message
 *     of the last error of a context is returned by rom_last_error.  A CUDA
 *     error inside a call is reported as ROM_ERR_CUDA and leaves the context
 *     in need of rom_destroy.
 *   - Arithmetic: sweeps and source updates in FP32, the source-iteration
 *     residual norms and the sample average in FP64.  Sweeps add each work
 *     item's (one to four ordinates') contribution to its sample's flux
 *     moments with atomic FP32 vector additions, so the order of the terms,
 *     and the last bits of phi, can differ from run to run.
 */
#ifndef ROM_GB300_H
#define ROM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define ROM_OK 0
#define ROM_ERR_INVALID_ARG (-1)   /* bad size, pointer, range, sigma_S >= sigma_T, q < 0 ... */
#define ROM_ERR_CUDA (-2)          /* a CUDA runtime call or kernel failed                    */
#define ROM_ERR_OOM (-3)           /* device or host allocation failed                         */
#define ROM_ERR_NOT_CONVERGED (-4) /* some sample reached max_iter above tol                   */
#define ROM_ERR_DIVERGED (-5)      /* a residual became NaN/Inf, or the change kept growing    */
#define ROM_ERR_STATE (-6)         /* call made before the data it needs was set               */
#define ROM_ERR_UNSUPPORTED (-7)   /* combination not built (e.g. an anisotropic kernel in 3D) */
#define ROM_ERR_TIMEOUT (-8)       /* a bounded wait between the warps of a sweep ran out      */

/* --------------------------------------------------------------- choices */
#define ROM_SCHEME_DD 0   /* diamond difference (Sec. 2)                      */
#define ROM_SCHEME_STEP 1 /* upwind step scheme (positive; not in the paper) */

#define ROM_KERNEL_ISO 0    /* P = 1                                              */
#define ROM_KERNEL_LINEAR 1 /* P = 1 + g cos(xi), eq. (anisotropic kernel)         */
#define ROM_KERNEL_HG 2     /* Henyey-Greenstein (1-g^2)/(1+g^2-2g cos xi)^{3/2}   */

#define ROM_KERNEL_FLAG_NORMALIZE 1 /* divide row l by sum_l' w_l' P(u_l', u_l)  (Remark, Sec. 3.1) */
#define ROM_KERNEL_FLAG_RAW 2       /* use G(cc'+ss'+zz') instead of the mirror average in zeta    */

#define ROM_FACE_XL 0 /* x = x_L */
#define ROM_FACE_XR 1 /* x = x_R */
#define ROM_FACE_YB 2 /* y = y_B */
#define ROM_FACE_YT 3 /* y = y_T */
#define ROM_FACE_ZB 4 /* z = z_B (3D) */
#define ROM_FACE_ZT 5 /* z = z_T (3D) */

#define ROM_QUAD_UNIFORM 0    /* 2D uniform set, Appendix A eq. (uniform2D): n1 = N, M = 4 N^2      */
#define ROM_QUAD_GAUSS 1      /* 2D Gaussian set, Appendix A: n1 = N, M = 2 N (N + 1)               */
#define ROM_QUAD_PRODUCT_GL 2 /* n1 positive Gauss-Legendre polar cosines x n2 azimuths, M = n1 n2 */

typedef struct rom_ctx rom_ctx; /* opaque */

/* Solver options (rom_default_options fills the defaults shown). */
typedef struct rom_options {
    int scheme;      /* ROM_SCHEME_DD                                                     */
    int max_iter;    /* 10000: cap on source-iteration sweeps per sample                  */
    double tol;      /* 1e-6: a sample stops when ||phi^k - phi^{k-1}||_2 < tol ||phi^k||_2 */
    int fixed_iters; /* 0; > 0 runs exactly this many sweeps for every sample, tol unused  */
    int check_every; /* 0 = device-side loop (one CUDA graph with a conditional node);     */
                     /* > 0: the host reads the number of unconverged samples after every  */
                     /* check_every sweeps                                                 */
    int tile_g;      /* ordinates per sweep work item: 1, 2 or 4; 0 = chosen from the      */
                     /* problem size; -1 = measured: at the first solve of a problem layout */
                     /* every candidate is timed on a few sweeps and the fastest is kept   */
                     /* (until the grid, the ordinate layout or the kernel changes)        */
    int time_kernels;/* 0; 1 records CUDA events around every sweep launch (host-driven     */
                     /* loop, check_every >= 1 is then used, 1 if it is 0) and reports the  */
                     /* summed sweep-kernel time in rom_stats.sweep_ms                     */
    int dense_source;/* 0: the scattering source from angular moments when the kernel has  */
                     /* them (isotropic; linear without flags), else from the dense        */
                     /* M x M operator; 1: always the dense operator                       */
    int dense_precision; /* the dense operator's product: 0 FP32 (CUDA cores); 1 split     */
                     /* BF16 on the tensor cores (tcgen05: (A_hi + A_lo)(Psi_hi + Psi_lo), */
                     /* all four products, FP32 accumulate, v_hi = v rounded to BF16, v_lo = */
                     /* bf16(v - v_hi); psi kept as BF16 hi/lo, the bytes of FP32; at most */
                     /* 128 ordinates per sample and 2048 samples per context, else        */
                     /* ROM_ERR_UNSUPPORTED)                                               */
    int rows_per_step; /* X-Y sweep: grid rows a lane advances per wavefront step; 0 = 4,  */
                     /* or the measured choice with tile_g = -1 (1, 2 or 4); 1, 2 or 4     */
                     /* forces it (2 only in the isotropic and linear-kernel moment modes: */
                     /* the dense operator mode runs 4 then; 1 solves each lane's 8-cell   */
                     /* upwind recurrence as a prefix of affine maps); other values are    */
                     /* ROM_ERR_INVALID_ARG                                                */
    int diverge_window; /* 16: a sample whose change ||phi^k - phi^{k-1}||_2 grew in this  */
                     /* many consecutive sweeps (while above tol) stops as diverged         */
                     /* (ROM_ERR_DIVERGED); 0 turns the test off                            */
    double wait_timeout_ms; /* 2000: bound of every wait of a sweep on another warp (the   */
                     /* x-edge ring of the 3D sweep, the test hook below); a wait that runs */
                     /* out ends the sweep and rom_solve returns ROM_ERR_TIMEOUT            */
    int test_stall_waits; /* 0; 1 makes every sweep warp (X-Y and 3D) wait on an mbarrier  */
                     /* that nothing completes: a test of the bounded waits -- with a short */
                     /* wait_timeout_ms the solve returns ROM_ERR_TIMEOUT, and the context  */
                     /* stays usable                                                       */
} rom_options;

/* Statistics of the last rom_solve. */
typedef struct rom_stats {
    int n_samples;
    int iterations_max;      /* most sweeps any sample took                              */
    int iterations_min;      /* fewest sweeps any sample took                            */
    int n_not_converged;     /* samples that stopped at max_iter above tol               */
    int64_t updates;         /* cell-ordinate updates: sum_s cells * M_s * sweeps_s      */
    double residual_max;     /* largest final relative change of phi over the samples    */
    double gpu_ms;           /* device time of the solve, CUDA events on the ctx stream  */
    int64_t kernel_launches; /* kernels the solve launched (graph nodes counted per run) */
    double sweep_ms;         /* summed duration of the sweep kernels (time_kernels = 1)   */
    int64_t sweep_launches;  /* sweep kernels timed                                       */
    double source_ms;        /* summed duration of the dense-operator contractions        */
    int64_t source_launches; /* contractions timed (dense operator only)                  */
    int tile_g;              /* ordinates per sweep work item used by this solve          */
    int rows_per_step;       /* X-Y sweep: grid rows a lane advances per wavefront step    */
                             /* (4, or 1 or 2 when the tile_g = -1 autotuner finds it      */
                             /* faster; 2 only in the moment modes); 0 for 3D grids        */
    double balance_max;      /* X-Y moment modes: largest relative particle-balance error  */
                             /* of each sample's last sweep (rom_get_balance); NaN when    */
                             /* not computed (3D, dense operator mode)                     */
    double phi_min;          /* smallest cell value of phi over the samples' last iterates */
                             /* (DD is not positive in 2D: it can be < 0)                  */
} rom_stats;

/* ------------------------------------------------------------- lifetime */

/* Create a context on CUDA device `cuda_device` with its own non-blocking
 * stream.  *out receives the handle (NULL on failure). */
int rom_create(rom_ctx **out, int cuda_device);

/* Free every device and host resource of the context (NULL is allowed). */
void rom_destroy(rom_ctx *ctx);

/* Message of the last failed call on ctx ("" if none).  Owned by ctx. */
const char *rom_last_error(const rom_ctx *ctx);

/* Issue all later device work on `cuda_stream` (a cudaStream_t of the
 * context's device; NULL restores the context's own stream).  The caller keeps
 * the stream alive while the context uses it. */
int rom_set_stream(rom_ctx *ctx, void *cuda_stream);

void rom_default_options(rom_options *opt);
int rom_set_options(rom_ctx *ctx, const rom_options *opt);

/* ---------------------------------------------------------------- problem */

/* Grid and coefficients (Sec. 1 eq. equ_1; Sec. 2 grid).  dim = 2: n[0] = I,
 * n[1] = J (>= 1 each, I <= 2048), lo = (x_L, y_B), hi = (x_R, y_T), n[2], lo[2],
 * hi[2] unused; dim = 3: also n[2] = K, lo[2] = z_B, hi[2] = z_T (each size
 * 1..4096).  hi > lo on every axis.  sigma_t, sigma_s, q: host FP64 [J][I] or
 * [K][J][I] with 0 <= sigma_S < sigma_T and q >= 0 (the paper's hypotheses,
 * Sec. 1).  Resets any inflow to vacuum.  3D grids support the isotropic kernel
 * (rom_solve returns ROM_ERR_UNSUPPORTED for any other). */
int rom_set_grid(rom_ctx *ctx, int dim, const int64_t n[3], const double lo[3], const double hi[3],
                 const double *sigma_t, const double *sigma_s, const double *q);

/* As rom_set_grid with FP32 device arrays [J][I] ([K][J][I]) on the context's device; they
 * are copied on the context stream and may be reused once the call returns.
 * The hypotheses on the coefficients are checked on the device. */
int rom_set_grid_device(rom_ctx *ctx, int dim, const int64_t n[3], const double lo[3],
                        const double hi[3], const float *sigma_t, const float *sigma_s,
                        const float *q);

/* Several X-Y grids in one context: the ROM samples are independent solves
 * (Sec. 3.1 runs one discrete-ordinate problem per sample; Sec. 4.1 averages
 * their scalar fluxes), so one batch may hold samples of different problems.
 * Grid p has n[2p] x n[2p+1] cells on [lo[2p], hi[2p]] x [lo[2p+1], hi[2p+1]]
 * and holds samples_per_grid[p] >= 1 consecutive samples: samples 0 ..
 * samples_per_grid[0]-1 are on grid 0, and so on.  sigma_t, sigma_s and q are
 * host FP64 arrays holding the grids' [J_p][I_p] blocks one after the other
 * (same hypotheses as rom_set_grid).  The ordinate sets set afterwards (or
 * before) must number sum_p samples_per_grid[p] samples; rom_solve checks
 * this (ROM_ERR_STATE).  The boundaries are vacuum (the inflow setters return
 * ROM_ERR_UNSUPPORTED) and the source iteration runs on angular moments:
 * the isotropic or (unflagged) linear kernel without dense_source; the dense
 * operator (Henyey-Greenstein, flagged kernels, dense_source = 1) returns
 * ROM_ERR_UNSUPPORTED at rom_solve.  rom_get_scalar_flux(sample >= 0) returns the sample's own
 * [J_p][I_p] grid; the average per grid comes from rom_get_grid_average
 * (sample = -1 and rom_get_partial_sum return an error).  rom_set_grid or
 * rom_set_grid_device returns the context to one grid.  Copies the arrays:
 * the caller keeps ownership. */
int rom_set_grids_xy(rom_ctx *ctx, int n_grids, const int64_t *n, const double *lo,
                     const double *hi, const double *sigma_t, const double *sigma_s,
                     const double *q, const int32_t *samples_per_grid);

/* Isotropic inflow psi_Gamma on one face (eq. equ_1_bc): host FP64 values per
 * face cell, >= 0; NULL = vacuum.  2D: J values for the x faces, I for the y
 * faces.  3D (faces 0..5): [K][J] for the x faces, [K][I] for the y faces,
 * [J][I] for the z faces. */
int rom_set_inflow_isotropic(rom_ctx *ctx, int face, const double *psi_face);

/* Inflow per ordinate on one face (eq. equ_random_bd): host FP64
 * [M_total][face cells], the ordinate index running over all samples in the
 * order of rom_set_ordinates / rom_set_ordinates_seed; only the values of
 * ordinates entering through the face are used.  Requires the ordinates. */
int rom_set_inflow_ordinates(rom_ctx *ctx, int face, const double *psi);

/* Explicit ordinate sets (Sec. 3.1 step 2, or any DOM set): n_samples sets with
 * m_per_sample[s] >= 1 ordinates each, concatenated.  dirs is host FP64
 * [sum M][3] = (c, s, zeta) with c^2 + s^2 + zeta^2 = 1 (to 1e-6), weights
 * [sum M] > 0.  Each ordinate sweeps from the x_L side if c >= 0 (else x_R) and
 * from the y_B side if s >= 0 (else y_T); on a 3D grid zeta is the direction
 * cosine mu_z, and the sweep starts from z_B if mu_z >= 0 (else z_T). */
int rom_set_ordinates(rom_ctx *ctx, int n_samples, const int32_t *m_per_sample,
                      const double *dirs, const double *weights);

/* Random ordinate sets generated on the device (Sec. 3.1, Sec. 4.2,
 * eq. 2Dordinates_symmetry, eq. wl).  Sample s (0-based, global index
 * first_sample + s) splits the first quadrant of (zeta, theta) into
 * n_zeta[s] x n_theta[s] equal cells, draws one point uniformly in each and
 * reflects it to the other quadrants; every weight is 1 / (4 n_zeta n_theta).
 * The uniform numbers are the SplitMix64 sequence of `seed` at counters
 * (global sample << 32) | (cell << 1) | {0: zeta, 1: theta}, top 53 bits.
 * Ordinates are stored per sample in the order quadrant 1 (cell l = (i-1) n_theta + j),
 * then the reflections l + m, l + 2m, l + 3m (m = n_zeta n_theta). */
int rom_set_ordinates_seed(rom_ctx *ctx, uint64_t seed, int n_samples, const int32_t *n_zeta,
                           const int32_t *n_theta);
int rom_set_ordinates_seed_offset(rom_ctx *ctx, uint64_t seed, int first_sample, int n_samples,
                                  const int32_t *n_zeta, const int32_t *n_theta);

/* Random ordinate sets on the whole sphere, for 3D grids (eq. equ_1 posed in
 * R^3; Sec. 3.1 construction): the 4 m points of rom_set_ordinates_seed_offset
 * (same counters, same order) followed by their mirror images (c, s, -zeta),
 * 8 m = 8 n_zeta n_theta ordinates per sample, one per octant cell of equal
 * area, every weight 1 / (8 m).  Directions are (c, s, mu_z). */
int rom_set_ordinates_seed_xyz(rom_ctx *ctx, uint64_t seed, int first_sample, int n_samples,
                               const int32_t *n_zeta, const int32_t *n_theta);

/* One deterministic DOM set as a single sample (Appendix A): see ROM_QUAD_*. */
int rom_set_quadrature(rom_ctx *ctx, int kind, int n1, int n2);

/* Fill a deterministic X-Y quadrature into host arrays (no context needed):
 * dirs [M][3] = (c, s, zeta), weights [M]; *m_out receives M.  Pass dirs =
 * weights = NULL to query M only.  Same sets as rom_set_quadrature. */
int rom_quadrature_xy(int kind, int n1, int n2, double *dirs, double *weights, int32_t *m_out);

/* Copy the context's ordinates (after the last set call) to host FP64
 * arrays: dirs [M_total][3], weights [M_total]. */
int rom_get_ordinates(rom_ctx *ctx, double *dirs, double *weights);

/* Scattering kernel P (Sec. 1; eq. anisotropic kernel; eq. wl): kind
 * ROM_KERNEL_*, asymmetry g in (-1, 1), flags ROM_KERNEL_FLAG_*.  Default ISO.
 * The isotropic and the (mirror-averaged, unnormalised) linear kernel use the
 * angular moments phi (and Jx, Jy); every other choice uses the dense operator
 * A[l][l'] = w_l' P(u_l', u_l) of each sample (eq. wl), which stores psi of every
 * ordinate: 8 bytes per cell and ordinate of device memory. */
int rom_set_kernel(rom_ctx *ctx, int kind, double g, int flags);

/* ------------------------------------------------------------------ solve */

/* Source iteration (Sec. 3.2, eq. psiexpansion) from psi = 0 for every sample,
 * then the FP64 sample average (Sec. 4.1).  Returns ROM_OK, or
 * ROM_ERR_NOT_CONVERGED / ROM_ERR_DIVERGED with the results still readable.
 * stats_out may be NULL.  The call returns when the device work is done. */
int rom_solve(rom_ctx *ctx, rom_stats *stats_out);

/* Scalar flux phi = sum_l w_l psi_l at the cell centres (Sec. 2) into host FP64
 * [J][I] ([K][J][I]): sample >= 0 one sample, sample = -1 the average over samples. */
int rom_get_scalar_flux(rom_ctx *ctx, int sample, double *out);

/* As rom_get_scalar_flux into a device FP64 buffer [J][I] or [K][J][I] (written on the
 * context stream; the call returns after enqueueing the copy). */
int rom_get_scalar_flux_device(rom_ctx *ctx, int sample, double *out);

/* Sweeps each sample took and its last relative change (host arrays [n_samples]). */
int rom_get_iterations(rom_ctx *ctx, int32_t *iters, double *residuals);

/* Particle balance of each sample's last sweep (host arrays [n_samples], any may be
 * NULL).  The cell equations of Sec. 2, multiplied by the cell area and summed over
 * the cells and, with the weights, over the ordinates, telescope to
 *   L + sum_cells sigma_T phi^k dA = sum_cells sum_l w_l S_l^{k-1} dA,
 * L = sum_l w_l (|c_l| dy sum_rows + |s_l| dx sum_cols)(psi_out - psi_in) the net
 * leakage through the boundary, phi^k the sweep's flux, S^{k-1} its source.
 * leakage receives L (FP64, accumulated from the FP32 boundary values by the
 * sweep), balance the relative error |L + absorbed - source| / (|L| + |absorbed| +
 * |source|) with the two cell sums formed in FP64, phi_min the smallest cell value of
 * phi^k.  X-Y moment modes (isotropic and linear kernel); leakage and balance are NaN
 * in 3D and in the dense operator mode.  Requires a solve. */
int rom_get_balance(rom_ctx *ctx, double *leakage, double *balance, double *phi_min);

/* Sum over this context's samples of phi (FP64 [J][I] or [K][J][I]) and their count, for
 * combining runs over disjoint sample ranges (rom_set_ordinates_seed_offset). */
int rom_get_partial_sum(rom_ctx *ctx, double *sum_out, int64_t *count_out);

/* FP64 average over the samples of grid `grid` (Sec. 4.1) into host [J_p][I_p];
 * with one grid, grid = 0 gives the same values as rom_get_scalar_flux(-1). */
int rom_get_grid_average(rom_ctx *ctx, int grid, double *out);

/* Library version string. */
const char *rom_version(void);

/* ------------------------------------------------ no-allocation variant */

/* Size in bytes of the fixed device scratch array of rom_sweep_xy_noalloc. */
#define ROM_NOALLOC_SCRATCH_BYTES (16u << 20)

/*
 * One transport sweep per sample that allocates no device memory.  The paper
 * has no counterpart: this is a deployment variant of the library's sweep.
 *
 * Who it is for: callers that must not call cudaMalloc -- plug-ins whose host
 * application owns all device memory through its own pool and forbids other
 * allocations, and latency-bound paths where an allocation (and the device
 * synchronisation it can imply) is not allowed.  The context API allocates its
 * buffers with cudaMalloc; this call
 * instead keeps its scratch (padded copies of the inputs and the per-sample
 * moment accumulators) in one array of ROM_NOALLOC_SCRATCH_BYTES that the library
 * places in device memory when it is loaded.  Every GPU that loads the
 * library holds that array until the process exits.
 *
 * What it computes: for each sample s, with vacuum inflow, the scalar flux
 *   phi_s = sum_l w_l psi_l,   psi_l = L_l^{-1} src_s,
 * where L_l is the diamond-difference (scheme = ROM_SCHEME_DD) or step
 * (ROM_SCHEME_STEP) discretisation of u_l . grad + sigma_T on the I x J grid
 * with cell sizes dx, dy, and src_s is the isotropic right-hand side of the
 * sample (for source iteration: sigma_S phi_s^{k-1} + q).  With src_s = q this
 * is the first sweep of rom_solve; with src_s = sigma_S phi_s + q the next one.
 *
 * Arguments: cuda_stream is the cudaStream_t to enqueue on (NULL = the legacy
 * default stream); sigma_t is a device FP32 array [J][I] on the current device;
 * src and phi are device FP32 arrays [n_samples][J][I]; m_per_sample (host,
 * [n_samples], each >= 1), dirs (host FP64 [sum M][3] = c, s, zeta, unit
 * vectors) and weights (host FP64 [sum M], > 0) give the ordinate sets, as in
 * rom_set_ordinates.  errbuf (may be NULL) receives a message on failure.
 * Limits: I <= 2048, n_samples <= 1024, sum M <= 8192, and the scratch the
 * problem needs (about 4 J ceil(I/8)*8 bytes times 1 + 2 n_samples, plus small
 * tables) must fit in
 * ROM_NOALLOC_SCRATCH_BYTES; larger problems return ROM_ERR_INVALID_ARG with
 * the needed size in errbuf.  No cudaMalloc, cudaFree or other allocating
 * routine is called.
 *
 * Behaviour: the first call on a device (with that device current) looks up
 * the device address of the scratch array once and caches it for the life of the
 * process; make that first call before any stream capture.  After
 * cudaDeviceReset on a device the cached address is stale: do not call this entry
 * point on that device again in the same process.  The call returns after enqueueing the work;
 * phi is ready when the stream reaches that point.  All calls on a device share
 * the one scratch array, which keeps the last call's contents; no part of it
 * needs to start at zero, because every call writes (or clears) each byte it
 * reads.  The work items of a sample add their moments to one accumulator, so
 * the last bits of phi depend on the order of those additions.  Calls
 * whose work overlaps on the GPU (other streams or host threads) race on the
 * array: serialise them.
 */
int rom_sweep_xy_noalloc(void *cuda_stream, int I, int J, double dx, double dy, int scheme,
                         const float *sigma_t, int n_samples, const int32_t *m_per_sample,
                         const double *dirs, const double *weights, const float *src,
                         float *phi, char *errbuf, size_t errbuf_len);

#ifdef __cplusplus
}
#endif

#endif /* ROM_GB300_H */
