/*
 * rom_oracle.c -- plain FP64 CPU oracle for the Random Ordinate Method (ROM)
 * of Li, Tang & Yang, "A random ordinate method for mitigating the ray effect
 * in radiative transport equation simulations" (arXiv 2407.12527), X-Y and
 * x-y-z geometry.
 *
 * TEST INFRASTRUCTURE ONLY.  The test-suite, the smoke check and the CPU
 * baseline leg of the benchmark are the only users of this file.  The CUDA
 * library never links, loads or calls it, and the two share no code: this
 * file was written from the paper alone, in double precision, with the loops
 * in the order the paper states the method and nothing blocked, fused or
 * reordered.  Parallelism (OpenMP) is only over independent ordinates inside
 * one source iteration; every sum that forms phi is taken in a fixed order.
 *
 * What is computed (paper references by section / equation):
 *   - ROM ordinates in X-Y geometry: a uniform partition of each quadrant of
 *     the (zeta, theta) rectangle, one uniform draw per cell, the other three
 *     quadrants by the reflections of eq. (2Dordinates_symmetry), weights
 *     |S_l|/|S| of eq. (wl)  [Sec. 3.1, Sec. 4.2].  The uniform draws come
 *     from the SplitMix64 sequence (Steele, Lea & Flood, OOPSLA 2014), the
 *     n-th draw of seed k being mix(k + (n+1)*0x9E3779B97F4A7C15).
 *   - The discrete ordinate system eq. (equ_random) with inflow eq.
 *     (equ_random_bd), discretised in space by diamond difference (Sec. 2,
 *     cell-centred unknowns) or, as an option, by the upwind step scheme.
 *   - Classical source iteration, the Neumann expansion of eq. (psiexpansion)
 *     [Sec. 3.2], started from psi = 0, stopped on the relative l2 change of
 *     the scalar flux.
 *   - Scattering source sigma_S * sum_l' w_l' P(u_l', u_l) psi_l' + q with
 *     P = 1 (isotropic), P = 1 + g cos(xi) (eq. anisotropic kernel) or the
 *     Henyey-Greenstein kernel, optionally row-normalised (Remark, Sec. 3.1).
 *   - 3D (x-y-z) geometry, in which eq. (equ_1) is posed (Sec. 1) though the
 *     paper tests only slab and X-Y: the X-Y set of the same draws mirrored in zeta (8 m ordinates on the whole
 *     sphere, weights 1/(8 m) each), DD or step on a uniform box grid with
 *     six inflow faces, isotropic scattering only.
 *
 * Readings of points the paper leaves open:
 *   - cell centres are x_L + (i + 1/2) dx, i = 0..I-1 (the grid definition in
 *     Sec. 2 indexes half-points inconsistently; eq. (l2norm2D) sums i = 0..I-1);
 *   - no negative-flux fix-up for diamond difference (none is mentioned);
 *   - X-Y ordinates live on the upper hemisphere (zeta in (0,1)); the kernel
 *     is evaluated, by default, as the mirror average
 *       1/2 [ G(cc'+ss'+zz') + G(cc'+ss'-zz') ],
 *     which is the exact full-sphere average for a solution even in zeta;
 *     `kernel_raw` = 1 uses G(cc'+ss'+zz') as printed;
 *   - SI starts from psi = 0 and stops when ||phi^k - phi^{k-1}||_2 <
 *     tol * ||phi^k||_2 (both norms zero counts as converged).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_EINVAL -1
#define ORACLE_ENOMEM -3
#define ORACLE_ENOTCONV -4

#define KERNEL_ISO 0
#define KERNEL_LINEAR 1
#define KERNEL_HG 2
#define SCHEME_DD 0
#define SCHEME_STEP 1

/* ------------------------------------------------------------------ RNG */

/* n-th output (n = 0, 1, ...) of the SplitMix64 generator seeded with seed. */
uint64_t oracle_splitmix64(uint64_t seed, uint64_t n)
{
    uint64_t z = seed + (n + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Uniform draw in [0, 1) from the top 53 bits of a SplitMix64 output. */
double oracle_uniform01(uint64_t seed, uint64_t n)
{
    return (double)(oracle_splitmix64(seed, n) >> 11) * (1.0 / 9007199254740992.0);
}

/* Counter of the draw for quadrant-1 cell l0 (0-based), component comp
 * (0 = zeta, 1 = theta), of ROM sample `sample`. */
static uint64_t draw_counter(int sample, int l0, int comp)
{
    return ((uint64_t)(uint32_t)sample << 32) | ((uint64_t)(uint32_t)l0 << 1) | (uint64_t)comp;
}

/*
 * ROM ordinates of one sample in X-Y geometry from given uniform numbers
 * (Sec. 4.2, eq. 2Dordinates_symmetry, eq. wl).  Quadrant 1 is split into
 * n_zeta x n_theta cells with nodes
 *   zeta_i  = (n_zeta - i + 1) / n_zeta,          i = 1..n_zeta+1,
 *   theta_j = (j - 1) * pi / (2 n_theta),         j = 1..n_theta+1,
 * and cell l = (i-1) n_theta + j is [zeta_{i+1}, zeta_i] x [theta_j, theta_{j+1}].
 * The point of cell l is zeta = zeta_{i+1} + u_zeta[l-1] (zeta_i - zeta_{i+1}),
 * theta = theta_j + u_theta[l-1] (theta_{j+1} - theta_j), i.e. uniform in the
 * cell when the u are U[0,1) draws.  The other quadrants follow by
 *   theta_{l+m} = pi - theta_l, theta_{l+2m} = theta_l - pi, theta_{l+3m} = 2 pi - theta_l,
 * all with the same zeta; (c, s) = sqrt(1 - zeta^2) (cos theta, sin theta).
 * Output order: quadrant 1 (l = 0..m-1), then l+m, l+2m, l+3m.  Every weight
 * is |S_l| / |S| = 1 / (4 m).
 */
int oracle_rom_ordinates_from_u(int n_zeta, int n_theta, const double *u_zeta,
                                const double *u_theta, double *c, double *s, double *zeta,
                                double *w)
{
    if (n_zeta < 1 || n_theta < 1) return ORACLE_EINVAL;
    const double pi = 3.14159265358979323846;
    const int m = n_zeta * n_theta;
    for (int i = 1; i <= n_zeta; ++i) {
        double z_hi = (double)(n_zeta - i + 1) / n_zeta; /* zeta_i     */
        double z_lo = (double)(n_zeta - i) / n_zeta;     /* zeta_{i+1} */
        for (int j = 1; j <= n_theta; ++j) {
            double t_lo = (double)(j - 1) * pi / (2.0 * n_theta); /* theta_j     */
            double t_hi = (double)j * pi / (2.0 * n_theta);       /* theta_{j+1} */
            int l0 = (i - 1) * n_theta + (j - 1);
            double zz = z_lo + u_zeta[l0] * (z_hi - z_lo);
            double th = t_lo + u_theta[l0] * (t_hi - t_lo);
            double rho = sqrt(1.0 - zz * zz);
            double th_q[4] = {th, pi - th, th - pi, 2.0 * pi - th};
            for (int q = 0; q < 4; ++q) {
                int l = l0 + q * m;
                c[l] = rho * cos(th_q[q]);
                s[l] = rho * sin(th_q[q]);
                zeta[l] = zz;
                w[l] = 1.0 / (4.0 * m);
            }
        }
    }
    return ORACLE_OK;
}

/* The uniform numbers of ROM sample `sample`: u_zeta[l0] and u_theta[l0] are
 * the SplitMix64 draws with counters (sample << 32) | (l0 << 1) | {0, 1}. */
int oracle_rom_draws(uint64_t seed, int sample, int m, double *u_zeta, double *u_theta)
{
    if (m < 1 || sample < 0) return ORACLE_EINVAL;
    for (int l0 = 0; l0 < m; ++l0) {
        u_zeta[l0] = oracle_uniform01(seed, draw_counter(sample, l0, 0));
        u_theta[l0] = oracle_uniform01(seed, draw_counter(sample, l0, 1));
    }
    return ORACLE_OK;
}

/* ROM ordinates of sample `sample` of the seeded sequence (draws + mapping above). */
int oracle_rom_ordinates_xy(uint64_t seed, int sample, int n_zeta, int n_theta,
                            double *c, double *s, double *zeta, double *w)
{
    if (n_zeta < 1 || n_theta < 1 || sample < 0) return ORACLE_EINVAL;
    const int m = n_zeta * n_theta;
    double *uz = malloc((size_t)m * sizeof(double)), *ut = malloc((size_t)m * sizeof(double));
    if (!uz || !ut) {
        free(uz);
        free(ut);
        return ORACLE_ENOMEM;
    }
    oracle_rom_draws(seed, sample, m, uz, ut);
    int rc = oracle_rom_ordinates_from_u(n_zeta, n_theta, uz, ut, c, s, zeta, w);
    free(uz);
    free(ut);
    return rc;
}

/* ------------------------------------------------------------- kernels */

/* Phase function G(cos xi): isotropic 1, linear 1 + g mu (eq. anisotropic
 * kernel), Henyey-Greenstein (1 - g^2) / (1 + g^2 - 2 g mu)^{3/2}. */
static double phase_G(int kernel, double g, double mu)
{
    if (kernel == KERNEL_ISO) return 1.0;
    if (kernel == KERNEL_LINEAR) return 1.0 + g * mu;
    return (1.0 - g * g) / pow(1.0 + g * g - 2.0 * g * mu, 1.5);
}

/* P(u_a, u_b) for two X-Y ordinates (see the header for the mirror reading). */
static double kernel_P(int kernel, double g, int raw,
                       double ca, double sa, double za, double cb, double sb, double zb)
{
    double inplane = ca * cb + sa * sb;
    if (raw) return phase_G(kernel, g, inplane + za * zb);
    return 0.5 * (phase_G(kernel, g, inplane + za * zb) + phase_G(kernel, g, inplane - za * zb));
}

/*
 * Dense discrete scattering operator of one ordinate set (eq. wl):
 *   A[l][l'] = w_l' * P(u_l', u_l),
 * divided by its row sum sum_l' w_l' P(u_l', u_l) when normalize_rows != 0
 * (the normalisation the Remark of Sec. 3.1 mentions).  A is M x M, row-major.
 */
int oracle_kernel_matrix(int M, const double *c, const double *s, const double *zeta,
                         const double *w, int kernel, double g, int raw, int normalize_rows,
                         double *A)
{
    if (M < 1) return ORACLE_EINVAL;
    for (int l = 0; l < M; ++l) {
        double rowsum = 0.0;
        for (int lp = 0; lp < M; ++lp) {
            double P = kernel_P(kernel, g, raw, c[lp], s[lp], zeta[lp], c[l], s[l], zeta[l]);
            A[(size_t)l * M + lp] = w[lp] * P;
            rowsum += w[lp] * P;
        }
        if (normalize_rows)
            for (int lp = 0; lp < M; ++lp) A[(size_t)l * M + lp] /= rowsum;
    }
    return ORACLE_OK;
}

/* -------------------------------------------------------------- sweeps */

typedef struct {
    int I, J;
    double dx, dy;
} grid_t;

/*
 * Transport sweep of one ordinate (c, s) over the I x J cells in upwind order.
 * src[k] is the right-hand side sigma_S * (scatter) + q of this ordinate at cell k.
 * Inflow: face values, layout [x = x_L: J][x = x_R: J][y = y_B: I][y = y_T: I];
 * NULL means vacuum.
 *
 * Diamond difference (Sec. 2): per cell, with mu = |c|, eta = |s|,
 *   mu (psi_xout - psi_xin)/dx + eta (psi_yout - psi_yin)/dy + sigma_T psi_c = src,
 *   psi_c = (psi_xin + psi_xout)/2 = (psi_yin + psi_yout)/2,
 * solved as psi_c = (src + 2mu/dx psi_xin + 2eta/dy psi_yin) / (sigma_T + 2mu/dx + 2eta/dy),
 * psi_xout = 2 psi_c - psi_xin, psi_yout = 2 psi_c - psi_yin.
 * Step scheme: psi_xout = psi_yout = psi_c, which gives the same formula with
 * mu/dx, eta/dy in place of 2mu/dx, 2eta/dy.
 *
 * psi_c is written to psi[k].  The ordinate's net outflow through the
 * boundary, mu dy sum_rows (exit - entry) + eta dx sum_cols (exit - entry),
 * is returned.
 */
static double sweep_ordinate(const grid_t *G, const double *sigma_t, const double *src,
                             double c, double s, int scheme, const double *inflow,
                             double *psi, double *psi_y /* scratch [I] */)
{
    const int I = G->I, J = G->J;
    const double mu = fabs(c), eta = fabs(s);
    const double f = (scheme == SCHEME_DD) ? 2.0 : 1.0;
    const double ax = f * mu / G->dx, by = f * eta / G->dy;
    const int xpos = (c >= 0.0), ypos = (s >= 0.0);
    double leak = 0.0;

    /* incoming y-edge values of the first row swept */
    for (int i = 0; i < I; ++i) {
        double in = 0.0;
        if (inflow) in = ypos ? inflow[2 * J + i] : inflow[2 * J + I + i];
        psi_y[i] = in;
        leak -= eta * G->dx * in;
    }
    for (int jj = 0; jj < J; ++jj) {
        const int j = ypos ? jj : J - 1 - jj;
        double psi_x = 0.0;
        if (inflow) psi_x = xpos ? inflow[j] : inflow[J + j];
        leak -= mu * G->dy * psi_x;
        for (int ii = 0; ii < I; ++ii) {
            const int i = xpos ? ii : I - 1 - ii;
            const size_t k = (size_t)j * I + i;
            double pc = (src[k] + ax * psi_x + by * psi_y[i]) / (sigma_t[k] + ax + by);
            psi[k] = pc;
            if (scheme == SCHEME_DD) {
                psi_x = 2.0 * pc - psi_x;
                psi_y[i] = 2.0 * pc - psi_y[i];
            } else {
                psi_x = pc;
                psi_y[i] = pc;
            }
        }
        leak += mu * G->dy * psi_x; /* exit through the far x face */
    }
    for (int i = 0; i < I; ++i) leak += eta * G->dx * psi_y[i];
    return leak;
}

/* --------------------------------------------------------------- solve */

static double l2diff_rel(const double *a, const double *b, size_t n)
{
    double d2 = 0.0, n2 = 0.0;
    for (size_t k = 0; k < n; ++k) {
        d2 += (a[k] - b[k]) * (a[k] - b[k]);
        n2 += a[k] * a[k];
    }
    if (n2 == 0.0) return d2 == 0.0 ? 0.0 : INFINITY;
    return sqrt(d2 / n2);
}

/*
 * Source iteration for every ordinate set (ROM sample) of a problem on the
 * I x J grid of [xl,xr] x [yb,yt].
 *
 *   sigma_t, sigma_s, q : [J*I] cell values, x fastest;
 *   n_samples, m_per_sample : ordinate sets, concatenated in c, s, zeta, w;
 *   inflow, inflow_ord_stride : NULL = vacuum; otherwise face values (layout of
 *       sweep_ordinate), the values of global ordinate n starting at
 *       inflow + n * inflow_ord_stride (stride 0 = isotropic inflow);
 *   kernel, g, kernel_raw, normalize_rows : scattering kernel;
 *   scheme : 0 diamond difference, 1 step;
 *   tol, max_iter : stop when the relative l2 change of phi is below tol;
 *   fixed_iters > 0 : run exactly that many sweeps instead;
 *   n_threads : OpenMP threads (<= 0: the runtime default).
 * Outputs, per sample: phi_out [n_samples][J*I], iters_out, resid_out (last
 * relative change), leak_out (net boundary outflow of phi of the last sweep,
 * sum_l w_l times the per-ordinate value of sweep_ordinate; may be NULL).
 * Returns ORACLE_ENOTCONV if some sample did not reach tol within max_iter
 * (its outputs are still written).
 */
int oracle_solve_xy(int I, int J, double xl, double xr, double yb, double yt,
                    const double *sigma_t, const double *sigma_s, const double *q,
                    int n_samples, const int *m_per_sample,
                    const double *c, const double *s, const double *zeta, const double *w,
                    const double *inflow, long inflow_ord_stride,
                    int kernel, double g, int kernel_raw, int normalize_rows,
                    int scheme, double tol, int max_iter, int fixed_iters, int n_threads,
                    double *phi_out, int *iters_out, double *resid_out, double *leak_out)
{
    if (I < 1 || J < 1 || n_samples < 0 || !(xr > xl) || !(yt > yb)) return ORACLE_EINVAL;
    if (kernel < KERNEL_ISO || kernel > KERNEL_HG || (scheme != SCHEME_DD && scheme != SCHEME_STEP))
        return ORACLE_EINVAL;
    if (fixed_iters <= 0 && max_iter < 1) return ORACLE_EINVAL;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
    const grid_t G = {I, J, (xr - xl) / I, (yt - yb) / J};
    const size_t nc = (size_t)I * J;
    int status = ORACLE_OK;
    long offset = 0; /* first global ordinate of the current sample */

    for (int smp = 0; smp < n_samples; ++smp) {
        const int M = m_per_sample[smp];
        const double *cs = c + offset, *ss = s + offset, *zs = zeta + offset, *ws = w + offset;
        double *phi = phi_out + (size_t)smp * nc;
        const int dense = (kernel != KERNEL_ISO);
        int nthr = 1;
#ifdef _OPENMP
        nthr = omp_get_max_threads();
#endif
        double *phi_new = calloc(nc, sizeof(double));
        double *part = calloc(nc * (size_t)nthr, sizeof(double)); /* per-thread phi partials */
        double *psi_tmp = malloc(nc * (size_t)nthr * sizeof(double));
        double *psi_y = malloc((size_t)I * nthr * sizeof(double));
        double *src = malloc(nc * (size_t)(dense ? M : 1) * sizeof(double));
        double *psi_all = dense ? calloc(nc * (size_t)M, sizeof(double)) : NULL;
        double *A = dense ? malloc((size_t)M * M * sizeof(double)) : NULL;
        double *leak_l = malloc((size_t)(M > 0 ? M : 1) * sizeof(double));
        if (!phi_new || !part || !psi_tmp || !psi_y || !src || !leak_l || (dense && (!psi_all || !A))) {
            free(phi_new); free(part); free(psi_tmp); free(psi_y); free(src); free(psi_all); free(A); free(leak_l);
            return ORACLE_ENOMEM;
        }
        if (dense) oracle_kernel_matrix(M, cs, ss, zs, ws, kernel, g, kernel_raw, normalize_rows, A);
        memset(phi, 0, nc * sizeof(double));

        int it = 0;
        double resid = INFINITY, leak = 0.0;
        const int limit = fixed_iters > 0 ? fixed_iters : max_iter;
        while (it < limit) {
            /* scattering source from the previous iterate (psi^0 = 0) */
            if (!dense) {
                for (size_t k = 0; k < nc; ++k) src[k] = sigma_s[k] * phi[k] + q[k];
            } else {
#pragma omp parallel for schedule(static)
                for (int l = 0; l < M; ++l) {
                    double *sl = src + (size_t)l * nc;
                    for (size_t k = 0; k < nc; ++k) {
                        double acc = 0.0;
                        for (int lp = 0; lp < M; ++lp)
                            acc += A[(size_t)l * M + lp] * psi_all[(size_t)lp * nc + k];
                        sl[k] = sigma_s[k] * acc + q[k];
                    }
                }
            }
            memset(part, 0, nc * (size_t)nthr * sizeof(double));
            /* one transport sweep per ordinate */
#pragma omp parallel for schedule(static)
            for (int l = 0; l < M; ++l) {
                int t = 0;
#ifdef _OPENMP
                t = omp_get_thread_num();
#endif
                const double *in = inflow ? inflow + (offset + l) * inflow_ord_stride : NULL;
                double *psi = dense ? psi_all + (size_t)l * nc : psi_tmp + (size_t)t * nc;
                const double *sl = dense ? src + (size_t)l * nc : src;
                leak_l[l] = sweep_ordinate(&G, sigma_t, sl, cs[l], ss[l], scheme, in, psi,
                                           psi_y + (size_t)t * I);
                double *pt = part + (size_t)t * nc;
                for (size_t k = 0; k < nc; ++k) pt[k] += ws[l] * psi[k];
            }
            /* phi = sum_l w_l psi_l */
            for (size_t k = 0; k < nc; ++k) {
                double acc = 0.0;
                for (int t = 0; t < nthr; ++t) acc += part[(size_t)t * nc + k];
                phi_new[k] = acc;
            }
            leak = 0.0;
            for (int l = 0; l < M; ++l) leak += ws[l] * leak_l[l];
            resid = l2diff_rel(phi_new, phi, nc);
            memcpy(phi, phi_new, nc * sizeof(double));
            ++it;
            if (fixed_iters <= 0 && resid < tol) break;
        }
        if (fixed_iters <= 0 && !(resid < tol)) status = ORACLE_ENOTCONV;
        if (iters_out) iters_out[smp] = it;
        if (resid_out) resid_out[smp] = resid;
        if (leak_out) leak_out[smp] = leak;
        free(phi_new); free(part); free(psi_tmp); free(psi_y); free(src); free(psi_all); free(A); free(leak_l);
        offset += M;
    }
    return status;
}

/*
 * Source iteration with the linear kernel P = 1 + g cos(xi) (eq. anisotropic
 * kernel) in its mirror-averaged form 1 + g (cc' + ss'), carried by three
 * angular moments instead of the dense operator: with phi = sum w psi,
 * Jx = sum w c psi, Jy = sum w s psi of the previous sweep,
 *   S_l = sigma_S (phi + g (c_l Jx + s_l Jy)) + q,
 * which is sum_l' w_l' P(u_l', u_l) psi_l' written out.  Vacuum inflow;
 * arguments as oracle_solve_xy.  Used for references with very many ordinates,
 * where the M x M operator does not fit.
 */
int oracle_solve_xy_linear_moments(int I, int J, double xl, double xr, double yb, double yt,
                                   const double *sigma_t, const double *sigma_s, const double *q,
                                   int n_samples, const int *m_per_sample, const double *c,
                                   const double *s, const double *w, double g, int scheme,
                                   double tol, int max_iter, int fixed_iters, int n_threads,
                                   double *phi_out, int *iters_out, double *resid_out)
{
    if (I < 1 || J < 1 || n_samples < 0 || !(xr > xl) || !(yt > yb)) return ORACLE_EINVAL;
    if (scheme != SCHEME_DD && scheme != SCHEME_STEP) return ORACLE_EINVAL;
    if (fixed_iters <= 0 && max_iter < 1) return ORACLE_EINVAL;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
    const grid_t G = {I, J, (xr - xl) / I, (yt - yb) / J};
    const size_t nc = (size_t)I * J;
    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    int status = ORACLE_OK;
    long offset = 0;
    for (int smp = 0; smp < n_samples; ++smp) {
        const int M = m_per_sample[smp];
        const double *cs = c + offset, *ss = s + offset, *ws = w + offset;
        double *phi = phi_out + (size_t)smp * nc;
        double *jx = calloc(nc, sizeof(double)), *jy = calloc(nc, sizeof(double));
        double *mom_new = calloc(3 * nc, sizeof(double));
        double *part = calloc(3 * nc * (size_t)nthr, sizeof(double));
        double *psi_tmp = malloc(nc * (size_t)nthr * sizeof(double));
        double *src_tmp = malloc(nc * (size_t)nthr * sizeof(double));
        double *psi_y = malloc((size_t)I * nthr * sizeof(double));
        if (!jx || !jy || !mom_new || !part || !psi_tmp || !src_tmp || !psi_y) {
            free(jx); free(jy); free(mom_new); free(part); free(psi_tmp); free(src_tmp); free(psi_y);
            return ORACLE_ENOMEM;
        }
        memset(phi, 0, nc * sizeof(double));
        int it = 0;
        double resid = INFINITY;
        const int limit = fixed_iters > 0 ? fixed_iters : max_iter;
        while (it < limit) {
            memset(part, 0, 3 * nc * (size_t)nthr * sizeof(double));
#pragma omp parallel for schedule(static)
            for (int l = 0; l < M; ++l) {
                int t = 0;
#ifdef _OPENMP
                t = omp_get_thread_num();
#endif
                double *psi = psi_tmp + (size_t)t * nc, *src = src_tmp + (size_t)t * nc;
                for (size_t k = 0; k < nc; ++k)
                    src[k] = sigma_s[k] * (phi[k] + g * (cs[l] * jx[k] + ss[l] * jy[k])) + q[k];
                sweep_ordinate(&G, sigma_t, src, cs[l], ss[l], scheme, NULL, psi,
                               psi_y + (size_t)t * I);
                double *pt = part + 3 * nc * (size_t)t;
                for (size_t k = 0; k < nc; ++k) {
                    pt[k] += ws[l] * psi[k];
                    pt[nc + k] += ws[l] * cs[l] * psi[k];
                    pt[2 * nc + k] += ws[l] * ss[l] * psi[k];
                }
            }
            for (size_t k = 0; k < 3 * nc; ++k) {
                double acc = 0.0;
                for (int t = 0; t < nthr; ++t) acc += part[3 * nc * (size_t)t + k];
                mom_new[k] = acc;
            }
            resid = l2diff_rel(mom_new, phi, nc);
            memcpy(phi, mom_new, nc * sizeof(double));
            memcpy(jx, mom_new + nc, nc * sizeof(double));
            memcpy(jy, mom_new + 2 * nc, nc * sizeof(double));
            ++it;
            if (fixed_iters <= 0 && resid < tol) break;
        }
        if (fixed_iters <= 0 && !(resid < tol)) status = ORACLE_ENOTCONV;
        if (iters_out) iters_out[smp] = it;
        if (resid_out) resid_out[smp] = resid;
        free(jx); free(jy); free(mom_new); free(part); free(psi_tmp); free(src_tmp); free(psi_y);
        offset += M;
    }
    return status;
}

/* Number of OpenMP threads a parallel region would use (1 without OpenMP). */
int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ============================================================ 3D (x-y-z) */

/*
 * ROM ordinates in 3D (the RTE of Sec. 1 posed for z in R^3): the draws and
 * the first-quadrant partition of the X-Y construction (Sec. 4.2) give the
 * upper-hemisphere points (c, s, zeta), zeta in (0, 1); their mirror images
 * (c, s, -zeta) complete the sphere, 8 octants of m points each, every weight
 * |S_l| / |S| = 1 / (8 m).  Output: the 4 m upper points in the X-Y order, then
 * their mirrors in the same order.  dirs are written as (c, s, mu_z).
 */
int oracle_rom_ordinates_xyz(uint64_t seed, int sample, int n_zeta, int n_theta, double *c,
                             double *s, double *mu_z, double *w)
{
    const int m = n_zeta * n_theta;
    int rc = oracle_rom_ordinates_xy(seed, sample, n_zeta, n_theta, c, s, mu_z, w);
    if (rc != ORACLE_OK) return rc;
    for (int l = 0; l < 4 * m; ++l) {
        c[4 * m + l] = c[l];
        s[4 * m + l] = s[l];
        mu_z[4 * m + l] = -mu_z[l];
        w[l] = 1.0 / (8.0 * m);
        w[4 * m + l] = 1.0 / (8.0 * m);
    }
    return ORACLE_OK;
}

typedef struct {
    int I, J, K;
    double dx, dy, dz;
} grid3_t;

/*
 * Diamond-difference (or step) sweep of one 3D ordinate (c, s, mu_z) in upwind
 * order: per cell, with a = f|c|/dx, b = f|s|/dy, e = f|mu_z|/dz (f = 2 for DD,
 * 1 for step), psi_c = (src + a psi_xin + b psi_yin + e psi_zin) / (sigma_T + a + b + e),
 * DD outflows 2 psi_c - inflow, step outflows psi_c.  Inflow: isotropic face
 * values, layout [x_L: K*J][x_R: K*J][y_B: K*I][y_T: K*I][z_B: J*I][z_T: J*I]
 * ([k][j], [k][i], [j][i]); NULL = vacuum.  Returns the net boundary outflow.
 */
static double sweep_ordinate3(const grid3_t *G, const double *sigma_t, const double *src,
                              double c, double s, double mz, int scheme, const double *inflow,
                              double *psi, double *psi_y /* [I] */, double *psi_z /* [J*I] */)
{
    const int I = G->I, J = G->J, K = G->K;
    const double f = (scheme == SCHEME_DD) ? 2.0 : 1.0;
    const double mu = fabs(c), eta = fabs(s), xi = fabs(mz);
    const double ax = f * mu / G->dx, by = f * eta / G->dy, ez = f * xi / G->dz;
    const int xpos = (c >= 0.0), ypos = (s >= 0.0), zpos = (mz >= 0.0);
    const size_t fx = (size_t)K * J, fy = (size_t)K * I;
    const size_t o_xl = 0, o_xr = fx, o_yb = 2 * fx, o_yt = 2 * fx + fy, o_zb = 2 * fx + 2 * fy,
                 o_zt = 2 * fx + 2 * fy + (size_t)J * I;
    double leak = 0.0;
    const double aX = mu * G->dy * G->dz, aY = eta * G->dx * G->dz, aZ = xi * G->dx * G->dy;

    for (int j = 0; j < J; ++j)
        for (int i = 0; i < I; ++i) {
            double in = inflow ? inflow[(zpos ? o_zb : o_zt) + (size_t)j * I + i] : 0.0;
            psi_z[(size_t)j * I + i] = in;
            leak -= aZ * in;
        }
    for (int kk = 0; kk < K; ++kk) {
        const int k = zpos ? kk : K - 1 - kk;
        for (int i = 0; i < I; ++i) {
            double in = inflow ? inflow[(ypos ? o_yb : o_yt) + (size_t)k * I + i] : 0.0;
            psi_y[i] = in;
            leak -= aY * in;
        }
        for (int jj = 0; jj < J; ++jj) {
            const int j = ypos ? jj : J - 1 - jj;
            double psi_x = inflow ? inflow[(xpos ? o_xl : o_xr) + (size_t)k * J + j] : 0.0;
            leak -= aX * psi_x;
            for (int ii = 0; ii < I; ++ii) {
                const int i = xpos ? ii : I - 1 - ii;
                const size_t cell = ((size_t)k * J + j) * I + i;
                double *pz = &psi_z[(size_t)j * I + i];
                double pc = (src[cell] + ax * psi_x + by * psi_y[i] + ez * *pz) /
                            (sigma_t[cell] + ax + by + ez);
                psi[cell] = pc;
                if (scheme == SCHEME_DD) {
                    psi_x = 2.0 * pc - psi_x;
                    psi_y[i] = 2.0 * pc - psi_y[i];
                    *pz = 2.0 * pc - *pz;
                } else {
                    psi_x = pc;
                    psi_y[i] = pc;
                    *pz = pc;
                }
            }
            leak += aX * psi_x;
        }
        for (int i = 0; i < I; ++i) leak += aY * psi_y[i];
    }
    for (size_t n = 0; n < (size_t)J * I; ++n) leak += aZ * psi_z[n];
    return leak;
}

/*
 * Source iteration in 3D with isotropic scattering (S = sigma_S phi + q), per
 * ordinate set, on the I x J x K grid of [xl,xr] x [yb,yt] x [zb,zt]; arrays
 * [K][J][I] (x fastest).  Arguments as oracle_solve_xy; dirs (c, s, mu_z).
 */
int oracle_solve_xyz(int I, int J, int K, const double *bounds /* xl xr yb yt zb zt */,
                     const double *sigma_t, const double *sigma_s, const double *q, int n_samples,
                     const int *m_per_sample, const double *c, const double *s, const double *mz,
                     const double *w, const double *inflow, int scheme, double tol, int max_iter,
                     int fixed_iters, int n_threads, double *phi_out, int *iters_out,
                     double *resid_out, double *leak_out)
{
    if (I < 1 || J < 1 || K < 1 || n_samples < 0) return ORACLE_EINVAL;
    if (!(bounds[1] > bounds[0]) || !(bounds[3] > bounds[2]) || !(bounds[5] > bounds[4]))
        return ORACLE_EINVAL;
    if (scheme != SCHEME_DD && scheme != SCHEME_STEP) return ORACLE_EINVAL;
    if (fixed_iters <= 0 && max_iter < 1) return ORACLE_EINVAL;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
    const grid3_t G = {I, J, K, (bounds[1] - bounds[0]) / I, (bounds[3] - bounds[2]) / J,
                       (bounds[5] - bounds[4]) / K};
    const size_t nc = (size_t)I * J * K;
    int status = ORACLE_OK;
    long offset = 0;
    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    for (int smp = 0; smp < n_samples; ++smp) {
        const int M = m_per_sample[smp];
        double *phi = phi_out + (size_t)smp * nc;
        double *phi_new = calloc(nc, sizeof(double));
        double *part = calloc(nc * (size_t)nthr, sizeof(double));
        double *psi_tmp = malloc(nc * (size_t)nthr * sizeof(double));
        double *psi_y = malloc((size_t)I * nthr * sizeof(double));
        double *psi_z = malloc((size_t)I * J * nthr * sizeof(double));
        double *src = malloc(nc * sizeof(double));
        double *leak_l = malloc((size_t)(M > 0 ? M : 1) * sizeof(double));
        if (!phi_new || !part || !psi_tmp || !psi_y || !psi_z || !src || !leak_l) {
            free(phi_new); free(part); free(psi_tmp); free(psi_y); free(psi_z); free(src); free(leak_l);
            return ORACLE_ENOMEM;
        }
        memset(phi, 0, nc * sizeof(double));
        int it = 0;
        double resid = INFINITY, leak = 0.0;
        const int limit = fixed_iters > 0 ? fixed_iters : max_iter;
        while (it < limit) {
            for (size_t n = 0; n < nc; ++n) src[n] = sigma_s[n] * phi[n] + q[n];
            memset(part, 0, nc * (size_t)nthr * sizeof(double));
#pragma omp parallel for schedule(static)
            for (int l = 0; l < M; ++l) {
                int t = 0;
#ifdef _OPENMP
                t = omp_get_thread_num();
#endif
                double *psi = psi_tmp + (size_t)t * nc;
                leak_l[l] = sweep_ordinate3(&G, sigma_t, src, c[offset + l], s[offset + l],
                                            mz[offset + l], scheme, inflow, psi,
                                            psi_y + (size_t)t * I, psi_z + (size_t)t * I * J);
                double *pt = part + (size_t)t * nc;
                for (size_t n = 0; n < nc; ++n) pt[n] += w[offset + l] * psi[n];
            }
            for (size_t n = 0; n < nc; ++n) {
                double acc = 0.0;
                for (int t = 0; t < nthr; ++t) acc += part[(size_t)t * nc + n];
                phi_new[n] = acc;
            }
            leak = 0.0;
            for (int l = 0; l < M; ++l) leak += w[offset + l] * leak_l[l];
            resid = l2diff_rel(phi_new, phi, nc);
            memcpy(phi, phi_new, nc * sizeof(double));
            ++it;
            if (fixed_iters <= 0 && resid < tol) break;
        }
        if (fixed_iters <= 0 && !(resid < tol)) status = ORACLE_ENOTCONV;
        if (iters_out) iters_out[smp] = it;
        if (resid_out) resid_out[smp] = resid;
        if (leak_out) leak_out[smp] = leak;
        free(phi_new); free(part); free(psi_tmp); free(psi_y); free(psi_z); free(src); free(leak_l);
        offset += M;
    }
    return status;
}
