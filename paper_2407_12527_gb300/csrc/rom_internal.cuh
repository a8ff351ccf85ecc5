// rom_internal.cuh -- device data layout and kernel launch interfaces shared by
// the translation units of the GB300 ROM library (not part of the public ABI).
//
// HBM layout (all FP32 unless noted; rows padded to a pitch of NXP = ceil(I/8)*8
// floats so every lane's 8-cell segment is one aligned 32-byte sector):
//   sigma_t, sigma_s, q      [J][NXP]
//   phi    (per sample)      [S][MOM][J][NXP]   current iterate, MOM scalar moments
//   src    (per sample)      [S][MOM][J][NXP]   source moments for the next sweep
//   part   (per sample)      [S][MOM][J][NXP]   moments the sweep's work items add
//   ordinates                c, s, w [M_total] (FP32) and c, s, zeta, w (FP64)
//   residual and balance sums [S][kNP] FP64, smallest phi [S] (ordered-int key)
// MOM = 1 for isotropic scattering (phi), 3 for the linear kernel (phi, Jx, Jy).
// 3D grids keep the arrays their sweep touches in diagonal storage (Skew3 below).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace romk {

constexpr int kCols = 8;       // cells per lane along x
constexpr int kMaxG = 4;       // ordinates per sweep work item
constexpr int kMaxWarps = 8;   // I <= 32 * 8 * 8 = 2048
constexpr int kMaxCtaItems3 = 256;  // 3D: work items per CTA list

// Per-sample sums the combine blocks add (FP64 atomics) and the finalize reads
// and clears: squared change and squared norm of phi (residual), sum of
// sigma_T phi, sums of the three source moments of the previous iterate
// (balance); beside them the smallest phi of the sweep as an ordered-int key.
constexpr int kNP = 6;
__device__ __forceinline__ int float_order_key(float f)
{
    const int b = __float_as_int(f);
    return b >= 0 ? b : b ^ 0x7FFFFFFF;
}
__device__ __forceinline__ float float_from_order_key(int k)
{
    return __int_as_float(k >= 0 ? k : k ^ 0x7FFFFFFF);
}

// One sweep work item: up to kMaxG ordinates of one quadrant of one sample.
// quad bit 0 set: c < 0 (sweep from x_R), bit 1 set: s < 0 (sweep from y_T),
// bit 2 set (3D): mu_z < 0 (sweep from z_T).
struct SweepItem {
    int sample;
    int quad;
    int n;
    int ord[kMaxG];
    int grid;  // batches of several X-Y grids: the sample's grid (else 0)
};

// One grid of a batch of several X-Y grids (rom_set_grids_xy): its sizes and
// cell widths, and where its [J][NXP] cell arrays start in the concatenated
// coefficient arrays.
struct GridDesc {
    int I, J, NXP;
    float inv_dx, inv_dy, dx, dy;
    long long off;    // first cell of the grid's coefficient arrays
    long long cells;  // J * NXP
};

struct SweepArgs {
    int I, J, NXP;
    float inv_dx, inv_dy;
    float sigma_t_homog;        // used when the grid has one sigma_T
    const float *sigma_t;       // [J][NXP]
    const float *src;           // [S][MOM][J][NXP]; dense mode: [M_total][J][NXP] per ordinate
    float *part;                // [S][MOM][J][NXP] accumulators (dense mode: phi only)
    float *psi;                 // dense mode: psi of every ordinate [M_total][J][NXP]
    uint32_t *psi_split;        // dense mode, tensor cores: psi as BF16 hi / lo parts,
                                // [M_total][J * NXP / 8][hi 8 | lo 8] (psi unused when set)
    const SweepItem *items;
    const float *oc, *os, *ow;  // ordinate c, s, w
    const float *inflow;        // nullptr = vacuum; else face values [x_L:J][x_R:J][y_B:I][y_T:I]
    long long inflow_stride;    // per ordinate (0 = same values for every ordinate)
    const int *active;          // [S] samples still iterating
    long long cells;            // J * NXP
    // several grids (nullptr: the one grid above): each item takes its grid's
    // sizes and coefficient block, and its sample's state starts at soff[sample]
    const GridDesc *grids;      // [grids]
    const long long *soff;      // [S] first float of the sample's [MOM][cells] block
    // moment modes: the net leakage of each sample's sweep (nullptr: not kept)
    double *leak;               // [S]
    float dx, dy;               // leakage weights |c| dy, |s| dx
    int *err;                   // bit 0: the test hook's wait ran out
    unsigned long long wait_ns; // bound of that wait
    int stall;                  // test hook: every warp waits on a barrier nothing completes
};
// The X-Y sweep adds the moments of every work item to part[sample] (vector
// reductions; the combine reads and clears them).

struct CombineArgs {
    int S, MOM;
    int chunks;                 // at most this many blocks per sample
    int I, NXP;                 // columns and row pitch (min phi skips padding columns)
    long long cells;
    float g;                    // linear-kernel asymmetry (MOM = 3)
    float *acc;                 // [S][MOM][cells] moments added by the sweep, cleared here
    float *phi;
    float *src;
    const float *sigma_s, *q;
    // balance sums (moment modes): sigma_T per cell, nullptr = sigma_t_homog
    int balance;
    const float *sigma_t;
    float sigma_t_homog;
    // several grids (nullptr: one): the sample's grid and state offset
    const GridDesc *grids;
    const int *sgrid;           // [S]
    const long long *soff;      // [S]
    const int *active;
    double *sums;               // [S][kNP] added with FP64 atomics
    int *minkey;                // [S] smallest phi (float_order_key), atomic min
};

// Diagonal storage of 3D cell arrays read or written by the sweep (source, sigma_T,
// flux accumulators).  Cell (i, j, k) with row block jb = j / 4, row hh = j % 4,
// strip = i / 8, c = i % 8 sits at
//   ((((diag * L + strip) * 4 + hh) * NBg + jb) * 8 + c,
//   family 0 ("plus", octants whose y and z directions agree): diag = k + jb,
//   family 1 ("minus"):                                        diag = k - jb + NBg - 1,
// with L = NXP / 8 strips, NBg = ceil(J / 4) blocks and K + NBg - 1 diagonals.  The
// lanes of a sweep warp sit on one diagonal at consecutive blocks, so each of
// their row accesses is one contiguous kilobyte.
struct Skew3 {
    int J, K, L, NBg;
    long long DS;     // floats per diagonal: L * 4 * NBg * 8
    long long cells;  // floats per array: (K + NBg - 1) * DS
};
__host__ __device__ inline Skew3 make_skew3(int J, int K, int NXP)
{
    Skew3 g;
    g.J = J;
    g.K = K;
    g.L = NXP / 8;
    g.NBg = (J + 3) / 4;
    g.DS = (long long)g.L * 4 * g.NBg * 8;
    g.cells = (long long)(K + g.NBg - 1) * g.DS;
    return g;
}
// offset of the 8-cell sector (k, j, strip) in family f
__host__ __device__ inline long long skew3_index(const Skew3 &g, int f, int k, int j, int strip)
{
    const int jb = j >> 2, hh = j & 3;
    const long long diag = f == 0 ? (long long)k + jb : (long long)k - jb + g.NBg - 1;
    return diag * g.DS + (((long long)strip * 4 + hh) * g.NBg + jb) * 8;
}

// 3D sweep (K9): G = 1 or 2 ordinates of one sample and octant per work item,
// CTAs over lists of items of one octant, x-y tiles swept by successive launches.
struct Sweep3Args {
    int I, J, K, NXP;
    float inv_dx, inv_dy, inv_dz;
    Skew3 sk;                   // diagonal storage of the three arrays below
    const float *sigma_t;       // [family][sk.cells]
    const float *src;           // [family][S][sk.cells] isotropic source sigma_S phi + q
    float *phi;                 // [family][S][sk.cells] flux accumulated by the sweep
    int S;
    const SweepItem *items;     // quad = octant bits, ord[0] the ordinate
    const int *cta_begin;       // [n_ctas + 1] ranges of cta_list
    const int *cta_list;        // item indices, one octant per CTA
    const float *oc, *os, *oz, *ow;
    const float *inflow;        // nullptr = vacuum; else [x_L: K*J][x_R: K*J][y_B: K*I][y_T: K*I]
                                //                        [z_B: J*I][z_T: J*I]
    long long inflow_stride;    // per ordinate (0 = same values for every ordinate)
    const int *active;          // [S]
    long long cells;            // K * J * NXP
    int tile_x, tile_y;         // tile of this launch, counted from the inflow corner
    int n_tx, n_ty;             // tiles along x and y
    float *xface;               // [items][G][K][J] x-edges handed to the next x tile
    float *yface;               // [items][G][K][NXP] y-edges handed to the next y tile
    int *err;                   // bit 0/1: an mbarrier wait timed out (bit 2: the test hook's)
    unsigned long long wait_ns; // bound of every wait
    int stall;                  // test hook: every warp waits on a barrier nothing completes
};

struct FinalizeArgs {
    int S, chunks;
    int fixed_iters, max_iter;
    double tol;
    int diverge_window;         // stop a sample after this many sweeps of growing change (0: off)
    double *sums;               // [S][kNP] read and cleared
    int *minkey;                // [S] read and reset
    int *active, *iters, *flags;
    double *resid;
    double *dprev;              // [S] ||phi^k - phi^{k-1}||_2 of the previous sweep
    int *grow;                  // [S] consecutive sweeps whose change grew
    // particle balance of the sweep (balance != 0): the net leakage the sweep
    // added per sample (read and cleared), the cell area and per-sample sums
    // sum_l w_l, sum_l w_l c_l, sum_l w_l s_l ([S][3])
    int balance;
    double *leak;
    double dA;
    const double *sdA;          // [S] cell area per sample (several grids), else nullptr
    const double *ordsum;
    double *bal_out, *leak_out, *phimin_out;  // [S] values of each sample's last sweep
    int *n_active;
    int use_cond;
    cudaGraphConditionalHandle cond;
};

// per-sample FP64 sums sum_l w_l, sum_l w_l c_l, sum_l w_l s_l -> out [S][3]
cudaError_t launch_ordsum(const double *c, const double *s, const double *w,
                          const long long *ord_off, const int *M, int S, double *out,
                          cudaStream_t st);

// Ordinate generation (one thread per quadrant-1 cell of a sample).
struct OrdGenArgs {
    unsigned long long seed;
    int n_samples;
    const int *nz, *nt;         // per sample partition
    const int *first_cell;      // [S+1] prefix sum of m = nz * nt
    const long long *ord_off;   // [S] first ordinate of the sample
    int first_sample;           // global index of local sample 0
    int total_cells;
    int octants;                // 1: 3D sets, the 4 quadrants mirrored in zeta (8 m points)
    double *c64, *s64, *z64, *w64;
    float *c32, *s32, *z32, *w32;
};

// Dense scattering operator A[l][l'] = w_l' P(u_l', u_l) per sample (K3).
struct PmatArgs {
    int S;
    const int *M;               // [S] ordinates per sample
    const long long *ord_off;   // [S] first ordinate of the sample
    const long long *a_off;     // [S] first element of the sample's A (row-major M x M)
    const double *c, *s, *z, *w;
    int kind;                   // 0 isotropic, 1 linear, 2 Henyey-Greenstein
    double g;
    int raw, normalize;
    float *A;
};

// Dense source S_l = sigma_S sum_l' A[l][l'] psi_l' + q for every sample (K4).
struct DenseArgs {
    int S;
    const int *M;
    const long long *ord_off, *a_off;
    const float *A;
    const float *psi;           // [M_total][cells]
    float *src;                 // [M_total][cells]
    const float *sigma_s, *q;   // [cells]
    long long cells;
    const int *active;
};

// Dense source on the tensor cores (split BF16, tcgen05): TMA maps of A_hi,
// A_lo [S][128][128] and of the split psi as one BF16 matrix [M_total][2 cells]
// (rows of [8 hi | 8 lo] per 8 cells).
struct DenseTcMaps {
    CUtensorMap a_hi, a_lo, b;
};
struct DenseTcArgs {
    int S;
    const int *M;               // [S], each <= 128
    const long long *ord_off;   // [S]
    long long cells;            // a multiple of 8
    const float *sigma_s, *q;
    float *src;                 // [M_total][cells]
    const int *active;
    int *err;                   // bits 2..7: a wait timed out
};
int dense_tc_max_m();
int dense_tc_max_samples();
cudaError_t make_dense_tc_maps(DenseTcMaps *maps, const void *a_hi, const void *a_lo, int S,
                               const void *psi_split, long long m_total, long long cells);
cudaError_t launch_dense_tc(const DenseTcMaps &maps, const DenseTcArgs &a, int n_ctas,
                            cudaStream_t st);
cudaError_t launch_pmat_split(const float *A, const int *M, const long long *a_off, int S,
                              void *hi, void *lo, cudaStream_t st);

cudaError_t launch_pmat(const PmatArgs &a, int max_m, cudaStream_t st);
cudaError_t launch_dense_source(const DenseArgs &a, int max_m, cudaStream_t st);
cudaError_t launch_dense_init(const float *q, long long cells, long long m_total, float *src,
                              cudaStream_t st);

// 256-bit (one full 32-byte sector) vector accesses of sm_100+, 32-byte aligned.
__device__ __forceinline__ void ldg8(const float *p, float (&v)[8])
{
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]),
          "=f"(v[7])
        : "l"(p));
}
// Same load kept in program order with the other volatile accesses (used to
// issue prefetches where they are written, ahead of the stores of a step).
__device__ __forceinline__ void ldg8_early(const float *p, float (&v)[8])
{
    asm volatile("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]),
                   "=f"(v[6]), "=f"(v[7])
                 : "l"(p));
}
__device__ __forceinline__ void ld8_volatile(const float *p, float (&v)[8])
{
    asm volatile("ld.global.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]),
                   "=f"(v[6]), "=f"(v[7])
                 : "l"(p));
}
__device__ __forceinline__ void stg8(float *p, const float (&v)[8])
{
    asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(v[0]),
                 "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]));
}

// psi of 8 cells as BF16 parts in one 32-byte sector, [8 hi | 8 lo] (the byte
// layout of the FP32 array): hi = v rounded to the nearest BF16 on its bit
// pattern (add half a BF16 unit, clear the low 16 bits; ties away from zero;
// two packed by one byte permute), lo = bf16_rn(v - hi) (the difference is exact
// in FP32; two converted by one packed conversion).  hi + lo carries 16
// significant bits of v, and lo has either sign, so the lo * lo term the
// product drops has no bias.
__device__ __forceinline__ void st8_split(uint32_t *psi2, long long off, const float (&v)[kCols])
{
    uint32_t h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const uint32_t b0 = (__float_as_uint(v[2 * e]) + 0x8000u) & 0xFFFF0000u;
        const uint32_t b1 = (__float_as_uint(v[2 * e + 1]) + 0x8000u) & 0xFFFF0000u;
        h[e] = __byte_perm(b0, b1, 0x7632);
        const float r0 = v[2 * e] - __uint_as_float(b0);
        const float r1 = v[2 * e + 1] - __uint_as_float(b1);
        const __nv_bfloat162 lo2 = __floats2bfloat162_rn(r0, r1);
        l[e] = *reinterpret_cast<const uint32_t *>(&lo2);
    }
    asm volatile("st.global.v8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(psi2 + off), "r"(h[0]),
                 "r"(h[1]), "r"(h[2]), "r"(h[3]), "r"(l[0]), "r"(l[1]), "r"(l[2]), "r"(l[3])
                 : "memory");
}

// mom: 1 isotropic, 3 linear-kernel moments, 0 dense kernel (per-ordinate
// source in, psi out).
// rows: rows a lane advances per wavefront step, 4 (every mode) or 2 (mom 1, 3).
cudaError_t launch_sweep2d(const SweepArgs &a, int n_items, int nwarps, int G, int scheme,
                           bool homog, int mom, int rows, cudaStream_t st);
cudaError_t launch_sweep2d_rows2(const SweepArgs &a, int n_items, int nwarps, int G, int scheme,
                                 bool homog, int mom, cudaStream_t st);
// batches of several grids (a.grids, a.soff set): mom 1 or 3, rows 2 or 4
cudaError_t launch_sweep2d_batch(const SweepArgs &a, int n_items, int nwarps, int G, int scheme,
                                 int mom, int rows, cudaStream_t st);
// one grid row per wavefront step (sweep2d_row.cuh): mom 1, 3 or 0 (dense operator)
cudaError_t launch_sweep2d_row(const SweepArgs &a, int n_items, int nwarps, int G, int scheme,
                               bool homog, int mom, cudaStream_t st);
cudaError_t launch_sweep2d_row_batch(const SweepArgs &a, int n_items, int nwarps, int G,
                                     int scheme, int mom, cudaStream_t st);
cudaError_t launch_sweep3d(const Sweep3Args &a, int n_ctas, int nwarps, int G, int scheme,
                           cudaStream_t st);
int sweep3d_ctas_per_sm(int nwarps, int G);
int sweep3d_tile_cols();  // x extent of a 3D tile (8-column strips x warps per CTA)
cudaError_t launch_combine(const CombineArgs &a, cudaStream_t st);
// 3D: phi = the sum of the two accumulators, residual sums, and the next
// source sigma_S phi + q in both diagonal families; phi, sigma_S, q in family 0.
struct Combine3Args {
    int S, chunks;
    int I;                      // columns (min phi skips padding columns)
    Skew3 sk;
    float *acc;                 // [2][S][sk.cells], cleared after reading
    float *src;                 // [2][S][sk.cells]
    float *phi;                 // [S][sk.cells] (family 0)
    const float *sigma_s, *q;   // [sk.cells] (family 0)
    const int *active;
    double *sums;               // [S][kNP]
    int *minkey;                // [S]
};
cudaError_t launch_combine3(const Combine3Args &a, cudaStream_t st);
cudaError_t launch_average3(const float *phi, int S, const Skew3 &sk, int I, double *avg,
                            double *sum, cudaStream_t st);
cudaError_t launch_extract3(const float *phi, int sample, const Skew3 &sk, int I, double *out,
                            cudaStream_t st);
// copies of a [K][J][NXP] array into diagonal families 0 .. n_fam-1, n_copies
// times per family (dst[f][copy][sk.cells]); padding entries are left as they are
cudaError_t launch_skew3_scatter(const float *in, const Skew3 &sk, int NXP, int n_fam,
                                 int n_copies, float *dst, cudaStream_t st);
cudaError_t launch_finalize(const FinalizeArgs &a, cudaStream_t st);
cudaError_t launch_init_state(int S, int MOM, long long cells, const float *q, float *phi,
                              float *src, int *active, int *iters, int *flags, double *resid,
                              cudaStream_t st);
// per-sample divergence and balance state of a new solve: dprev = +inf, grow = 0,
// leak = 0, bal / leak_out / phimin = NaN, sums = 0, minkey = INT_MAX
cudaError_t launch_init_checks(int S, double *dprev, int *grow, double *leak, double *bal,
                               double *leak_out, double *phimin, double *sums, int *minkey,
                               cudaStream_t st);
cudaError_t launch_average(const float *phi, int S, int MOM, int I, int J, int NXP, double *avg,
                           double *sum, cudaStream_t st);
// several grids: phi = 0 and the first source q for every sample on its own grid
cudaError_t launch_init_grids(int S, int MOM, const GridDesc *grids, const int *sgrid,
                              const long long *soff, int max_cells, const float *q, float *phi,
                              float *src, cudaStream_t st);
cudaError_t launch_extract(const float *phi, int sample, int MOM, int I, int J, int NXP,
                           double *out, cudaStream_t st);
cudaError_t launch_pad_grid(const float *st_in, const float *ss_in, const float *q_in, int I,
                            int J, int NXP, float *st_out, float *ss_out, float *q_out,
                            unsigned int *stats /*[3]: min sigma_t bits, max bits, bad cells*/,
                            cudaStream_t st);
cudaError_t launch_ordgen(const OrdGenArgs &a, cudaStream_t st);

}  // namespace romk
