// sweep2d_impl.cuh -- the X-Y transport sweep kernels (K1), compiled once per
// number of rows a lane advances per wavefront step: the including translation
// unit defines SWEEP2D_ROWS (and SWEEP2D_WITH_DENSE = 1 to include the dense-mode
// variants), so that the variants build in parallel.  The algorithm and its GPU
// mapping are described in sweep2d.cu.
#pragma once
#ifndef SWEEP2D_ROWS
#error "define SWEEP2D_ROWS before including sweep2d_impl.cuh"
#endif
#ifndef SWEEP2D_WITH_DENSE
#define SWEEP2D_WITH_DENSE 0
#endif
#ifndef SWEEP2D_BATCH
#define SWEEP2D_BATCH 0  // 1: the kernels of batches of several grids (SweepArgs::grids)
#endif
#include "rom_internal.cuh"

namespace romk {
namespace {

constexpr int kH = SWEEP2D_ROWS;  // rows per lane per wavefront step
constexpr int kPrefetch = 1;  // steps between the load of a block's rows and their use

// ---- packs: one ordinate (float), or two ordinates (float2, FP32x2 ops)
template <int G>
struct Pack {
    using T = float2;
    static constexpr int N = G / 2;
};
template <>
struct Pack<1> {
    using T = float;
    static constexpr int N = 1;
};

__device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float2 fma_(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float mul_(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float2 mul_(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float add_(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float2 add_(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float neg_(float a) { return -a; }
__device__ __forceinline__ float2 neg_(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float sub_(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float2 sub_(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }

// mbarrier helpers of the test hook (a bounded wait on a barrier nothing completes)
__device__ __forceinline__ unsigned smem_u32a(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ bool never_wait(unsigned long long *b, unsigned long long budget_ns)
{
    unsigned long long t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (;;) {
        unsigned ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_u32a(b)), "r"(0u)
            : "memory");
        if (__all_sync(0xffffffffu, ok != 0)) return true;
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (__any_sync(0xffffffffu, t - t0 > budget_ns)) return false;
    }
}
// 1 / (sigma_T + a + b) of a cell with varying sigma_T: the hardware reciprocal
// (rcp.approx, within 1 ulp; the argument is >= sigma_T > 0, never subnormal)
__device__ __forceinline__ float rcp_(float a)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ float2 rcp_(float2 a) { return make_float2(rcp_(a.x), rcp_(a.y)); }
__device__ __forceinline__ float hsum(float a) { return a; }
__device__ __forceinline__ float hsum(float2 a) { return a.x + a.y; }
__device__ __forceinline__ void setc(float &a, int, float v) { a = v; }
__device__ __forceinline__ void setc(float2 &a, int i, float v)
{
    if (i) a.y = v;
    else a.x = v;
}
template <class T>
__device__ __forceinline__ T splat(float s);
template <>
__device__ __forceinline__ float splat<float>(float s) { return s; }
template <>
__device__ __forceinline__ float2 splat<float2>(float s) { return make_float2(s, s); }

// Compensated (Kahan) FP32 sum of the boundary terms of the leakage, one term per
// step (a pack of ordinates at a time): a few ulps of the total instead of n ulps;
// widened to FP64 once per lane.
template <class T>
struct Kahan {
    T s = splat<T>(0.f), c = splat<T>(0.f);
    __device__ __forceinline__ void add(T v)
    {
        const T y = sub_(v, c);
        const T t = add_(s, y);
        c = sub_(sub_(t, s), y);
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)hsum(s) - (double)hsum(c); }
};

template <bool DOWN>
__device__ __forceinline__ float shfl1(float v)
{
    return DOWN ? __shfl_down_sync(0xffffffffu, v, 1) : __shfl_up_sync(0xffffffffu, v, 1);
}
template <bool DOWN>
__device__ __forceinline__ float2 shfl1(float2 v)
{
    return make_float2(shfl1<DOWN>(v.x), shfl1<DOWN>(v.y));
}

__device__ __forceinline__ void ld8(const float *__restrict__ p, float (&v)[kCols]) { ldg8_early(p, v); }
__device__ __forceinline__ void st8(float *__restrict__ p, const float (&v)[kCols]) { stg8(p, v); }
// add 8 moments to the sample's accumulator: two 4-wide vector reductions
__device__ __forceinline__ void red8(float *p, const float (&v)[kCols])
{
    asm volatile("red.global.add.v4.f32 [%0], {%1,%2,%3,%4};" ::"l"(p), "f"(v[0]), "f"(v[1]),
                 "f"(v[2]), "f"(v[3])
                 : "memory");
    asm volatile("red.global.add.v4.f32 [%0], {%1,%2,%3,%4};" ::"l"(p + 4), "f"(v[4]), "f"(v[5]),
                 "f"(v[6]), "f"(v[7])
                 : "memory");
}
// the moments of a row, added to the sample's accumulator (every work item of the
// sample adds into the same array; the reductions run in L2, and the combine reads
// and clears the array)
template <int MOM>
__device__ __forceinline__ void put8(float *p, const float (&v)[kCols])
{
    red8(p, v);
}
// Per-ordinate constants of a work item, grouped in packs.
template <int G>
struct OrdPacks {
    using T = typename Pack<G>::T;
    static constexpr int N = Pack<G>::N;
    T a[N], b[N], ab[N], w[N], rd[N], c[N], s[N], wc[N], ws[N];
    // uniform sigma_T: the cell update folded into one FMA per upwind chain
    //   DD:   x_out  = al x + 2rd (S + b py),   al = 2a rd - 1
    //         py_out = a2 x + 2rd S + be py,    a2 = 2a rd, be = 2b rd - 1
    //         psi_c  = (x + x_out) / 2
    //   step: psi_c  = ar x + rd (S + b py) = x_out = py_out,  ar = a rd, br = b rd
    T al[N], a2[N], b2[N], be[N], r2[N], wh[N], ar[N], br[N];
    T lx[N], ly[N];  // leakage weights w |c| dy and w |s| dx
    int ord[G];
};

// Source modes (template parameter MOM): 1 isotropic (one source moment in,
// phi out), 3 linear kernel (three source moments in, phi, Jx, Jy out), 0 dense
// kernel (one source per ordinate in, psi of every ordinate and phi out).
__host__ __device__ constexpr int n_src(int mom, int g) { return mom == 0 ? g : mom; }
__host__ __device__ constexpr int n_out(int mom) { return mom == 0 ? 1 : mom; }

// Arrays read per cell: NS sources, plus sigma_T when it varies.
template <int NS, bool HOMOG>
struct RowBuf {
    static constexpr int NA = NS + (HOMOG ? 0 : 1);
    float v[NA][kH][kCols];
};

// Offset of row h of block blk for the lane's columns: base + h * rs.
struct RowAddr {
    long long base, rs;
    __device__ __forceinline__ RowAddr(const SweepArgs &A, int blk, bool yneg, int col0)
    {
        const int jl0 = blk * kH;
        base = (long long)(yneg ? (A.J - 1 - jl0) : jl0) * A.NXP + col0;
        rs = yneg ? -(long long)A.NXP : (long long)A.NXP;
    }
};

// Issue the loads of the rows of block `blk` (rows past J are skipped).
template <int NS, bool HOMOG>
__device__ __forceinline__ void load_block(const SweepArgs &A, int blk, bool yneg, int col0,
                                           const float *const (&srcp)[NS], RowBuf<NS, HOMOG> &b)
{
    const RowAddr ra(A, blk, yneg, col0);
#pragma unroll
    for (int h = 0; h < kH; ++h) {
        if (blk * kH + h < A.J) {
            const long long row = ra.base + h * ra.rs;
#pragma unroll
            for (int m = 0; m < NS; ++m) ld8(srcp[m] + row, b.v[m][h]);
            if (!HOMOG) ld8(A.sigma_t + row, b.v[NS][h]);
        }
    }
}

// One H x 8 block of cells for all G ordinates of the item, from the rows in b.
// Cell value psi_c of the ordinates of pack p at column r, kept for the row store.
__device__ __forceinline__ void psi_put(float (&row)[1][kCols], int, int r, float v) { row[0][r] = v; }
template <int R>
__device__ __forceinline__ void psi_put(float (&row)[R][kCols], int p, int r, float2 v)
{
    if constexpr (R >= 2) {
        row[(2 * p) % R][r] = v.x;
        row[(2 * p + 1) % R][r] = v.y;
    }
}

// The block's moments are left in out[][][] (LATE: the caller stores them
// after the shuffle), or stored row by row at part_i (three moments: the
// registers for holding them are not there).
template <int G, int MOM, int SCHEME, bool HOMOG, bool XNEG, bool CHECK, bool LATE>
__device__ __forceinline__ void sweep_block(const SweepArgs &A, int blk, bool yneg, int col0,
                                            const OrdPacks<G> &o,
                                            typename Pack<G>::T (&py)[kCols][Pack<G>::N],
                                            const typename Pack<G>::T (&xin)[kH][Pack<G>::N],
                                            typename Pack<G>::T (&xo)[kH][Pack<G>::N],
                                            const RowBuf<n_src(MOM, G), HOMOG> &b,
                                            float (&out)[LATE ? n_out(MOM) : 1][kH][kCols],
                                            float *__restrict__ part_i)
{
    constexpr int NS = n_src(MOM, G);
    using T = typename Pack<G>::T;
    constexpr int N = Pack<G>::N;
    const T two = splat<T>(2.f);
#pragma unroll
    for (int h = 0; h < kH; ++h) {
        if (CHECK && blk * kH + h >= A.J) {
#pragma unroll
            for (int p = 0; p < N; ++p) xo[h][p] = splat<T>(0.f);
            continue;
        }
        T x[N];
#pragma unroll
        for (int p = 0; p < N; ++p) x[p] = xin[h][p];
        T acc0[kCols], acc1[kCols], acc2[kCols];
#pragma unroll
        for (int r = 0; r < kCols; ++r) acc0[r] = acc1[r] = acc2[r] = splat<T>(0.f);
        float psi_row[MOM == 0 ? G : 1][kCols];  // dense mode: psi of the row, per ordinate
#pragma unroll
        for (int rr = 0; rr < kCols; ++rr) {
            const int r = XNEG ? (kCols - 1 - rr) : rr;
            const bool ok = !CHECK || (col0 + r < A.I);
            const T s0 = splat<T>(b.v[0][h][r]);
#pragma unroll
            for (int p = 0; p < N; ++p) {
                T S = s0;
                if (MOM == 3)
                    S = fma_(o.c[p], splat<T>(b.v[1][h][r]), fma_(o.s[p], splat<T>(b.v[2][h][r]), S));
                if (MOM == 0) {  // per-ordinate sources of the pack
                    if constexpr (G == 1) setc(S, 0, b.v[0][h][r]);
                    else {
                        setc(S, 0, b.v[(2 * p) % NS][h][r]);
                        setc(S, 1, b.v[(2 * p + 1) % NS][h][r]);
                    }
                }
                if (HOMOG && SCHEME == 0) {
                    // x_out = al x + b2 py + 2 rd S; sum = x + x_out = 2 psi_c;
                    // py_out = sum - py (the DD closure), w psi_c = (w / 2) sum
                    const T xn = fma_(o.al[p], x[p], fma_(o.b2[p], py[r][p], mul_(S, o.r2[p])));
                    const T sm = add_(x[p], xn);
                    if (MOM == 0) psi_put(psi_row, p, r, mul_(sm, splat<T>(0.5f)));
                    if (ok) {
                        acc0[r] = fma_(o.wh[p], sm, acc0[r]);
                        if (MOM == 3) {
                            acc1[r] = fma_(mul_(o.wc[p], splat<T>(0.5f)), sm, acc1[r]);
                            acc2[r] = fma_(mul_(o.ws[p], splat<T>(0.5f)), sm, acc2[r]);
                        }
                        py[r][p] = sub_(sm, py[r][p]);
                        x[p] = xn;
                    }
                } else if (HOMOG) {
                    const T pc = fma_(o.ar[p], x[p], fma_(o.br[p], py[r][p], mul_(S, o.rd[p])));
                    if (MOM == 0) psi_put(psi_row, p, r, pc);
                    if (ok) {
                        x[p] = pc;
                        py[r][p] = pc;
                        acc0[r] = fma_(o.w[p], pc, acc0[r]);
                        if (MOM == 3) {
                            acc1[r] = fma_(o.wc[p], pc, acc1[r]);
                            acc2[r] = fma_(o.ws[p], pc, acc2[r]);
                        }
                    }
                } else {
                    const T num = fma_(o.a[p], x[p], fma_(o.b[p], py[r][p], S));
                    const T rden =
                        rcp_(add_(splat<T>(b.v[RowBuf<NS, HOMOG>::NA - 1][h][r]), o.ab[p]));
                    const T pc = mul_(num, rden);
                    if (MOM == 0) psi_put(psi_row, p, r, pc);
                    if (ok) {
                        if (SCHEME == 0) {
                            x[p] = fma_(two, pc, neg_(x[p]));
                            py[r][p] = fma_(two, pc, neg_(py[r][p]));
                        } else {
                            x[p] = pc;
                            py[r][p] = pc;
                        }
                        acc0[r] = fma_(o.w[p], pc, acc0[r]);
                        if (MOM == 3) {
                            acc1[r] = fma_(o.wc[p], pc, acc1[r]);
                            acc2[r] = fma_(o.ws[p], pc, acc2[r]);
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int p = 0; p < N; ++p) xo[h][p] = x[p];
        if constexpr (LATE) {
#pragma unroll
            for (int r = 0; r < kCols; ++r) out[0][h][r] = hsum(acc0[r]);
            if constexpr (MOM == 3) {
#pragma unroll
                for (int r = 0; r < kCols; ++r) {
                    out[MOM - 2][h][r] = hsum(acc1[r]);
                    out[MOM - 1][h][r] = hsum(acc2[r]);
                }
            }
        } else {
            const RowAddr ra(A, blk, yneg, col0);
            float v[kCols];
#pragma unroll
            for (int r = 0; r < kCols; ++r) v[r] = hsum(acc0[r]);
            put8<MOM>(part_i + ra.base + h * ra.rs, v);
            if constexpr (MOM == 0) {
#pragma unroll
                for (int k = 0; k < G; ++k) {
                    const long long off = (long long)o.ord[k] * A.cells + ra.base + h * ra.rs;
                    if (A.psi_split) st8_split(A.psi_split, off, psi_row[k]);
                    else st8(A.psi + off, psi_row[k]);
                }
            }
            if (MOM == 3) {
#pragma unroll
                for (int r = 0; r < kCols; ++r) v[r] = hsum(acc1[r]);
                put8<MOM>(part_i + A.cells + ra.base + h * ra.rs, v);
#pragma unroll
                for (int r = 0; r < kCols; ++r) v[r] = hsum(acc2[r]);
                put8<MOM>(part_i + 2 * A.cells + ra.base + h * ra.rs, v);
            }
        }
    }
}

template <int G, int MOM, int SCHEME, bool HOMOG, bool XNEG>
__device__ __forceinline__ void sweep_item(const SweepArgs &A, const SweepItem &it,
                                           const OrdPacks<G> &o)
{
    using T = typename Pack<G>::T;
    constexpr int N = Pack<G>::N;
    __shared__ T xbuf[2][kMaxWarps][kH][N];
    const int g = threadIdx.x;
    const int nwarps = blockDim.x >> 5;
    const int L = (A.I + kCols - 1) / kCols;  // lanes that own cells
    const bool lane_on = g < L;
    const int d = XNEG ? (L - 1 - g) : g;     // lanes between this one and the inflow face
    const int col0 = g * kCols;
    const bool yneg = (it.quad >> 1) & 1;
    const int nblk = (A.J + kH - 1) / kH;
    const int T_steps = nblk + L - 1;
    const bool full_cols = col0 + kCols <= A.I;

    // incoming y-edge values of the lane's columns (face y_B, or y_T when s < 0)
    T py[kCols][N];
#pragma unroll
    for (int r = 0; r < kCols; ++r)
#pragma unroll
        for (int k = 0; k < G; ++k) {
            float v = 0.f;
            if (A.inflow && lane_on && col0 + r < A.I && k < it.n)
                v = A.inflow[(long long)o.ord[k] * A.inflow_stride + 2 * A.J + (yneg ? A.I : 0) +
                             col0 + r];
            setc(py[r][G == 1 ? 0 : k >> 1], G == 1 ? 0 : k & 1, v);
        }
    // net leakage of the item (moment modes): sum_l w_l (|c_l| dy sum_rows +
    // |s_l| dx sum_cols) (psi_out - psi_in), Kahan-summed per lane.  The x-face
    // terms use weights that are zero except on the boundary lanes, so every
    // lane runs the same instructions (no branch in the step).
    Kahan<T> leak;
    T lx_out[N], lx_in[N];
#pragma unroll
    for (int p = 0; p < N; ++p) {
        lx_out[p] = d == L - 1 ? o.lx[p] : splat<T>(0.f);
        lx_in[p] = d == 0 ? o.lx[p] : splat<T>(0.f);
    }
    if (A.leak && lane_on) {
        T lin = splat<T>(0.f);
#pragma unroll
        for (int r = 0; r < kCols; ++r)
#pragma unroll
            for (int p = 0; p < N; ++p) lin = fma_(o.ly[p], py[r][p], lin);
        leak.add(neg_(lin));
    }

    T xin[kH][N];
#pragma unroll
    for (int h = 0; h < kH; ++h)
#pragma unroll
        for (int p = 0; p < N; ++p) xin[h][p] = splat<T>(0.f);

    constexpr int NS = n_src(MOM, G);
    // source arrays of the item: the sample's moments, or (dense) one per ordinate
    const float *srcp[NS];
#pragma unroll
    for (int m = 0; m < NS; ++m)
        srcp[m] = MOM == 0 ? A.src + (long long)o.ord[m] * A.cells
                           : A.src + (A.soff ? A.soff[it.sample]
                                             : (long long)it.sample * MOM * A.cells) +
                                 m * A.cells;
    // moments: the sample's accumulator [n_out][cells]
    float *part_i = A.part + (A.soff ? A.soff[it.sample]
                                     : (long long)it.sample * n_out(MOM) * A.cells);

    // The rows of the lane's block for step t + PD are loaded at the start of
    // step t into a ring of PD + 1 register buffers indexed by t (the same index
    // for every lane: lane d at step t works on block t - d).  With more than
    // two arrays per cell (linear kernel) the registers are not there; the rows
    // are then loaded at the start of their step.
    constexpr int NA = RowBuf<NS, HOMOG>::NA;
    constexpr bool PF = NA <= 2;
    constexpr int PD = NA == 1 ? kPrefetch : (NA == 2 ? 1 : 0);
    // moments are stored row by row inside the block (holding a whole block's
    // moments until the end of the step measured slower on GB300)
    constexpr bool STORE_LATE = false;
    RowBuf<NS, HOMOG> buf[PD + 1];
    auto step = [&](int t, RowBuf<NS, HOMOG> &cur, RowBuf<NS, HOMOG> &nxt) {
        const int blk = t - d;
        const bool active = lane_on && blk >= 0 && blk < nblk;
        if (PF && lane_on && blk + PD >= 0 && blk + PD < nblk)
            load_block<NS, HOMOG>(A, blk + PD, yneg, col0, srcp, nxt);
        T xo[kH][N];
        float out[STORE_LATE ? n_out(MOM) : 1][kH][kCols];
        if (active) {
            if (!PF) load_block<NS, HOMOG>(A, blk, yneg, col0, srcp, cur);
            if (d == 0) {  // incoming x-edge values (face x_L, or x_R when c < 0)
#pragma unroll
                for (int h = 0; h < kH; ++h)
#pragma unroll
                    for (int k = 0; k < G; ++k) {
                        const int jl = blk * kH + h;
                        float v = 0.f;
                        if (A.inflow && jl < A.J && k < it.n) {
                            const int j = yneg ? (A.J - 1 - jl) : jl;
                            v = A.inflow[(long long)o.ord[k] * A.inflow_stride + (XNEG ? A.J : 0) +
                                         j];
                        }
                        setc(xin[h][G == 1 ? 0 : k >> 1], G == 1 ? 0 : k & 1, v);
                    }
            }
            if (A.leak && A.inflow) {  // x inflow (lane d == 0; rows past J carry zeros)
                T lin = splat<T>(0.f);
#pragma unroll
                for (int h = 0; h < kH; ++h)
#pragma unroll
                    for (int p = 0; p < N; ++p) lin = fma_(lx_in[p], xin[h][p], lin);
                leak.add(neg_(lin));
            }
            const bool full = full_cols && (blk + 1) * kH <= A.J;
            if (full)
                sweep_block<G, MOM, SCHEME, HOMOG, XNEG, false, STORE_LATE>(
                    A, blk, yneg, col0, o, py, xin, xo, cur, out, part_i);
            else
                sweep_block<G, MOM, SCHEME, HOMOG, XNEG, true, STORE_LATE>(
                    A, blk, yneg, col0, o, py, xin, xo, cur, out, part_i);
            if (A.leak) {  // the outflow x face (lane d == L - 1); rows past J leave zeros
                T lo = splat<T>(0.f);
#pragma unroll
                for (int h = 0; h < kH; ++h)
#pragma unroll
                    for (int p = 0; p < N; ++p) lo = fma_(lx_out[p], xo[h][p], lo);
                leak.add(lo);
            }
        } else {
#pragma unroll
            for (int h = 0; h < kH; ++h)
#pragma unroll
                for (int p = 0; p < N; ++p) xo[h][p] = splat<T>(0.f);
        }
        // hand the outgoing x-edge values to the downstream lane
#pragma unroll
        for (int h = 0; h < kH; ++h)
#pragma unroll
            for (int p = 0; p < N; ++p) xin[h][p] = shfl1<XNEG>(xo[h][p]);
        // the step's moments to global memory (when not stored row by row)
        if (STORE_LATE && active) {
            const RowAddr ra(A, blk, yneg, col0);
#pragma unroll
            for (int h = 0; h < kH; ++h)
                if (blk * kH + h < A.J)
#pragma unroll
                    for (int m = 0; m < (STORE_LATE ? n_out(MOM) : 1); ++m)
                        put8<MOM>(part_i + m * A.cells + ra.base + h * ra.rs, out[m][h]);
        }
        if (nwarps > 1) {
            const int lane = g & 31, w = g >> 5;
            const bool sender = XNEG ? (lane == 0 && w > 0) : (lane == 31 && w + 1 < nwarps);
            if (sender) {
#pragma unroll
                for (int h = 0; h < kH; ++h)
#pragma unroll
                    for (int p = 0; p < N; ++p) xbuf[t & 1][w][h][p] = xo[h][p];
            }
            __syncthreads();
            const bool recv = XNEG ? (lane == 31 && w + 1 < nwarps) : (lane == 0 && w > 0);
            if (recv) {
                const int src_w = XNEG ? w + 1 : w - 1;
#pragma unroll
                for (int h = 0; h < kH; ++h)
#pragma unroll
                    for (int p = 0; p < N; ++p) xin[h][p] = xbuf[t & 1][src_w][h][p];
            }
        }
    };
    if constexpr (PF) {
        // blocks of steps 0 .. PD-1 (buffer k holds the block of step k)
#pragma unroll
        for (int k = 0; k < PD; ++k)
            if (lane_on && k - d >= 0 && k - d < nblk)
                load_block<NS, HOMOG>(A, k - d, yneg, col0, srcp, buf[k]);
        int t = 0;
        for (; t + PD < T_steps; t += PD + 1) {
#pragma unroll
            for (int k = 0; k <= PD; ++k) step(t + k, buf[k], buf[(k + PD) % (PD + 1)]);
        }
#pragma unroll
        for (int k = 0; k < PD; ++k)
            if (t + k < T_steps) step(t + k, buf[k], buf[(k + PD) % (PD + 1)]);
    } else {
        for (int t = 0; t < T_steps; ++t) step(t, buf[0], buf[0]);
    }
    if (A.leak) {  // outgoing y-edges of the lane's columns, then one FP64 add per warp
        if (lane_on) {
            T lo = splat<T>(0.f);
#pragma unroll
            for (int r = 0; r < kCols; ++r)
                if (col0 + r < A.I)
#pragma unroll
                    for (int p = 0; p < N; ++p) lo = fma_(o.ly[p], py[r][p], lo);
            leak.add(lo);
        }
        double lk = leak.value();
#pragma unroll
        for (int dd = 16; dd > 0; dd >>= 1) lk += __shfl_xor_sync(0xffffffffu, lk, dd);
        if ((g & 31) == 0 && lk != 0.0) atomicAdd(A.leak + it.sample, lk);
    }
}

template <int G, int MOM, int SCHEME, bool HOMOG, bool BATCH>
__global__ void __launch_bounds__(32 * kMaxWarps) sweep2d_kernel(const SweepArgs A0)
{
    const SweepItem it = A0.items[blockIdx.x];
    if (!A0.active[it.sample]) return;
    SweepArgs A = A0;
    if constexpr (BATCH) {  // the item's own grid
        const GridDesc g = A0.grids[it.grid];
        A.I = g.I;
        A.J = g.J;
        A.NXP = g.NXP;
        A.inv_dx = g.inv_dx;
        A.inv_dy = g.inv_dy;
        A.dx = g.dx;
        A.dy = g.dy;
        A.sigma_t = A0.sigma_t + g.off;
        A.cells = g.cells;
    }
    if (A.stall) {  // test hook: every warp waits on a barrier that nothing completes
        __shared__ unsigned long long never;
        if (threadIdx.x == 0)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32a(&never)) : "memory");
        __syncthreads();
        if (!never_wait(&never, A.wait_ns)) {
            if ((threadIdx.x & 31) == 0) atomicOr(A.err, 1);
            return;
        }
    }
    OrdPacks<G> o;
    const float f = SCHEME == 0 ? 2.f : 1.f;
#pragma unroll
    for (int k = 0; k < G; ++k) {
        float c = 0.f, s = 0.f, w = 0.f;
        int ord = 0;
        if (k < it.n) {
            ord = it.ord[k];
            c = A.oc[ord];
            s = A.os[ord];
            w = A.ow[ord];
        }
        o.ord[k] = ord;
        const float a = f * fabsf(c) * A.inv_dx, b = f * fabsf(s) * A.inv_dy;
        const int p = G == 1 ? 0 : k >> 1, i = G == 1 ? 0 : k & 1;
        setc(o.a[p], i, a);
        setc(o.b[p], i, b);
        setc(o.ab[p], i, a + b);
        setc(o.w[p], i, w);
        setc(o.rd[p], i, HOMOG ? 1.f / (A.sigma_t_homog + a + b) : 0.f);
        setc(o.c[p], i, c);
        setc(o.s[p], i, s);
        setc(o.wc[p], i, w * c);
        setc(o.ws[p], i, w * s);
        const float rd = 1.f / (A.sigma_t_homog + a + b);
        setc(o.al[p], i, (a - b - A.sigma_t_homog) * rd);
        setc(o.a2[p], i, 2.f * a * rd);
        setc(o.b2[p], i, 2.f * b * rd);
        setc(o.be[p], i, (b - a - A.sigma_t_homog) * rd);
        setc(o.r2[p], i, 2.f * rd);
        setc(o.wh[p], i, 0.5f * w);
        setc(o.ar[p], i, a * rd);
        setc(o.br[p], i, b * rd);
        setc(o.lx[p], i, w * fabsf(c) * A.dy);
        setc(o.ly[p], i, w * fabsf(s) * A.dx);
    }
    if (it.quad & 1)
        sweep_item<G, MOM, SCHEME, HOMOG, true>(A, it, o);
    else
        sweep_item<G, MOM, SCHEME, HOMOG, false>(A, it, o);
}

template <int G, int MOM>
cudaError_t launch_g(const SweepArgs &a, int n_items, int nwarps, int scheme, bool homog,
                     cudaStream_t st)
{
    const dim3 grid(n_items), block(32 * nwarps);
#if SWEEP2D_BATCH
    // several grids: sigma_T read per cell (the grids' coefficient blocks)
    (void)homog;
    if (scheme == 0) sweep2d_kernel<G, MOM, 0, false, true><<<grid, block, 0, st>>>(a);
    else sweep2d_kernel<G, MOM, 1, false, true><<<grid, block, 0, st>>>(a);
#else
    if (scheme == 0) {
        if (homog) sweep2d_kernel<G, MOM, 0, true, false><<<grid, block, 0, st>>>(a);
        else sweep2d_kernel<G, MOM, 0, false, false><<<grid, block, 0, st>>>(a);
    } else {
        if (homog) sweep2d_kernel<G, MOM, 1, true, false><<<grid, block, 0, st>>>(a);
        else sweep2d_kernel<G, MOM, 1, false, false><<<grid, block, 0, st>>>(a);
    }
#endif
    return cudaGetLastError();
}

// G, source mode and scheme of one launch of this translation unit's kernels
cudaError_t launch_rows(const SweepArgs &a, int n_items, int nwarps, int G, int scheme,
                        bool homog, int mom, cudaStream_t st)
{
    if (n_items <= 0) return cudaSuccess;
    if (nwarps < 1 || nwarps > kMaxWarps) return cudaErrorInvalidValue;
    if (mom == 1) {
        if (G == 1) return launch_g<1, 1>(a, n_items, nwarps, scheme, homog, st);
        if (G == 2) return launch_g<2, 1>(a, n_items, nwarps, scheme, homog, st);
        if (G == 4) return launch_g<4, 1>(a, n_items, nwarps, scheme, homog, st);
    } else if (mom == 3) {
        if (G == 1) return launch_g<1, 3>(a, n_items, nwarps, scheme, homog, st);
        if (G == 2) return launch_g<2, 3>(a, n_items, nwarps, scheme, homog, st);
        if (G == 4) return launch_g<4, 3>(a, n_items, nwarps, scheme, homog, st);
    }
#if SWEEP2D_WITH_DENSE
    else if (mom == 0) {
        if (G == 1) return launch_g<1, 0>(a, n_items, nwarps, scheme, homog, st);
        if (G == 2) return launch_g<2, 0>(a, n_items, nwarps, scheme, homog, st);
        if (G == 4) return launch_g<4, 0>(a, n_items, nwarps, scheme, homog, st);
    }
#endif
    return cudaErrorInvalidValue;
}

}  // namespace
}  // namespace romk
