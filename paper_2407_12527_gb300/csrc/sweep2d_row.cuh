// sweep2d_row.cuh -- the X-Y transport sweep (K1) with one grid row per wavefront
// step, for the angular-moment source modes (isotropic, linear kernel).
//
// Same cell equations as sweep2d_impl.cuh (Sec. 2, eq. (equ_random)), same work
// items (up to G ordinates of one quadrant of one sample) and the same moment
// accumulators; what changes is the schedule.  Lane g owns the 8 cells
// [8g, 8g + 8) of every row and sweeps row t - d at step t (d: its distance in
// lanes from the inflow face), so the x-edge flux passes one lane per step by a
// shuffle and the y-edge fluxes of its columns stay in registers, as in the
// blocked kernel -- but a step covers one row, so the lane pipeline fills and
// drains in L - 1 steps out of J + L - 1 instead of L - 1 out of J / H + L - 1.
//
// Along its 8 cells a lane solves the upwind x-recurrence in parallel: every cell
// is an affine map of its incoming x-flux, x_out = A x_in + Y, with
//   diamond difference  A = (a - b - sigma_T) rd,  Y = 2 rd (S + b psi_y,in),
//   step scheme          A = a rd,                 Y = rd (S + b psi_y,in),
//   rd = 1 / (sigma_T + a + b),  a, b = 2|c|/dx, 2|s|/dy (DD) or |c|/dx, |s|/dy,
// so the fluxes with x_in = 0 are a prefix (Kogge-Stone, three levels) of the
// cells' maps and the true ones follow in one FMA each once x_in arrives from
// the upstream lane: x_r = Apre_r x_in + P_r.  From x_in and x_out of a cell,
//   DD:   psi_c = (x_in + x_out) / 2,  psi_y,out = x_in + x_out - psi_y,in,
//   step: psi_c = x_out,               psi_y,out = x_out,
// and the moments w psi_c (and w c psi_c, w s psi_c) go to the sample's
// accumulator.  With one sigma_T for the grid the products of A are constants
// of the lane, computed once per work item.
//
// The rows a lane reads (source moments, and sigma_T when it varies) are loaded
// PD steps ahead into a ring of registers.  Ordinates are processed in pairs
// with the packed FP32x2 instructions.  Cells past I (the padding of a ragged
// last lane) are identity maps with no moment (RAGGED instantiations only).
#pragma once
#include <type_traits>

#include "rom_internal.cuh"

namespace romk {
namespace {

template <int G>
struct RowPack {
    using T = float2;
    static constexpr int N = G / 2;
};
template <>
struct RowPack<1> {
    using T = float;
    static constexpr int N = 1;
};

__device__ __forceinline__ float rfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float2 rfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float2 rmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float2 radd(float2 a, float2 b) { return __fadd2_rn(a, b); }
template <class T>
__device__ __forceinline__ T rsplat(float s);
template <>
__device__ __forceinline__ float rsplat<float>(float s) { return s; }
template <>
__device__ __forceinline__ float2 rsplat<float2>(float s) { return make_float2(s, s); }
__device__ __forceinline__ float rhsum(float a) { return a; }
__device__ __forceinline__ float rhsum(float2 a) { return a.x + a.y; }
__device__ __forceinline__ void rset(float &a, int, float v) { a = v; }
__device__ __forceinline__ void rset(float2 &a, int i, float v)
{
    if (i) a.y = v;
    else a.x = v;
}
__device__ __forceinline__ float rrcp(float a)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));  // within 1 ulp; a >= sigma_T > 0
    return r;
}
__device__ __forceinline__ float2 rrcp(float2 a) { return make_float2(rrcp(a.x), rrcp(a.y)); }
template <bool DOWN>
__device__ __forceinline__ float rshfl(float v)
{
    return DOWN ? __shfl_down_sync(0xffffffffu, v, 1) : __shfl_up_sync(0xffffffffu, v, 1);
}
template <bool DOWN>
__device__ __forceinline__ float2 rshfl(float2 v)
{
    return make_float2(rshfl<DOWN>(v.x), rshfl<DOWN>(v.y));
}
// A row for a later step: with one or two ordinates per item a coherent load, which
// stays in order with the moment reductions issued before it and so keeps its place
// PD steps ahead of its use (the read-only .nc form measured 4-5% slower there); with
// four ordinates the .nc form measured faster.  The rows are not written during the
// sweep, so both forms read the same values.
template <int G>
__device__ __forceinline__ void rld8(const float *p, float (&v)[kCols])
{
    if constexpr (G == 4) ldg8_early(p, v);
    else ld8_volatile(p, v);
}
// adds 8 moments to the accumulator; a lane that owns no cells adds nothing (the
// reductions are predicated off, not branched around)
__device__ __forceinline__ void rred8(float *p, const float (&v)[kCols], bool on)
{
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %5, 0;\n\t"
                 "@q red.global.add.v4.f32 [%0], {%1,%2,%3,%4};\n\t}" ::"l"(p), "f"(v[0]),
                 "f"(v[1]), "f"(v[2]), "f"(v[3]), "r"((unsigned)on)
                 : "memory");
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %5, 0;\n\t"
                 "@q red.global.add.v4.f32 [%0], {%1,%2,%3,%4};\n\t}" ::"l"(p + 4), "f"(v[4]),
                 "f"(v[5]), "f"(v[6]), "f"(v[7]), "r"((unsigned)on)
                 : "memory");
}
__device__ __forceinline__ unsigned row_smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}
// test hook: a wait, bounded in time, on an mbarrier that nothing completes
__device__ __forceinline__ bool row_never_wait(unsigned long long *b, unsigned long long budget_ns)
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
            : "r"(row_smem_u32(b)), "r"(0u)
            : "memory");
        if (__all_sync(0xffffffffu, ok != 0)) return true;
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (__any_sync(0xffffffffu, t - t0 > budget_ns)) return false;
    }
}

// arrays read per cell: the source moments (dense mode: one source per ordinate of
// the item), and sigma_T when it varies
__host__ __device__ constexpr int row_arrays(int mom, int g, bool homog)
{
    return (mom == 0 ? g : mom) + (homog ? 0 : 1);
}
// steps between the load of a row and its use (registers: 8 floats per array and slot;
// with four ordinates a deeper ring spills)
__host__ __device__ constexpr int row_pd(int na, int g)
{
    return g == 4 ? (na <= 2 ? 2 : 1) : (na == 1 ? 6 : (na == 2 ? 4 : (na == 3 ? 2 : 1)));
}

template <int G, int MOM, int SCHEME, bool HOMOG, bool XNEG, bool RAGGED, bool MULTI, bool INFLOW>
__device__ __forceinline__ void row_item(const SweepArgs &A, const SweepItem &it)
{
    using T = typename RowPack<G>::T;
    constexpr int N = RowPack<G>::N;
    constexpr int PER = G == 1 ? 1 : 2;  // ordinates per pack
    constexpr int NA = row_arrays(MOM, G, HOMOG);
    constexpr int NS = MOM == 0 ? G : MOM;  // source arrays (the rest: sigma_T)
    constexpr int PD = row_pd(NA, G);
    const int g = threadIdx.x;
    const int nwarps = MULTI ? (int)(blockDim.x >> 5) : 1;
    const int L = (A.I + kCols - 1) / kCols;  // lanes that own cells
    const bool on = g < L;
    const int d = XNEG ? (L - 1 - g) : g;     // lanes between this one and the inflow face
    const int col0 = g * kCols;
    const bool yneg = (it.quad >> 1) & 1;
    const int J = A.J;
    const float st = A.sigma_t_homog;
    const float f = SCHEME == 0 ? 2.f : 1.f;

    // per-ordinate constants in packs
    T ca[N], cb[N], cw[N], cwc[N], cws[N], lx[N], ly[N];
    T aX[N], bY[N], rY[N];  // uniform sigma_T: x_out = aX x + bY py + rY S
    int ord[G];
#pragma unroll
    for (int k = 0; k < G; ++k) {
        float c = 0.f, s = 0.f, w = 0.f;
        int o = it.ord[0];
        if (k < it.n) {
            o = it.ord[k];
            c = A.oc[o];
            s = A.os[o];
            w = A.ow[o];
        }
        ord[k] = o;
        const int p = k / PER, i = k % PER;
        const float a = f * fabsf(c) * A.inv_dx, b = f * fabsf(s) * A.inv_dy;
        // DD moments use (x_in + x_out) = 2 psi_c: half weights
        const float wm = SCHEME == 0 ? 0.5f * w : w;
        rset(ca[p], i, a);
        rset(cb[p], i, b);
        rset(cw[p], i, wm);
        rset(cwc[p], i, wm * c);
        rset(cws[p], i, wm * s);
        rset(lx[p], i, w * fabsf(c) * A.dy);
        rset(ly[p], i, w * fabsf(s) * A.dx);
        const float rd = HOMOG ? 1.f / (st + a + b) : 0.f;
        rset(aX[p], i, SCHEME == 0 ? (a - b - st) * rd : a * rd);
        rset(bY[p], i, SCHEME == 0 ? 2.f * b * rd : b * rd);
        rset(rY[p], i, SCHEME == 0 ? 2.f * rd : rd);
    }
    T cc[N], cs[N];  // linear kernel: S_l = S0 + c_l S1 + s_l S2
#pragma unroll
    for (int k = 0; k < G; ++k) {
        const int p = k / PER, i = k % PER;
        rset(cc[p], i, k < it.n ? A.oc[ord[k]] : 0.f);
        rset(cs[p], i, k < it.n ? A.os[ord[k]] : 0.f);
    }

    // real[rr]: the cell at sweep position rr (r = XNEG ? 7 - rr : rr) is inside the grid
    bool real[kCols];
#pragma unroll
    for (int rr = 0; rr < kCols; ++rr)
        real[rr] = !RAGGED || col0 + (XNEG ? kCols - 1 - rr : rr) < A.I;
    // uniform sigma_T: prefix products of the real cells' A and the tree's powers
    T apow[HOMOG ? kCols : 1][N], pw2[N], pw4[N];
    if constexpr (HOMOG) {
#pragma unroll
        for (int p = 0; p < N; ++p) {
            T acc = rsplat<T>(1.f);
#pragma unroll
            for (int rr = 0; rr < kCols; ++rr) {
                if (real[rr]) acc = rmul(acc, aX[p]);
                apow[rr][p] = acc;
            }
            pw2[p] = rmul(aX[p], aX[p]);
            pw4[p] = rmul(pw2[p], pw2[p]);
        }
    }

    // incoming y-edge fluxes of the lane's columns (face y_B, or y_T when s < 0)
    T py[kCols][N];
#pragma unroll
    for (int r = 0; r < kCols; ++r)
#pragma unroll
        for (int k = 0; k < G; ++k) {
            float v = 0.f;
            if (INFLOW && on && col0 + r < A.I && k < it.n)
                v = A.inflow[(long long)ord[k] * A.inflow_stride + 2 * J + (yneg ? A.I : 0) + col0 +
                             r];
            rset(py[r][k / PER], k % PER, v);
        }
    // net leakage (moment modes): outflow minus inflow through the four faces,
    // sum_l w_l (|c_l| dy sum_rows + |s_l| dx sum_cols) psi; the x-face terms of a
    // step use weights that are zero except on the boundary lanes; FP32 sums over
    // 16 steps go to an FP64 total
    double leak = 0.0;
    T lk = rsplat<T>(0.f);
    float lk_s = 0.f, lk_c = 0.f;  // compensated (Kahan) sum of the ring cycles
    T lx_out[N], lx_in[N];
    const bool keep = A.leak != nullptr;
#pragma unroll
    for (int p = 0; p < N; ++p) {
        lx_out[p] = (keep && on && d == L - 1) ? lx[p] : rsplat<T>(0.f);
        lx_in[p] = (keep && on && d == 0) ? lx[p] : rsplat<T>(0.f);
    }
    if (A.leak && on) {
#pragma unroll
        for (int r = 0; r < kCols; ++r)
#pragma unroll
            for (int p = 0; p < N; ++p) lk = rfma(ly[p], py[r][p], lk);
        leak -= (double)rhsum(lk);
        lk = rsplat<T>(0.f);
    }

    // the item's arrays: source moments of its sample (dense mode: the source of each
    // of its ordinates), sigma_T; its accumulator
    constexpr int NOUT = MOM == 0 ? 1 : MOM;
    const long long soff = A.soff ? A.soff[it.sample] : (long long)it.sample * NOUT * A.cells;
    // A lane that owns no cells points at column 0 with row stride 0: its loads in
    // the unchecked cycles below read a valid row, and its moments are not added.
    const int colb = on ? col0 : 0;
    const float *arr[NA];
#pragma unroll
    for (int m = 0; m < NS; ++m)
        arr[m] = MOM == 0 ? A.src + (long long)ord[m] * A.cells + colb
                          : A.src + soff + (long long)m * A.cells + colb;
    if constexpr (!HOMOG) arr[NA - 1] = A.sigma_t + colb;
    float *part = A.part + soff + colb;
    const long long rs = !on ? 0 : (yneg ? -(long long)A.NXP : (long long)A.NXP);
    const long long row0 = yneg ? (long long)(J - 1) * A.NXP : 0;
    const int T_steps = J + L - 1;

    float buf[PD + 1][NA][kCols];
#pragma unroll
    for (int k = 0; k < PD; ++k) {
        const int jl = k - d;
        if (on && jl >= 0 && jl < J)
#pragma unroll
            for (int m = 0; m < NA; ++m) rld8<G>(arr[m] + row0 + (long long)jl * rs, buf[k][m]);
    }
    __shared__ T xbuf[MULTI ? 2 : 1][MULTI ? kMaxWarps : 1][N];
    T xin[N];
#pragma unroll
    for (int p = 0; p < N; ++p) xin[p] = rsplat<T>(0.f);
    if (INFLOW && on && d == 0) {  // the inflow lane's first row is row 0, at step 0
        const int j = yneg ? J - 1 : 0;
#pragma unroll
        for (int k = 0; k < G; ++k)
            if (k < it.n)
                rset(xin[k / PER], k % PER,
                     A.inflow[(long long)ord[k] * A.inflow_stride + (XNEG ? J : 0) + j]);
    }

    // A ring cycle whose steps all lie where every lane that owns cells has a row to
    // sweep and a row to prefetch runs without the per-lane range checks, so that no
    // branch splits its unrolled steps; the cycles of the pipeline's fill and drain
    // keep them.  Lanes past the grid's width run the same steps on a valid row, with
    // their moments predicated off and a zero outgoing flux, as in the checked steps;
    // psi stores (dense mode) ask for every lane to own cells.
    const bool full = MOM != 0 || L == 32 * nwarps;
    auto cycle = [&](const int t0, auto checked) {
        constexpr bool CK = decltype(checked)::value;
#pragma unroll
        for (int u = 0; u <= PD; ++u) {
            const int t = t0 + u;
            if (CK && t >= T_steps) break;  // uniform over the CTA
            const int jl = t - d;
            {
                const int jp = jl + PD;
                if (!CK || (on && jp >= 0 && jp < J))
#pragma unroll
                    for (int m = 0; m < NA; ++m)
                        rld8<G>(arr[m] + row0 + (long long)jp * rs, buf[(u + PD) % (PD + 1)][m]);
            }
            T xo[N];
            if (!CK || (on && jl >= 0 && jl < J)) {
                const long long row = row0 + (long long)jl * rs;
                const float(&B)[NA][kCols] = buf[u];
                // pass 1: each cell's map with x_in = 0, prefix over the lane's cells
                T P[kCols][N], Am[HOMOG ? 1 : kCols][N];
#pragma unroll
                for (int rr = 0; rr < kCols; ++rr) {
                    const int r = XNEG ? kCols - 1 - rr : rr;
#pragma unroll
                    for (int p = 0; p < N; ++p) {
                        T S = rsplat<T>(B[0][r]);
                        if constexpr (MOM == 0) {  // the pack's own per-ordinate sources
                            rset(S, 0, B[(p * PER) % NS][r]);
                            if constexpr (PER == 2) rset(S, 1, B[(p * PER + 1) % NS][r]);
                        }
                        if constexpr (MOM == 3)
                            S = rfma(cc[p], rsplat<T>(B[1][r]), rfma(cs[p], rsplat<T>(B[2][r]), S));
                        T Y;
                        if constexpr (HOMOG) {
                            Y = rfma(bY[p], py[r][p], rmul(S, rY[p]));
                        } else {
                            const T rden = rrcp(radd(rsplat<T>(B[NA - 1][r]), radd(ca[p], cb[p])));
                            const T rf = SCHEME == 0 ? radd(rden, rden) : rden;
                            Y = rmul(rf, rfma(cb[p], py[r][p], S));
                            Am[rr][p] = SCHEME == 0 ? rfma(radd(ca[p], ca[p]), rden, rsplat<T>(-1.f))
                                                    : rmul(ca[p], rden);
                            if (RAGGED && !real[rr]) Am[rr][p] = rsplat<T>(1.f);
                        }
                        P[rr][p] = (RAGGED && !real[rr]) ? rsplat<T>(0.f) : Y;
                    }
                }
                // Kogge-Stone over the 8 cells: P[rr] = sum_{i <= rr} (prod_{i < m <= rr} A_m) Y_i
#pragma unroll
                for (int lev = 1; lev < kCols; lev <<= 1) {
#pragma unroll
                    for (int rr = kCols - 1; rr >= lev; --rr)
#pragma unroll
                        for (int p = 0; p < N; ++p) {
                            if constexpr (HOMOG) {
                                const T pw = lev == 1 ? aX[p] : (lev == 2 ? pw2[p] : pw4[p]);
                                P[rr][p] = rfma(pw, P[rr - lev][p], P[rr][p]);
                            } else {
                                P[rr][p] = rfma(Am[rr][p], P[rr - lev][p], P[rr][p]);
                                Am[rr][p] = rmul(Am[rr][p], Am[rr - lev][p]);
                            }
                        }
                }
                // pass 2: the cells with their true incoming flux
                float v0[kCols], v1[kCols], v2[kCols];
                float psi_row[MOM == 0 ? G : 1][kCols];  // dense mode: psi_c of each ordinate
                T xprev[N];
#pragma unroll
                for (int p = 0; p < N; ++p) xprev[p] = xin[p];
#pragma unroll
                for (int rr = 0; rr < kCols; ++rr) {
                    const int r = XNEG ? kCols - 1 - rr : rr;
                    T a0 = rsplat<T>(0.f), a1 = rsplat<T>(0.f), a2 = rsplat<T>(0.f);
#pragma unroll
                    for (int p = 0; p < N; ++p) {
                        const T apre = HOMOG ? apow[HOMOG ? rr : 0][p] : Am[HOMOG ? 0 : rr][p];
                        const T xn = rfma(apre, xin[p], P[rr][p]);
                        // DD: x_in + x_out = 2 psi_c; step: x_out = psi_c
                        const T m = SCHEME == 0 ? radd(xprev[p], xn) : xn;
                        a0 = rfma(cw[p], m, a0);
                        if constexpr (MOM == 0) {
                            const T pc = SCHEME == 0 ? rmul(m, rsplat<T>(0.5f)) : xn;
                            const bool rl1 = !RAGGED || real[rr];
                            if constexpr (PER == 2) {
                                psi_row[(2 * p) % G][r] = rl1 ? reinterpret_cast<const float2 &>(pc).x : 0.f;
                                psi_row[(2 * p + 1) % G][r] = rl1 ? reinterpret_cast<const float2 &>(pc).y : 0.f;
                            } else {
                                psi_row[0][r] = rl1 ? reinterpret_cast<const float &>(pc) : 0.f;
                            }
                        }
                        if constexpr (MOM == 3) {
                            a1 = rfma(cwc[p], m, a1);
                            a2 = rfma(cws[p], m, a2);
                        }
                        if (!RAGGED || real[rr]) {
                            py[r][p] = SCHEME == 0 ? rfma(py[r][p], rsplat<T>(-1.f), m) : xn;
                            xprev[p] = xn;
                        }
                    }
                    const bool rl = !RAGGED || real[rr];
                    v0[r] = rl ? rhsum(a0) : 0.f;
                    if constexpr (MOM == 3) {
                        v1[r] = rl ? rhsum(a1) : 0.f;
                        v2[r] = rl ? rhsum(a2) : 0.f;
                    }
                }
#pragma unroll
                for (int p = 0; p < N; ++p) xo[p] = (CK || on) ? xprev[p] : rsplat<T>(0.f);
                rred8(part + row, v0, on);
                if constexpr (MOM == 0) {  // psi of every ordinate of the item, for the contraction
#pragma unroll
                    for (int k = 0; k < G; ++k)
                        if (k < it.n) {
                            const long long off = (long long)ord[k] * A.cells + row + col0;
                            if (A.psi_split) st8_split(A.psi_split, off, psi_row[k]);
                            else stg8(A.psi + off, psi_row[k]);
                        }
                }
                if constexpr (MOM == 3) {
                    rred8(part + A.cells + row, v1, on);
                    rred8(part + 2 * A.cells + row, v2, on);
                }
                // x-face leakage terms (zero weights except on the boundary lanes)
#pragma unroll
                for (int p = 0; p < N; ++p) {
                    lk = rfma(lx_out[p], xo[p], lk);
                    if constexpr (INFLOW) lk = rfma(rsplat<T>(-1.f), rmul(lx_in[p], xin[p]), lk);
                }
            } else {
#pragma unroll
                for (int p = 0; p < N; ++p) xo[p] = rsplat<T>(0.f);
            }
            // the outgoing x-flux to the downstream lane; the inflow lane takes the
            // boundary value of its next row (x_L, or x_R when c < 0; 0 for vacuum)
#pragma unroll
            for (int p = 0; p < N; ++p) xin[p] = rshfl<XNEG>(xo[p]);
            if constexpr (INFLOW) {
                const int jn = t + 1 - d;
                const bool take = on && d == 0 && jn < J;
                const int j = yneg ? (J - 1 - jn) : jn;
#pragma unroll
                for (int k = 0; k < G; ++k) {
                    const float v = (take && k < it.n)
                                         ? A.inflow[(long long)ord[k] * A.inflow_stride +
                                                    (XNEG ? J : 0) + j]
                                         : 0.f;
                    if (d == 0) rset(xin[k / PER], k % PER, v);
                }
            } else {
#pragma unroll
                for (int p = 0; p < N; ++p) xin[p] = d == 0 ? rsplat<T>(0.f) : xin[p];
            }
            if (MULTI && nwarps > 1) {  // across warps through shared memory, one barrier per step
                const int lane = g & 31, w = g >> 5;
                const bool sender = XNEG ? (lane == 0 && w > 0) : (lane == 31 && w + 1 < nwarps);
                if (sender)
#pragma unroll
                    for (int p = 0; p < N; ++p) xbuf[MULTI ? (t & 1) : 0][w][p] = xo[p];
                __syncthreads();
                const bool recv = XNEG ? (lane == 31 && w + 1 < nwarps) : (lane == 0 && w > 0);
                if (recv) {
                    const int src_w = XNEG ? w + 1 : w - 1;
#pragma unroll
                    for (int p = 0; p < N; ++p) xin[p] = xbuf[MULTI ? (t & 1) : 0][src_w][p];
                }
            }
        }
        // the ring cycle's leakage sum into a compensated FP32 total (no FP64
        // arithmetic in the loop: GB300's FP64 pipe is narrow and slow)
        {
            const float y = rhsum(lk) - lk_c;
            const float tt = lk_s + y;
            lk_c = (tt - lk_s) - y;
            lk_s = tt;
            lk = rsplat<T>(0.f);
        }
    };
    for (int t0 = 0; t0 < T_steps; t0 += PD + 1) {
        if (full && t0 >= L - 1 && t0 + 2 * PD <= J - 1) cycle(t0, std::false_type{});
        else cycle(t0, std::true_type{});
    }
    if (A.leak) {  // the x-face sums, the outgoing y-edges; one FP64 add per warp
        leak += (double)lk_s - (double)lk_c;
        if (on) {
            T lo = rsplat<T>(0.f);
#pragma unroll
            for (int r = 0; r < kCols; ++r)
                if (col0 + r < A.I)
#pragma unroll
                    for (int p = 0; p < N; ++p) lo = rfma(ly[p], py[r][p], lo);
            leak += (double)rhsum(lo);
        }
#pragma unroll
        for (int dd = 16; dd > 0; dd >>= 1) leak += __shfl_xor_sync(0xffffffffu, leak, dd);
        if ((g & 31) == 0 && leak != 0.0) atomicAdd(A.leak + it.sample, leak);
    }
}

template <int G, int MOM, int SCHEME, bool HOMOG, bool BATCH, bool MULTI, bool INFLOW>
__global__ void __launch_bounds__(32 * kMaxWarps) sweep2d_row_kernel(const SweepArgs A0)
{
    const SweepItem it = A0.items[blockIdx.x];
    if (!A0.active[it.sample]) return;
    SweepArgs A = A0;
    if constexpr (BATCH) {  // the item's own grid
        const GridDesc gd = A0.grids[it.grid];
        A.I = gd.I;
        A.J = gd.J;
        A.NXP = gd.NXP;
        A.inv_dx = gd.inv_dx;
        A.inv_dy = gd.inv_dy;
        A.dx = gd.dx;
        A.dy = gd.dy;
        A.sigma_t = A0.sigma_t + gd.off;
        A.cells = gd.cells;
    }
    if (A.stall) {  // test hook: every warp waits on a barrier that nothing completes
        __shared__ unsigned long long never;
        if (threadIdx.x == 0)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(row_smem_u32(&never))
                         : "memory");
        __syncthreads();
        if (!row_never_wait(&never, A.wait_ns)) {
            if ((threadIdx.x & 31) == 0) atomicOr(A.err, 1);
            return;
        }
    }
    const bool ragged = A.I % kCols != 0;
    if (it.quad & 1) {
        if (ragged) row_item<G, MOM, SCHEME, HOMOG, true, true, MULTI, INFLOW>(A, it);
        else row_item<G, MOM, SCHEME, HOMOG, true, false, MULTI, INFLOW>(A, it);
    } else {
        if (ragged) row_item<G, MOM, SCHEME, HOMOG, false, true, MULTI, INFLOW>(A, it);
        else row_item<G, MOM, SCHEME, HOMOG, false, false, MULTI, INFLOW>(A, it);
    }
}

// one kernel per (G, homog, multi-warp, inflow) of this translation unit's source
// mode MOM and scheme SCHEME; items of one ordinate run on the two-ordinate
// kernel (the empty second slot has zero weight)
template <int MOM, int SCHEME, bool BATCH>
cudaError_t row_launch(const SweepArgs &a, int n_items, int nwarps, int G, bool homog,
                       cudaStream_t st)
{
    if (n_items <= 0) return cudaSuccess;
    if (nwarps < 1 || nwarps > kMaxWarps || (G != 1 && G != 2 && G != 4))
        return cudaErrorInvalidValue;
    const dim3 grid(n_items), block(32 * nwarps);
    const bool multi = nwarps > 1, inflow = a.inflow != nullptr;
#define ROW_K(GG, HH, MM, II) sweep2d_row_kernel<GG, MOM, SCHEME, HH, BATCH, MM, II><<<grid, block, 0, st>>>(a)
#define ROW_G(GG, HH)                                        \
    do {                                                     \
        if (multi) {                                         \
            if (inflow) ROW_K(GG, HH, true, true);           \
            else ROW_K(GG, HH, true, false);                 \
        } else {                                             \
            if (inflow) ROW_K(GG, HH, false, true);          \
            else ROW_K(GG, HH, false, false);                \
        }                                                    \
    } while (0)
    if constexpr (BATCH) {
        (void)homog;  // several grids: sigma_T read per cell, vacuum boundaries
        if (G == 4) {
            if (multi) ROW_K(4, false, true, false);
            else ROW_K(4, false, false, false);
        } else {
            if (multi) ROW_K(2, false, true, false);
            else ROW_K(2, false, false, false);
        }
    } else {
        if (G == 4) {
            if (homog) ROW_G(4, true);
            else ROW_G(4, false);
        } else {
            if (homog) ROW_G(2, true);
            else ROW_G(2, false);
        }
    }
#undef ROW_G
#undef ROW_K
    return cudaGetLastError();
}

}  // namespace
}  // namespace romk
