// sweep3d.cu -- transport sweep of the discrete ordinate system in 3D (x-y-z)
// geometry (K9).
//
// The RTE of Sec. 1 (eq. equ_1) is posed for z in R^3; the paper tests only
// slab and X-Y.  Here every ordinate u_l = (c, s, mu_z) of every active sample
// is swept on an I x J x K grid with the 3D form of the cell balance of Sec. 2:
//   psi_c = (S + a psi_xin + b psi_yin + e psi_zin) / (sigma_T + a + b + e),
//   DD:   a = 2|c|/dx, b = 2|s|/dy, e = 2|mu_z|/dz, psi_out = 2 psi_c - psi_in,
//   step: a =  |c|/dx, b =  |s|/dy, e =  |mu_z|/dz, psi_out = psi_c,
// and phi_s += w_l psi_c is accumulated per sample (isotropic scattering:
// S = sigma_S phi + q, formed by the combine kernel).
//
// GB300 mapping.  A CTA owns one x-y tile of up to 64 x 128 cells and sweeps
// a list of work items (G = 1 or 2 ordinates of one sample, all items of one
// octant) through every z-plane, item after item without draining.  Warp w is
// the w-th 8-column strip of the tile counted from the inflow side (one
// aligned 32-byte sector of FP32 per row); lane d is the d-th block of 4 rows
// counted from the inflow side.  Plane p of the item stream reaches lane d of
// every warp at the warp's step p + d, so
//   - the z-dependence (the 4 x 8 z-edges of the lane's block, per ordinate)
//     stays in registers from one plane to the next;
//   - the y-dependence (8 columns) moves one lane per step by a warp shuffle;
//   - the x-dependence (4 rows) moves from warp w to warp w + 1 through a
//     ring of shared-memory slots guarded by mbarriers, so warps run ahead of
//     each other by up to the ring depth instead of meeting at a CTA barrier.
// The wavefront surface of the item (one z-edge per column of the tile and
// ordinate) therefore lives in the register file.  Global memory sees only
// the source and sigma_T rows, which each lane loads one step ahead (a row is
// reloaded for the next plane as soon as it has been used, so the load
// latency overlaps a whole step; a coherent load, which stays in order with the
// flux reductions before it, measured 1% faster per step than the read-only .nc
// form; the rows are not written during the sweep), and the flux accumulation, one vector
// reduction (red.global.add.v4.f32) per 4 cells and item into the sample's
// phi: no per-item partial arrays, whose size (cells x ordinates) would
// exceed the flux itself by the ordinate count.  Those three arrays are kept
// in diagonal storage (Skew3): the 32 lanes of a warp sit on one diagonal of
// the (plane, row block) wavefront at consecutive blocks, so every row access
// of a warp instruction is one contiguous kilobyte instead of 32 lines.  Two ordinates share each
// source load and flux reduction and run as FP32x2 pairs (__ffma2_rn ...).
// With 255 registers per thread a CTA is 8 warps, one per SM.  Wider x-y
// extents are cut into tiles swept by successive launches in upwind order; a
// tile hands its downstream x- and y-edges to the next tile through per-item
// face buffers.  Every mbarrier wait is bounded in time (globaltimer): on
// timeout the kernel raises an error flag and returns.
#include "rom_internal.cuh"

namespace romk {
namespace {

constexpr int kH3 = 4;                  // rows per lane
constexpr int kStrips = 8;              // 8-column strips (warps) per tile: 64 columns
constexpr int kTileRows = 32 * kH3;     // 128 rows per tile
constexpr int kSlots = 4;               // x-edge ring depth between neighbouring warps

struct Smem3 {
    float4 ring[kStrips][kSlots][32][2];  // 4 rows x up to 2 ordinates per lane
    unsigned long long full[kStrips][kSlots];
    unsigned long long empty[kStrips][kSlots];
    unsigned long long never;  // test hook: a barrier no thread arrives on
    int sample[kMaxCtaItems3];
    int ord[kMaxCtaItems3][2];
    int item[kMaxCtaItems3];
    int n_list;
};

// one ordinate (float) or a pair (float2, packed FP32x2 arithmetic)
template <int G>
struct V3 {
    using T = float2;
};
template <>
struct V3<1> {
    using T = float;
};
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float vneg(float a) { return -a; }
__device__ __forceinline__ float2 vneg(float2 a) { return make_float2(-a.x, -a.y); }
template <class T>
__device__ __forceinline__ T vsplat(float s);
template <>
__device__ __forceinline__ float vsplat<float>(float s) { return s; }
template <>
__device__ __forceinline__ float2 vsplat<float2>(float s) { return make_float2(s, s); }
__device__ __forceinline__ float vget(float a, int) { return a; }
__device__ __forceinline__ float vget(float2 a, int g) { return g ? a.y : a.x; }
__device__ __forceinline__ void vset(float &a, int, float v) { a = v; }
__device__ __forceinline__ void vset(float2 &a, int g, float v)
{
    if (g) a.y = v;
    else a.x = v;
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float vrcp(float a) { return rcp_approx(a); }
__device__ __forceinline__ float2 vrcp(float2 a) { return make_float2(rcp_approx(a.x), rcp_approx(a.y)); }
// sum over the ordinates of w_g psi_g
__device__ __forceinline__ float wsum(float w, float p) { return w * p; }
__device__ __forceinline__ float wsum(float2 w, float2 p) { return fmaf(w.y, p.y, w.x * p.x); }

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long *b, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *b)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(
                     smem_u32(b))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *b, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity), "r"(1000u)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long gtimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait (all lanes of the warp together) for the phase of `parity` to complete,
// for at most budget_ns nanoseconds (the decision to give up is warp-uniform).
__device__ __forceinline__ bool wait_warp(unsigned long long *b, unsigned parity,
                                          unsigned long long budget_ns)
{
    if (__all_sync(0xffffffffu, mbar_try_wait(b, parity))) return true;
    const unsigned long long t0 = gtimer_ns();
    for (;;) {
        if (__all_sync(0xffffffffu, mbar_try_wait(b, parity))) return true;
        if (__any_sync(0xffffffffu, gtimer_ns() - t0 > budget_ns)) return false;
    }
}

__device__ __forceinline__ void red8(float *p, const float (&v)[kCols])
{
    asm volatile("red.global.add.v4.f32 [%0], {%1,%2,%3,%4};" ::"l"(p), "f"(v[0]), "f"(v[1]),
                 "f"(v[2]), "f"(v[3])
                 : "memory");
    asm volatile("red.global.add.v4.f32 [%0], {%1,%2,%3,%4};" ::"l"(p + 4), "f"(v[4]), "f"(v[5]),
                 "f"(v[6]), "f"(v[7])
                 : "memory");
}

// One step of a lane: its 4 x 8 block for the G ordinates of the item.  The
// cells are taken by anti-diagonals of the block (cell (h, r) at diagonal h + r,
// r counted from the x inflow side), so the up to four cells of a diagonal are
// independent and their dependent FMA chains overlap.  A row's flux goes out
// (one vector reduction per 4 cells) as soon as the row is done, and its source
// and sigma_T registers are reloaded with the row of the next step.
template <int G, int SCHEME, bool XNEG, bool CHECK>
__device__ __forceinline__ void block_diag(
    const typename V3<G>::T a, const typename V3<G>::T b, const typename V3<G>::T e,
    const typename V3<G>::T abe, const typename V3<G>::T wg, const typename V3<G>::T (&xin)[kH3],
    typename V3<G>::T (&y)[kCols], typename V3<G>::T (&z)[kH3][kCols], float (&pS)[kH3][kCols],
    float (&pT)[kH3][kCols], const bool (&rok)[kH3], const bool (&cok)[kCols], float *phi_k,
    const float *sp2, const float *tp2, const int (&rowpart)[kH3], bool act2,
    typename V3<G>::T (&xo)[kH3])
{
    using T = typename V3<G>::T;
    T x[kH3];
    float out[kH3][kCols];
#pragma unroll
    for (int h = 0; h < kH3; ++h) x[h] = xin[h];
#pragma unroll
    for (int d = 0; d < kCols + kH3 - 1; ++d) {
#pragma unroll
        for (int h = 0; h < kH3; ++h) {
            const int rr = d - h;
            if (rr < 0 || rr >= kCols) continue;
            const int r = XNEG ? kCols - 1 - rr : rr;
            if (CHECK && !(rok[h] && cok[r])) {
                out[h][r] = 0.f;
                continue;
            }
            const T num = vfma(a, x[h], vfma(b, y[r], vfma(e, z[h][r], vsplat<T>(pS[h][r]))));
            const T pc = vmul(num, vrcp(vadd(vsplat<T>(pT[h][r]), abe)));
            if (SCHEME == 0) {
                const T two = vsplat<T>(2.f);
                x[h] = vfma(two, pc, vneg(x[h]));
                y[r] = vfma(two, pc, vneg(y[r]));
                z[h][r] = vfma(two, pc, vneg(z[h][r]));
            } else {
                x[h] = pc;
                y[r] = pc;
                z[h][r] = pc;
            }
            out[h][r] = wsum(wg, pc);
        }
        const int hf = d - (kCols - 1);  // the row finished at this diagonal
        if (hf >= 0 && hf < kH3) {
            xo[hf] = x[hf];
            if (!CHECK || rok[hf]) {
                red8(phi_k + rowpart[hf], out[hf]);
                if (act2) {
                    ld8_volatile(sp2 + rowpart[hf], pS[hf]);
                    ld8_volatile(tp2 + rowpart[hf], pT[hf]);
                }
            }
        }
    }
}

template <int G, int SCHEME, bool XNEG>
__device__ __forceinline__ void sweep3_body(const Sweep3Args &A, Smem3 &sm, int oct)
{
    using T = typename V3<G>::T;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int L = (A.I + kCols - 1) / kCols;  // 8-column strips of the grid
    const int ls0 = A.tile_x * kStrips;       // first strip of the tile (upwind order)
    const int nw = min(kStrips, L - ls0);
    if (w >= nw) return;
    // rows counted from the inflow side over Jp = 4 ceil(J / 4) rows: with s < 0 the
    // count starts at row Jp - 1, so the 4-row blocks of every lane are aligned
    const int Jp = 4 * A.sk.NBg;
    const int jt0 = A.tile_y * kTileRows;     // first row of the tile (upwind order)
    const int nrows = min(kTileRows, Jp - jt0);
    const int NB = nrows / kH3;               // lanes with rows
    const bool yneg = (oct >> 1) & 1, zneg = (oct >> 2) & 1;
    const int col0 = (XNEG ? (L - 1 - (ls0 + w)) : (ls0 + w)) * kCols;
    const bool first_x = w == 0, last_x = w == nw - 1;
    const bool up_x = A.tile_x > 0, down_x = A.tile_x + 1 < A.n_tx;
    const bool up_y = A.tile_y > 0, down_y = A.tile_y + 1 < A.n_ty;
    const int I = A.I, J = A.J, K = A.K, NXP = A.NXP;
    const long long plane = A.sk.DS;  // one z-plane further: one diagonal further
    const int fam = yneg == zneg ? 0 : 1;
    const float *const sig_f = A.sigma_t + (long long)fam * A.sk.cells;
    const float *const src_f = A.src + (long long)fam * A.S * A.sk.cells;
    float *const phi_f = A.phi + (long long)fam * A.S * A.sk.cells;
    const long long fx = (long long)K * J, fy = (long long)K * I, fz = (long long)J * I;
    const float f = SCHEME == 0 ? 2.f : 1.f;
    const int n_items = sm.n_list;
    const int T_steps = n_items * K + NB - 1;

    int jrow[kH3];
    bool rok[kH3];
    int rowpart[kH3];  // diagonal-storage offset of the row at plane 0 (sk.cells < 2^31)
#pragma unroll
    for (int h = 0; h < kH3; ++h) {
        const int r = lane * kH3 + h;  // row within the tile, upwind order
        const int jl = jt0 + r;
        jrow[h] = yneg ? Jp - 1 - jl : jl;
        rok[h] = r < nrows && jrow[h] >= 0 && jrow[h] < J;
        rowpart[h] = rok[h] ? (int)skew3_index(A.sk, fam, 0, jrow[h], col0 / kCols) : 0;
    }
    bool cok[kCols];
#pragma unroll
    for (int r = 0; r < kCols; ++r) cok[r] = col0 + r < I;
    // warp-uniform: every lane's block is 4 full rows of 8 valid cells
    const bool full = col0 + kCols <= I && J == Jp;

    T a = vsplat<T>(0.f), b = a, e = a, abe = vsplat<T>(1.f), wg = a;
    float *phip = phi_f;
    int item = 0;
    T z[kH3][kCols], y[kCols], xin[kH3];
    float pS[kH3][kCols], pT[kH3][kCols];  // the lane's rows for the current step
#pragma unroll
    for (int h = 0; h < kH3; ++h) {
        xin[h] = vsplat<T>(0.f);
#pragma unroll
        for (int r = 0; r < kCols; ++r) z[h][r] = vsplat<T>(0.f);
    }
#pragma unroll
    for (int r = 0; r < kCols; ++r) y[r] = vsplat<T>(0.f);

    // stream position of the lane at step t: p = t - lane, item n = p / K, plane kl = p % K
    int kl = -lane, n = 0;
    if (lane == 0 && n_items > 0 && 0 < NB) {  // rows of the first step
        const long long off = (long long)(zneg ? K - 1 : 0) * plane;
        const float *sp = src_f + (long long)sm.sample[0] * A.sk.cells + off;
#pragma unroll
        for (int h = 0; h < kH3; ++h)
            if (rok[h]) {
                ld8_volatile(sp + rowpart[h], pS[h]);
                ld8_volatile(sig_f + off + rowpart[h], pT[h]);
            }
    }

    for (int t = 0; t < T_steps; ++t) {
        const bool act = lane < NB && kl >= 0 && n < n_items;
        int kl2 = kl + 1, n2 = n;
        if (kl2 == K) {
            kl2 = 0;
            ++n2;
        }
        const bool act2 = lane < NB && kl2 >= 0 && n2 < n_items;
        const int slot = t % kSlots;
        const unsigned par = (unsigned)(t / kSlots) & 1u;
        if (act && kl == 0) {  // the item's ordinates reach this lane
            item = sm.item[n];
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const int o = sm.ord[n][g];
                const float ag = f * fabsf(A.oc[o]) * A.inv_dx;
                const float bg = f * fabsf(A.os[o]) * A.inv_dy;
                const float eg = f * fabsf(A.oz[o]) * A.inv_dz;
                vset(a, g, ag);
                vset(b, g, bg);
                vset(e, g, eg);
                vset(abe, g, ag + bg + eg);
                vset(wg, g, g < A.items[item].n ? A.ow[o] : 0.f);
            }
            phip = phi_f + (long long)sm.sample[n] * A.sk.cells;
            const long long zf = 2 * fx + 2 * fy + (zneg ? fz : 0);
#pragma unroll
            for (int h = 0; h < kH3; ++h)
#pragma unroll
                for (int r = 0; r < kCols; ++r)
#pragma unroll
                    for (int g = 0; g < G; ++g) {
                        float v = 0.f;
                        if (A.inflow && rok[h] && cok[r])
                            v = A.inflow[(long long)sm.ord[n][g] * A.inflow_stride + zf +
                                         (long long)jrow[h] * I + col0 + r];
                        vset(z[h][r], g, v);
                    }
        }
        const int k = zneg ? K - 1 - kl : kl;
        // incoming x-edges of the lane's rows
        if (first_x) {
            if (act) {
#pragma unroll
                for (int h = 0; h < kH3; ++h)
#pragma unroll
                    for (int g = 0; g < G; ++g) {
                        float v = 0.f;
                        if (rok[h]) {
                            const long long fi = (long long)k * J + jrow[h];
                            if (up_x) v = A.xface[((long long)item * G + g) * fx + fi];
                            else if (A.inflow)
                                v = A.inflow[(long long)sm.ord[n][g] * A.inflow_stride +
                                             (XNEG ? fx : 0) + fi];
                        }
                        vset(xin[h], g, v);
                    }
            }
        } else {
            if (!wait_warp(&sm.full[w - 1][slot], par, A.wait_ns)) {
                if (lane == 0) atomicOr(A.err, 1);
                return;
            }
            const float4 v0 = sm.ring[w - 1][slot][lane][0];
            if constexpr (G == 1) {
                xin[0] = v0.x;
                xin[1] = v0.y;
                xin[2] = v0.z;
                xin[3] = v0.w;
            } else {
                const float4 v1 = sm.ring[w - 1][slot][lane][1];
                vset(xin[0], 0, v0.x); vset(xin[0], 1, v0.y);
                vset(xin[1], 0, v0.z); vset(xin[1], 1, v0.w);
                vset(xin[2], 0, v1.x); vset(xin[2], 1, v1.y);
                vset(xin[3], 0, v1.z); vset(xin[3], 1, v1.w);
            }
            mbar_arrive(&sm.empty[w - 1][slot]);
        }
        // incoming y-edges of the first row block (the others arrive by shuffle)
        if (lane == 0 && act) {
#pragma unroll
            for (int r = 0; r < kCols; ++r)
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    float v = 0.f;
                    if (cok[r]) {
                        if (up_y)
                            v = A.yface[((long long)item * G + g) * K * NXP + (long long)k * NXP +
                                        col0 + r];
                        else if (A.inflow)
                            v = A.inflow[(long long)sm.ord[n][g] * A.inflow_stride + 2 * fx +
                                         (yneg ? fy : 0) + (long long)k * I + col0 + r];
                    }
                    vset(y[r], g, v);
                }
        }
        // the rows of the next step are loaded as soon as this step has used them
        const int k2 = zneg ? K - 1 - kl2 : kl2;
        const long long off2 = (long long)k2 * plane;
        const float *sp2 = src_f + (long long)sm.sample[act2 ? n2 : 0] * A.sk.cells + off2;
        const float *tp2 = sig_f + off2;
        T xo[kH3];
        const long long pk = (long long)k * plane;
        if (act) {
            if (full)
                block_diag<G, SCHEME, XNEG, false>(a, b, e, abe, wg, xin, y, z, pS, pT, rok, cok,
                                                    phip + pk, sp2, tp2, rowpart, act2, xo);
            else
                block_diag<G, SCHEME, XNEG, true>(a, b, e, abe, wg, xin, y, z, pS, pT, rok, cok,
                                                   phip + pk, sp2, tp2, rowpart, act2, xo);
        } else {
#pragma unroll
            for (int h = 0; h < kH3; ++h) {
                xo[h] = vsplat<T>(0.f);
                if (act2 && rok[h]) {
                    ld8_volatile(sp2 + rowpart[h], pS[h]);
                    ld8_volatile(tp2 + rowpart[h], pT[h]);
                }
            }
        }
        // outgoing x-edges to the next strip (or the next tile)
        if (last_x) {
            if (act && down_x) {
#pragma unroll
                for (int h = 0; h < kH3; ++h)
                    if (rok[h])
#pragma unroll
                        for (int g = 0; g < G; ++g)
                            A.xface[((long long)item * G + g) * fx + (long long)k * J + jrow[h]] =
                                vget(xo[h], g);
            }
        } else {
            if (t >= kSlots && !wait_warp(&sm.empty[w][slot], par ^ 1u, A.wait_ns)) {
                if (lane == 0) atomicOr(A.err, 2);
                return;
            }
            if constexpr (G == 1) {
                sm.ring[w][slot][lane][0] = make_float4(xo[0], xo[1], xo[2], xo[3]);
            } else {
                sm.ring[w][slot][lane][0] = make_float4(xo[0].x, xo[0].y, xo[1].x, xo[1].y);
                sm.ring[w][slot][lane][1] = make_float4(xo[2].x, xo[2].y, xo[3].x, xo[3].y);
            }
            mbar_arrive(&sm.full[w][slot]);
        }
        // outgoing y-edges: the last row block of the tile to the next tile
        if (down_y && act && lane == NB - 1) {
#pragma unroll
            for (int g = 0; g < G; ++g) {
                float v[kCols];
#pragma unroll
                for (int r = 0; r < kCols; ++r) v[r] = vget(y[r], g);
                stg8(A.yface + ((long long)item * G + g) * K * NXP + (long long)k * NXP + col0, v);
            }
        }
#pragma unroll
        for (int r = 0; r < kCols; ++r) {
            if constexpr (G == 1) {
                y[r] = __shfl_up_sync(0xffffffffu, y[r], 1);
            } else {
                y[r].x = __shfl_up_sync(0xffffffffu, y[r].x, 1);
                y[r].y = __shfl_up_sync(0xffffffffu, y[r].y, 1);
            }
        }
        kl = kl2;
        n = n2;
    }
}

template <int G, int SCHEME>
__global__ void __launch_bounds__(32 * kStrips, 1) sweep3d_kernel(const Sweep3Args A)
{
    __shared__ Smem3 sm;
    const int lb = A.cta_begin[blockIdx.x], le = A.cta_begin[blockIdx.x + 1];
    if (threadIdx.x < 32) {
        // the CTA's items whose sample is still iterating, in list order
        const int lane = threadIdx.x;
        int n = 0;
        for (int i0 = lb; i0 < le; i0 += 32) {
            const int i = i0 + lane;
            int it = 0;
            SweepItem si{};
            bool keep = false;
            if (i < le) {
                it = A.cta_list[i];
                si = A.items[it];
                keep = A.active[si.sample] != 0;
            }
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                const int d = n + __popc(m & ((1u << lane) - 1u));
                sm.item[d] = it;
                sm.sample[d] = si.sample;
                sm.ord[d][0] = si.ord[0];
                sm.ord[d][1] = si.ord[si.n > 1 ? 1 : 0];
            }
            n += __popc(m);
        }
        if (lane == 0) sm.n_list = n;
        for (int i = lane; i < kStrips * kSlots; i += 32) {
            mbar_init(&sm.full[i / kSlots][i % kSlots], 32);
            mbar_init(&sm.empty[i / kSlots][i % kSlots], 32);
        }
        if (lane == 0) mbar_init(&sm.never, 1);
    }
    __syncthreads();
    if (sm.n_list == 0) return;
    if (A.stall) {  // test hook: wait for a phase that never completes
        if (!wait_warp(&sm.never, 0u, A.wait_ns)) {
            if ((threadIdx.x & 31) == 0) atomicOr(A.err, 4);
            return;
        }
    }
    const int oct = A.items[sm.item[0]].quad;
    if (oct & 1) sweep3_body<G, SCHEME, true>(A, sm, oct);
    else sweep3_body<G, SCHEME, false>(A, sm, oct);
}

}  // namespace

int sweep3d_ctas_per_sm(int nwarps, int G)
{
    int n = 0;
    const cudaError_t e =
        G == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep3d_kernel<1, 0>, 32 * nwarps, 0)
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep3d_kernel<2, 0>, 32 * nwarps, 0);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

int sweep3d_tile_cols() { return kStrips * kCols; }

cudaError_t launch_sweep3d(const Sweep3Args &a, int n_ctas, int nwarps, int G, int scheme,
                           cudaStream_t st)
{
    if (n_ctas <= 0) return cudaSuccess;
    if (nwarps < 1 || nwarps > kStrips) return cudaErrorInvalidValue;
    const dim3 grid(n_ctas), block(32 * nwarps);
    if (G == 1) {
        if (scheme == 0) sweep3d_kernel<1, 0><<<grid, block, 0, st>>>(a);
        else sweep3d_kernel<1, 1><<<grid, block, 0, st>>>(a);
    } else if (G == 2) {
        if (scheme == 0) sweep3d_kernel<2, 0><<<grid, block, 0, st>>>(a);
        else sweep3d_kernel<2, 1><<<grid, block, 0, st>>>(a);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace romk
