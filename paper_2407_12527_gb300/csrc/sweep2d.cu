// sweep2d.cu -- transport sweep of the discrete ordinate system (K1).
//
// One sweep solves, for every ordinate l of every active sample, the
// diamond-difference cell equations of eq. (equ_random) on the I x J grid
// (Sec. 2) in upwind order, given the scattering source of the previous source
// iteration, and accumulates the scalar-flux moments of each work item:
//   psi_c = (S_l + a psi_xin + b psi_yin) / (sigma_T + a + b),
//   DD:   a = 2|c|/dx, b = 2|s|/dy, psi_out = 2 psi_c - psi_in,
//   step: a =  |c|/dx, b =  |s|/dy, psi_out = psi_c,
//   phi += w_l psi_c   (and Jx += w_l c_l psi_c, Jy += w_l s_l psi_c).
//
// GB300 mapping.  A CTA sweeps one work item: up to G ordinates of one
// quadrant of one sample, i.e. ordinates that share the upwind order.  Lanes
// run along x: lane g owns the 8 cells [8g, 8g+8) of every row (one aligned
// 32-byte sector of FP32), and the CTA covers the full width with
// ceil(I/8) lanes.  The sweep advances along y in blocks of H rows; lane g
// processes block t - d at step t, where d is its distance in lanes from the
// inflow face, so the x-dependence (the upwind x-flux of H rows x G ordinates)
// passes one lane per step by a warp shuffle (shared memory plus one barrier
// per step between warps).  The y-dependence (8 columns x G ordinates) stays
// in registers across steps.  Each cell is visited once per ordinate group:
// source loads and moment stores are full sectors, and the G ordinates and the
// H x 8 block give the instruction-level parallelism that hides the
// FMA -> MUL -> FMA chain of each cell.  No ordinate or cell values are
// stored: only the moments of each item, which a later kernel sums per sample.
#include "rom_internal.cuh"

namespace romk {
namespace {

constexpr int kH = 4;  // rows per lane per wavefront step

__device__ __forceinline__ void ld8(const float *__restrict__ p, float (&v)[kCols])
{
    const float4 a = __ldg(reinterpret_cast<const float4 *>(p));
    const float4 b = __ldg(reinterpret_cast<const float4 *>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

__device__ __forceinline__ void st8(float *__restrict__ p, const float (&v)[kCols])
{
    reinterpret_cast<float4 *>(p)[0] = make_float4(v[0], v[1], v[2], v[3]);
    reinterpret_cast<float4 *>(p)[1] = make_float4(v[4], v[5], v[6], v[7]);
}

template <int G>
struct OrdRegs {
    float a[G], b[G], w[G], rd[G], c[G], s[G], wc[G], ws[G];
    int ord[G];
};

// Arrays read per cell: MOM source moments, plus sigma_T when it varies.
template <int MOM, bool HOMOG>
struct RowBuf {
    static constexpr int NA = MOM + (HOMOG ? 0 : 1);
    float v[NA][kH][kCols];
};

// Issue the loads of the rows of block `blk` (rows past J are skipped).
template <int MOM, bool HOMOG>
__device__ __forceinline__ void load_block(const SweepArgs &A, int blk, bool yneg, int col0,
                                           const float *__restrict__ src_s, RowBuf<MOM, HOMOG> &b)
{
#pragma unroll
    for (int h = 0; h < kH; ++h) {
        const int jl = blk * kH + h;
        if (jl < A.J) {
            const int j = yneg ? (A.J - 1 - jl) : jl;
            const long long row = (long long)j * A.NXP + col0;
#pragma unroll
            for (int m = 0; m < MOM; ++m) ld8(src_s + m * A.cells + row, b.v[m][h]);
            if (!HOMOG) ld8(A.sigma_t + row, b.v[MOM][h]);
        }
    }
}

// One H x 8 block of cells for all G ordinates of the item, from the rows in b.
template <int G, int MOM, int SCHEME, bool HOMOG, bool XNEG, bool CHECK>
__device__ __forceinline__ void sweep_block(const SweepArgs &A, int blk, bool yneg, int col0,
                                            const OrdRegs<G> &o, float (&py)[kCols][G],
                                            const float (&xin)[kH][G], float (&xo)[kH][G],
                                            const RowBuf<MOM, HOMOG> &b,
                                            float *__restrict__ part_i)
{
#pragma unroll
    for (int h = 0; h < kH; ++h) {
        const int jl = blk * kH + h;
        if (CHECK && jl >= A.J) {
#pragma unroll
            for (int k = 0; k < G; ++k) xo[h][k] = 0.f;
            continue;
        }
        const int j = yneg ? (A.J - 1 - jl) : jl;
        const long long row = (long long)j * A.NXP + col0;
        float x[G];
#pragma unroll
        for (int k = 0; k < G; ++k) x[k] = xin[h][k];
        float p0[kCols], p1[kCols], p2[kCols];
#pragma unroll
        for (int r = 0; r < kCols; ++r) p0[r] = p1[r] = p2[r] = 0.f;
#pragma unroll
        for (int rr = 0; rr < kCols; ++rr) {
            const int r = XNEG ? (kCols - 1 - rr) : rr;
            const bool ok = !CHECK || (col0 + r < A.I);
#pragma unroll
            for (int k = 0; k < G; ++k) {
                float S = b.v[0][h][r];
                if (MOM == 3) S = fmaf(o.c[k], b.v[1][h][r], fmaf(o.s[k], b.v[2][h][r], S));
                const float num = fmaf(o.a[k], x[k], fmaf(o.b[k], py[r][k], S));
                const float rden =
                    HOMOG ? o.rd[k]
                          : __frcp_rn(b.v[RowBuf<MOM, HOMOG>::NA - 1][h][r] + o.a[k] + o.b[k]);
                const float pc = num * rden;
                if (ok) {
                    if (SCHEME == 0) {
                        x[k] = fmaf(2.f, pc, -x[k]);
                        py[r][k] = fmaf(2.f, pc, -py[r][k]);
                    } else {
                        x[k] = pc;
                        py[r][k] = pc;
                    }
                    p0[r] = fmaf(o.w[k], pc, p0[r]);
                    if (MOM == 3) {
                        p1[r] = fmaf(o.wc[k], pc, p1[r]);
                        p2[r] = fmaf(o.ws[k], pc, p2[r]);
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < G; ++k) xo[h][k] = x[k];
        st8(part_i + row, p0);
        if (MOM == 3) {
            st8(part_i + A.cells + row, p1);
            st8(part_i + 2 * A.cells + row, p2);
        }
    }
}

template <int G, int MOM, int SCHEME, bool HOMOG, bool XNEG>
__device__ __forceinline__ void sweep_item(const SweepArgs &A, const SweepItem &it,
                                           const OrdRegs<G> &o)
{
    __shared__ float xbuf[2][kMaxWarps][kH][G];
    const int g = threadIdx.x;
    const int nwarps = blockDim.x >> 5;
    const int L = (A.I + kCols - 1) / kCols;  // lanes that own cells
    const bool lane_on = g < L;
    const int d = XNEG ? (L - 1 - g) : g;     // lanes between this one and the inflow face
    const int col0 = g * kCols;
    const bool yneg = (it.quad >> 1) & 1;
    const int nblk = (A.J + kH - 1) / kH;
    const int T = nblk + L - 1;
    const bool full_cols = col0 + kCols <= A.I;

    // incoming y-edge values of the lane's columns (face y_B, or y_T when s < 0)
    float py[kCols][G];
#pragma unroll
    for (int r = 0; r < kCols; ++r)
#pragma unroll
        for (int k = 0; k < G; ++k) {
            float v = 0.f;
            if (A.inflow && lane_on && col0 + r < A.I && k < it.n)
                v = A.inflow[(long long)o.ord[k] * A.inflow_stride + 2 * A.J + (yneg ? A.I : 0) +
                             col0 + r];
            py[r][k] = v;
        }

    float xin[kH][G];
#pragma unroll
    for (int h = 0; h < kH; ++h)
#pragma unroll
        for (int k = 0; k < G; ++k) xin[h][k] = 0.f;

    const float *src_s = A.src + (long long)it.sample * MOM * A.cells;
    float *part_i = A.part + (long long)blockIdx.x * MOM * A.cells;

    // Rows of the lane's next block are loaded one step ahead (two register
    // buffers used in turn), so their latency overlaps the current block.  With
    // more than two arrays per cell (linear kernel) the registers are not
    // there; the rows are then loaded at the start of their step.
    constexpr bool PF = RowBuf<MOM, HOMOG>::NA <= 2;
    RowBuf<MOM, HOMOG> buf0, buf1;
    auto step = [&](int t, RowBuf<MOM, HOMOG> &cur, RowBuf<MOM, HOMOG> &nxt) {
        const int blk = t - d;
        if (PF && lane_on && blk + 1 >= 0 && blk + 1 < nblk)
            load_block<MOM, HOMOG>(A, blk + 1, yneg, col0, src_s, nxt);
        float xo[kH][G];
        if (lane_on && blk >= 0 && blk < nblk) {
            if (!PF) load_block<MOM, HOMOG>(A, blk, yneg, col0, src_s, cur);
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
                        xin[h][k] = v;
                    }
            }
            if (full_cols && (blk + 1) * kH <= A.J)
                sweep_block<G, MOM, SCHEME, HOMOG, XNEG, false>(A, blk, yneg, col0, o, py, xin, xo,
                                                                 cur, part_i);
            else
                sweep_block<G, MOM, SCHEME, HOMOG, XNEG, true>(A, blk, yneg, col0, o, py, xin, xo,
                                                                cur, part_i);
        } else {
#pragma unroll
            for (int h = 0; h < kH; ++h)
#pragma unroll
                for (int k = 0; k < G; ++k) xo[h][k] = 0.f;
        }
        // hand the outgoing x-edge values to the downstream lane
#pragma unroll
        for (int h = 0; h < kH; ++h)
#pragma unroll
            for (int k = 0; k < G; ++k)
                xin[h][k] = XNEG ? __shfl_down_sync(0xffffffffu, xo[h][k], 1)
                                 : __shfl_up_sync(0xffffffffu, xo[h][k], 1);
        if (nwarps > 1) {
            const int lane = g & 31, w = g >> 5;
            const bool sender = XNEG ? (lane == 0 && w > 0) : (lane == 31 && w + 1 < nwarps);
            if (sender) {
#pragma unroll
                for (int h = 0; h < kH; ++h)
#pragma unroll
                    for (int k = 0; k < G; ++k) xbuf[t & 1][w][h][k] = xo[h][k];
            }
            __syncthreads();
            const bool recv = XNEG ? (lane == 31 && w + 1 < nwarps) : (lane == 0 && w > 0);
            if (recv) {
                const int src_w = XNEG ? w + 1 : w - 1;
#pragma unroll
                for (int h = 0; h < kH; ++h)
#pragma unroll
                    for (int k = 0; k < G; ++k) xin[h][k] = xbuf[t & 1][src_w][h][k];
            }
        }
    };
    if (PF) {
        if (lane_on && d == 0) load_block<MOM, HOMOG>(A, 0, yneg, col0, src_s, buf0);
        int t = 0;
        for (; t + 1 < T; t += 2) {
            step(t, buf0, buf1);
            step(t + 1, buf1, buf0);
        }
        if (t < T) step(t, buf0, buf1);
    } else {
        for (int t = 0; t < T; ++t) step(t, buf0, buf0);
    }
}

template <int G, int MOM, int SCHEME, bool HOMOG>
__global__ void __launch_bounds__(32 * kMaxWarps) sweep2d_kernel(const SweepArgs A)
{
    const SweepItem it = A.items[blockIdx.x];
    if (!A.active[it.sample]) return;
    OrdRegs<G> o;
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
        o.a[k] = f * fabsf(c) * A.inv_dx;
        o.b[k] = f * fabsf(s) * A.inv_dy;
        o.w[k] = w;
        o.rd[k] = HOMOG ? 1.f / (A.sigma_t_homog + o.a[k] + o.b[k]) : 0.f;
        o.c[k] = c;
        o.s[k] = s;
        o.wc[k] = w * c;
        o.ws[k] = w * s;
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
    if (scheme == 0) {
        if (homog) sweep2d_kernel<G, MOM, 0, true><<<grid, block, 0, st>>>(a);
        else sweep2d_kernel<G, MOM, 0, false><<<grid, block, 0, st>>>(a);
    } else {
        if (homog) sweep2d_kernel<G, MOM, 1, true><<<grid, block, 0, st>>>(a);
        else sweep2d_kernel<G, MOM, 1, false><<<grid, block, 0, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sweep2d(const SweepArgs &a, int n_items, int nwarps, int G, int scheme,
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
    return cudaErrorInvalidValue;
}

}  // namespace romk
