// reduce.cu -- scattering-source update, source-iteration residual and sample
// average (K2, K5, K6) plus small data-movement kernels.
//
// combine:  phi_s = the moments the work items of sample s added to its
//           accumulator during the sweep (read and cleared), the new source moments
//             isotropic: S = sigma_S phi + q                       (P = 1)
//             linear:    S0 = sigma_S phi + q, S1 = g sigma_S (Jx, Jy)
//           so that the next sweep forms S_l = S0 + c_l S1x + s_l S1y
//           (eq. equ_random with eq. anisotropic kernel, mirror-averaged in
//           zeta, where sum_l' w_l' (1 + g u_l'.u_l) psi_l' = phi + g (c Jx + s Jy)),
//           and per-block FP64 partial sums of |phi^k - phi^{k-1}|^2 and |phi^k|^2
//           (and, in the X-Y moment modes, of sigma_T phi^k and of the previous
//           iterate's source moments, for the particle balance), and min phi.
//           Summation precision: each thread sums its few cells (8 to 32) in
//           FP32, the 32 lanes of a warp add by an FP32 tree (5 levels), and from
//           the warp sums on everything is FP64 (across warps, blocks and in the
//           finalize).  A term passes through at most ~37 FP32 additions, so the
//           relative error of each block partial is below ~37 * 2^-24 = 2.2e-6
//           in the worst case (random rounding: ~sqrt(37) * 2^-24 = 3.6e-7); the
//           relative residual sqrt(d2 / n2) then carries about half of that,
//           well below the tolerances of 1e-6 and above that FP32 sweeps reach.
//           The FP64 units of GB300 are few: a per-thread FP64 sum (or an FP64
//           warp tree) in every combine block costs more than the FP32 work.
// finalize: relative l2 change per sample (Sec. 3.2 source iteration stopping
//           rule of this library), sweep counters, the active flags, and the
//           number of samples still iterating (optionally the condition of the
//           device-side loop of a CUDA graph).
// average:  phi_bar = (1/t) sum_s phi^{xi_s} in FP64 (Sec. 4.1).
#include <math.h>

#include <algorithm>

#include "rom_internal.cuh"

namespace romk {
namespace {

// The block's contribution to its sample's sums: six FP32 per-thread sums
// (squared change, squared norm, sigma_T phi, three source moments) and a min,
// reduced by an FP32 warp tree, then in FP64 across the warps, and added to the
// sample's FP64 sums with one atomic per value (the min by an atomic min on the
// ordered-int key).  Every thread of the block calls it.
__device__ __forceinline__ void block_partials(float (&v)[6], float mn, double *sums, int *minkey)
{
    __shared__ double red[6][32];
    __shared__ float redm[32];
#pragma unroll
    for (int k = 0; k < 6; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < 6; ++k) red[k][w] = (double)v[k];
        redm[w] = mn;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        double acc = 0.0;
        for (int k = 0; k < nw; ++k) acc += red[threadIdx.x][k];
        if (acc != 0.0) atomicAdd(sums + threadIdx.x, acc);
    } else if (threadIdx.x == 6) {
        float m = redm[0];
        for (int k = 1; k < nw; ++k) m = fminf(m, redm[k]);
        if (m < INFINITY) atomicMin(minkey, float_order_key(m));
    }
}

template <int MOM>
__global__ void __launch_bounds__(256) combine_kernel(const CombineArgs A0)
{
    const int s = blockIdx.y;
    if (!A0.active[s]) return;
    CombineArgs A = A0;
    long long base = (long long)s * MOM * A0.cells;  // the sample's [MOM][cells] block
    if (A0.grids) {  // several grids: the sample's own grid and coefficient block
        const GridDesc g = A0.grids[A0.sgrid[s]];
        A.cells = g.cells;
        A.I = g.I;
        A.NXP = g.NXP;
        A.sigma_s = A0.sigma_s + g.off;
        A.q = A0.q + g.off;
        if (A0.sigma_t) A.sigma_t = A0.sigma_t + g.off;
        base = A0.soff[s];
    }
    const long long cells = A.cells;  // a multiple of 8: a thread takes whole 32-byte sectors
    float *phi = A.phi + base;
    float *src = A.src + base;
    float d2f = 0.f, n2f = 0.f, mn = INFINITY, a1f = 0.f, b0f = 0.f, b1f = 0.f, b2f = 0.f;
    // KS sectors per thread and pass, all loaded before any store (the loads and
    // stores are ordered volatile accesses): KS times the bytes in flight per thread
    constexpr int KS = MOM == 1 ? 2 : 1;
    const long long stride = 8LL * gridDim.x * blockDim.x;
    for (long long v0 = 8 * ((long long)blockIdx.x * blockDim.x + threadIdx.x); v0 < cells;
         v0 += KS * stride) {
        float acc[KS][MOM][8], old[KS][MOM][8], ss[KS][8], qq[KS][8], st[KS][8];
#pragma unroll
        for (int k = 0; k < KS; ++k) {
            const long long v = v0 + k * stride;
            if (v >= cells) continue;
            ld8_volatile(phi + v, old[k][0]);
            if (MOM == 3 && A.balance) {
                ld8_volatile(phi + cells + v, old[k][MOM == 3 ? 1 : 0]);
                ld8_volatile(phi + 2 * cells + v, old[k][MOM == 3 ? 2 : 0]);
            }
#pragma unroll
            for (int m = 0; m < MOM; ++m) ld8_volatile(A.acc + base + m * cells + v, acc[k][m]);
            ldg8(A.sigma_s + v, ss[k]);
            ldg8(A.q + v, qq[k]);
            if (A.balance && A.sigma_t) ldg8(A.sigma_t + v, st[k]);
        }
#pragma unroll
        for (int k = 0; k < KS; ++k) {
            const long long v = v0 + k * stride;
            if (v >= cells) continue;
            if (A.balance) {
                // the source moments of the previous iterate (the sweep's input) and
                // sigma_T phi of the new one, for the particle balance; padding
                // columns hold phi = 0 and sigma_S = q = 0
#pragma unroll
                for (int e = 0; e < 8; ++e) b0f += fmaf(ss[k][e], old[k][0][e], qq[k][e]);
                if (MOM == 3) {
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        b1f = fmaf(A.g * ss[k][e], old[k][MOM == 3 ? 1 : 0][e], b1f);
                        b2f = fmaf(A.g * ss[k][e], old[k][MOM == 3 ? 2 : 0][e], b2f);
                    }
                }
                if (!A.sigma_t)
#pragma unroll
                    for (int e = 0; e < 8; ++e) st[k][e] = A.sigma_t_homog;
            }
            // per-element squares in FP32 (a few terms per thread), norms in FP64 below
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const float dd = acc[k][0][e] - old[k][0][e];
                d2f = fmaf(dd, dd, d2f);
                n2f = fmaf(acc[k][0][e], acc[k][0][e], n2f);
                if (A.balance) a1f = fmaf(st[k][e], acc[k][0][e], a1f);  // sigma_T phi
                // padding columns (x >= I) hold phi = 0 and would hide a negative min
                if ((v % A.NXP) + e < A.I) mn = fminf(mn, acc[k][0][e]);
            }
            // the accumulated moments cleared for the next sweep; phi and the next
            // source moments written
            float zero[8], out[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) zero[e] = 0.f;
#pragma unroll
            for (int m = 0; m < MOM; ++m) {
                stg8(A.acc + base + m * cells + v, zero);
                stg8(phi + m * cells + v, acc[k][m]);
            }
#pragma unroll
            for (int e = 0; e < 8; ++e) out[e] = fmaf(ss[k][e], acc[k][0][e], qq[k][e]);
            stg8(src + v, out);
            if (MOM == 3) {
#pragma unroll
                for (int m = 1; m < 3; ++m) {
#pragma unroll
                    for (int e = 0; e < 8; ++e) out[e] = A.g * ss[k][e] * acc[k][m][e];
                    stg8(src + m * cells + v, out);
                }
            }
        }
    }
    float v6[6] = {d2f, n2f, a1f, b0f, b1f, b2f};
    block_partials(v6, mn, A.sums + (long long)s * kNP, A.minkey + s);
}

// 3D: phi of each sample from its two diagonal-storage accumulators (read and
// cleared), the residual partials against the previous phi, and the next
// source sigma_S phi + q in both diagonal families.  phi, sigma_S and q are kept
// in family-0 storage too, and the threads walk that storage in order (one
// 8-cell sector each, padding sectors skipped), so that only the family-1
// accumulator and source are visited out of order.
__global__ void __launch_bounds__(256) combine3_kernel(const Combine3Args A)
{
    const int s = blockIdx.y;
    if (!A.active[s]) return;
    const Skew3 g = A.sk;
    const int n_sec = (int)(g.cells / 8);
    float *acc0 = A.acc + (long long)s * g.cells;
    float *acc1 = A.acc + ((long long)A.S + s) * g.cells;
    float *src0 = A.src + (long long)s * g.cells;
    float *src1 = A.src + ((long long)A.S + s) * g.cells;
    float *phi = A.phi + (long long)s * g.cells;
    float d2f = 0.f, n2f = 0.f, mn = INFINITY;
    for (int sec = blockIdx.x * blockDim.x + threadIdx.x; sec < n_sec;
         sec += gridDim.x * blockDim.x) {
        // sec = ((diag * L + strip) * 4 + hh) * NBg + jb
        int t = sec / g.NBg;
        const int jb = sec - t * g.NBg;
        const int hh = t & 3;
        t >>= 2;
        const int diag = t / g.L, strip = t - diag * g.L;
        const int k = diag - jb, j = 4 * jb + hh;
        if (k < 0 || k >= g.K || j >= g.J) continue;
        const long long i0 = (long long)sec * 8, i1 = skew3_index(g, 1, k, j, strip);
        float a0[8], a1[8], old[8], ss[8], qq[8], now[8], out[8], zero[8];
        ld8_volatile(acc0 + i0, a0);
        ld8_volatile(acc1 + i1, a1);
        ld8_volatile(phi + i0, old);
        ldg8(A.sigma_s + i0, ss);
        ldg8(A.q + i0, qq);
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            zero[e] = 0.f;
            now[e] = a0[e] + a1[e];
            const float dd = now[e] - old[e];
            d2f = fmaf(dd, dd, d2f);
            n2f = fmaf(now[e], now[e], n2f);
            if (strip * 8 + e < A.I) mn = fminf(mn, now[e]);
            out[e] = fmaf(ss[e], now[e], qq[e]);
        }
        stg8(acc0 + i0, zero);
        stg8(acc1 + i1, zero);
        stg8(phi + i0, now);
        stg8(src0 + i0, out);
        stg8(src1 + i1, out);
    }
    float v6[6] = {d2f, n2f, 0.f, 0.f, 0.f, 0.f};
    block_partials(v6, mn, A.sums + (long long)s * kNP, A.minkey + s);
}

// 3D average / extraction from family-0 diagonal storage [S][sk.cells] into [K][J][I]
__global__ void average3_kernel(const float *phi, int S, Skew3 g, int I, double *avg, double *sum)
{
    const long long n = (long long)I * g.J * g.K;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        const long long row = v / I;
        const int i = (int)(v - row * I);
        const int k = (int)(row / g.J), j = (int)(row - (long long)k * g.J);
        const long long o = skew3_index(g, 0, k, j, i >> 3) + (i & 7);
        double acc = 0.0;
        for (int s = 0; s < S; ++s) acc += (double)phi[(long long)s * g.cells + o];
        if (sum) sum[v] = acc;
        if (avg) avg[v] = S > 0 ? acc / S : 0.0;
    }
}
__global__ void extract3_kernel(const float *phi, int sample, Skew3 g, int I, double *out)
{
    const long long n = (long long)I * g.J * g.K;
    const float *p = phi + (long long)sample * g.cells;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        const long long row = v / I;
        const int i = (int)(v - row * I);
        const int k = (int)(row / g.J), j = (int)(row - (long long)k * g.J);
        out[v] = (double)p[skew3_index(g, 0, k, j, i >> 3) + (i & 7)];
    }
}

// dst[f][copy][sk.cells] = in[K][J][NXP] in diagonal family f < n_fam, for every copy
__global__ void skew3_scatter_kernel(const float *in, Skew3 g, int NXP, int n_fam, int n_copies,
                                     float *dst)
{
    const long long n_sec = (long long)g.K * g.J * g.L;
    for (long long sec = (long long)blockIdx.x * blockDim.x + threadIdx.x; sec < n_sec;
         sec += (long long)gridDim.x * blockDim.x) {
        const long long row = sec / g.L;
        const int strip = (int)(sec - row * g.L);
        const int k = (int)(row / g.J), j = (int)(row - (long long)k * g.J);
        float v[8];
        ldg8(in + row * NXP + strip * 8, v);
        for (int f = 0; f < n_fam; ++f) {
            const long long i = skew3_index(g, f, k, j, strip);
            for (int c = 0; c < n_copies; ++c)
                stg8(dst + ((long long)f * n_copies + c) * g.cells + i, v);
        }
    }
}

__global__ void __launch_bounds__(256) finalize_kernel(const FinalizeArgs A)
{
    int cnt = 0;
    for (int s = threadIdx.x; s < A.S; s += blockDim.x) {
        if (!A.active[s]) continue;
        // the sums the combine blocks added, cleared for the next sweep
        double *sm = A.sums + (long long)s * kNP;
        const double d2 = sm[0], n2 = sm[1], a1 = sm[2], b0 = sm[3], b1 = sm[4], b2 = sm[5];
#pragma unroll
        for (int k = 0; k < kNP; ++k) sm[k] = 0.0;
        const int mk = A.minkey[s];
        A.minkey[s] = 0x7FFFFFFF;
        const double mn = mk == 0x7FFFFFFF ? (double)NAN : (double)float_from_order_key(mk);
        const double r = n2 > 0.0 ? sqrt(d2 / n2) : (d2 == 0.0 ? 0.0 : (double)INFINITY);
        const int it = A.iters[s] + 1;
        A.iters[s] = it;
        A.resid[s] = r;
        const bool bad = !isfinite(r);
        // divergence: the change ||phi^k - phi^{k-1}|| itself grows sweep after
        // sweep (for a contracting iteration it shrinks by the spectral radius)
        const double dn = sqrt(d2);
        const int gr = (dn > A.dprev[s] && !(r < A.tol)) ? A.grow[s] + 1 : 0;
        A.grow[s] = gr;
        A.dprev[s] = dn;
        const bool growing = A.diverge_window > 0 && gr >= A.diverge_window;
        if (bad) A.flags[s] |= 1;
        if (growing) A.flags[s] |= 2;
        A.phimin_out[s] = mn;
        if (A.balance) {
            // leakage + sum sigma_T phi^k dA = sum_l w_l sum S_l^{k-1} dA, exact for
            // the cell equations of the sweep up to its rounding
            const double lk = A.leak[s];
            A.leak[s] = 0.0;
            const double *os = A.ordsum + 3LL * s;
            const double dA = A.sdA ? A.sdA[s] : A.dA;
            const double rhs = dA * (os[0] * b0 + os[1] * b1 + os[2] * b2);
            const double rem = dA * a1;
            const double den = fabs(lk) + fabs(rem) + fabs(rhs);
            A.bal_out[s] = den > 0.0 ? fabs(lk + rem - rhs) / den : 0.0;
            A.leak_out[s] = lk;
        }
        bool stop;
        if (A.fixed_iters > 0) stop = it >= A.fixed_iters;
        else stop = (r < A.tol) || it >= A.max_iter || bad || growing;
        if (stop) A.active[s] = 0;
        else ++cnt;
    }
    __shared__ int red[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
        *A.n_active = tot;
        if (A.use_cond) cudaGraphSetConditional(A.cond, tot > 0 ? 1u : 0u);
    }
}

__global__ void init_checks_kernel(int S, double *dprev, int *grow, double *leak, double *bal,
                                   double *leak_out, double *phimin, double *sums, int *minkey)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    dprev[s] = (double)INFINITY;
    grow[s] = 0;
    leak[s] = 0.0;
    bal[s] = (double)NAN;
    leak_out[s] = (double)NAN;
    phimin[s] = (double)NAN;
#pragma unroll
    for (int k = 0; k < kNP; ++k) sums[(long long)s * kNP + k] = 0.0;
    minkey[s] = 0x7FFFFFFF;
}

__global__ void ordsum_kernel(const double *c, const double *s, const double *w,
                              const long long *ord_off, const int *M, int S, double *out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= S) return;
    double sw = 0.0, swc = 0.0, sws = 0.0;
    for (long long o = ord_off[k]; o < ord_off[k] + M[k]; ++o) {
        sw += w[o];
        swc += w[o] * c[o];
        sws += w[o] * s[o];
    }
    out[3 * k] = sw;
    out[3 * k + 1] = swc;
    out[3 * k + 2] = sws;
}

__global__ void init_state_kernel(int S, int MOM, long long cells, const float *q, float *phi,
                                  float *src, int *active, int *iters, int *flags, double *resid)
{
    const long long n = (long long)S * MOM * cells;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        const long long cell = v % cells;
        const int m = (int)((v / cells) % MOM);
        phi[v] = 0.f;
        if (src) src[v] = m == 0 ? q[cell] : 0.f;  // psi^0 = 0: the first source is q
    }
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < S) {
        active[t] = 1;
        iters[t] = 0;
        flags[t] = 0;
        resid[t] = (double)INFINITY;
    }
}

// several grids: phi = 0 and the first source q (psi^0 = 0) for each sample on its grid
__global__ void init_grids_kernel(int MOM, const GridDesc *grids, const int *sgrid,
                                  const long long *soff, const float *q, float *phi, float *src)
{
    const int s = blockIdx.y;
    const GridDesc g = grids[sgrid[s]];
    const long long n = (long long)MOM * g.cells;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        const long long cell = v % g.cells;
        phi[soff[s] + v] = 0.f;
        src[soff[s] + v] = v < g.cells ? q[g.off + cell] : 0.f;
    }
}

__global__ void average_kernel(const float *phi, int S, int MOM, int I, int J, int NXP,
                               double *avg, double *sum)
{
    const long long cells = (long long)J * NXP;
    const long long n = (long long)I * J;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        const long long j = v / I, i = v - j * I;
        double acc = 0.0;
        for (int s = 0; s < S; ++s) acc += (double)phi[(long long)s * MOM * cells + j * NXP + i];
        if (sum) sum[v] = acc;
        if (avg) avg[v] = S > 0 ? acc / S : 0.0;
    }
}

__global__ void extract_kernel(const float *phi, int sample, int MOM, int I, int J, int NXP,
                               double *out)
{
    const long long cells = (long long)J * NXP;
    const long long n = (long long)I * J;
    const float *p = phi + (long long)sample * MOM * cells;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        const long long j = v / I, i = v - j * I;
        out[v] = (double)p[j * NXP + i];
    }
}

// Copy [J][I] device inputs into the padded [J][NXP] layout and check the
// hypotheses 0 <= sigma_S < sigma_T, q >= 0 (all finite).
__global__ void pad_grid_kernel(const float *st_in, const float *ss_in, const float *q_in, int I,
                                int J, int NXP, float *st_out, float *ss_out, float *q_out,
                                unsigned int *stats)
{
    const long long n = (long long)J * NXP;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        const long long j = v / NXP, i = v - j * NXP;
        if (i < I) {
            const float a = st_in[j * I + i], b = ss_in[j * I + i], c = q_in[j * I + i];
            st_out[v] = a;
            ss_out[v] = b;
            q_out[v] = c;
            const bool ok = isfinite(a) && isfinite(b) && isfinite(c) && b >= 0.f && b < a &&
                            c >= 0.f;
            if (!ok) atomicAdd(&stats[2], 1u);
            else {  // a > 0 here, so its bit pattern orders like its value
                atomicMin(&stats[0], __float_as_uint(a));
                atomicMax(&stats[1], __float_as_uint(a));
            }
        } else {
            st_out[v] = 1.f;  // padding columns are never swept
            ss_out[v] = 0.f;
            q_out[v] = 0.f;
        }
    }
}

int blocks_for(long long n, int threads)
{
    long long b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 4096) b = 4096;
    return (int)b;
}

}  // namespace

cudaError_t launch_combine(const CombineArgs &a, cudaStream_t st)
{
    // need = passes of a 256-thread block taking KS sectors per thread (combine_kernel);
    // at most a.chunks blocks per sample unless that takes more than 4 passes per thread
    // (large, HBM-bound batches stream better with more blocks), and each thread making
    // the same number of passes (an uneven last pass measured up to 30% slower on the
    // L2-resident point source: 14.4 us per launch at 4 or 8 blocks per sample, 16.9-18.6
    // at 3, 5, 6 or 16)
    const long long ks = a.MOM == 1 ? 2 : 1;
    const long long need = (a.cells / 8 + 256 * ks - 1) / (256 * ks);
    const long long passes =
        std::min(4LL, (need + std::max(1, a.chunks) - 1) / std::max(1, a.chunks));
    const long long blocks = (need + passes - 1) / passes;
    const dim3 grid((unsigned)std::max(1LL, blocks), a.S), block(256);
    if (a.MOM == 1) combine_kernel<1><<<grid, block, 0, st>>>(a);
    else if (a.MOM == 3) combine_kernel<3><<<grid, block, 0, st>>>(a);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_combine3(const Combine3Args &a, cudaStream_t st)
{
    const dim3 grid(a.chunks, a.S), block(256);
    combine3_kernel<<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_average3(const float *phi, int S, const Skew3 &sk, int I, double *avg,
                            double *sum, cudaStream_t st)
{
    average3_kernel<<<blocks_for((long long)I * sk.J * sk.K, 256), 256, 0, st>>>(phi, S, sk, I,
                                                                                 avg, sum);
    return cudaGetLastError();
}

cudaError_t launch_extract3(const float *phi, int sample, const Skew3 &sk, int I, double *out,
                            cudaStream_t st)
{
    extract3_kernel<<<blocks_for((long long)I * sk.J * sk.K, 256), 256, 0, st>>>(phi, sample, sk,
                                                                                 I, out);
    return cudaGetLastError();
}

cudaError_t launch_skew3_scatter(const float *in, const Skew3 &sk, int NXP, int n_fam,
                                 int n_copies, float *dst, cudaStream_t st)
{
    const long long n_sec = (long long)sk.K * sk.J * sk.L;
    long long b = (n_sec + 255) / 256;
    if (b > 4096) b = 4096;
    if (b < 1) b = 1;
    skew3_scatter_kernel<<<(unsigned)b, 256, 0, st>>>(in, sk, NXP, n_fam, n_copies, dst);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const FinalizeArgs &a, cudaStream_t st)
{
    finalize_kernel<<<1, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_init_state(int S, int MOM, long long cells, const float *q, float *phi,
                              float *src, int *active, int *iters, int *flags, double *resid,
                              cudaStream_t st)
{
    long long n = (long long)S * MOM * cells;
    if (n < S) n = S;
    int b = blocks_for(n, 256);
    if ((long long)b * 256 < S) b = (S + 255) / 256;
    init_state_kernel<<<b, 256, 0, st>>>(S, MOM, cells, q, phi, src, active, iters, flags, resid);
    return cudaGetLastError();
}

cudaError_t launch_init_grids(int S, int MOM, const GridDesc *grids, const int *sgrid,
                              const long long *soff, int max_cells, const float *q, float *phi,
                              float *src, cudaStream_t st)
{
    const dim3 grid(blocks_for((long long)MOM * max_cells, 256), S);
    init_grids_kernel<<<grid, 256, 0, st>>>(MOM, grids, sgrid, soff, q, phi, src);
    return cudaGetLastError();
}

cudaError_t launch_average(const float *phi, int S, int MOM, int I, int J, int NXP, double *avg,
                           double *sum, cudaStream_t st)
{
    average_kernel<<<blocks_for((long long)I * J, 256), 256, 0, st>>>(phi, S, MOM, I, J, NXP, avg,
                                                                       sum);
    return cudaGetLastError();
}

cudaError_t launch_extract(const float *phi, int sample, int MOM, int I, int J, int NXP,
                           double *out, cudaStream_t st)
{
    extract_kernel<<<blocks_for((long long)I * J, 256), 256, 0, st>>>(phi, sample, MOM, I, J, NXP,
                                                                       out);
    return cudaGetLastError();
}

cudaError_t launch_pad_grid(const float *st_in, const float *ss_in, const float *q_in, int I,
                            int J, int NXP, float *st_out, float *ss_out, float *q_out,
                            unsigned int *stats, cudaStream_t st)
{
    pad_grid_kernel<<<blocks_for((long long)J * NXP, 256), 256, 0, st>>>(
        st_in, ss_in, q_in, I, J, NXP, st_out, ss_out, q_out, stats);
    return cudaGetLastError();
}

cudaError_t launch_ordsum(const double *c, const double *s, const double *w,
                          const long long *ord_off, const int *M, int S, double *out,
                          cudaStream_t st)
{
    ordsum_kernel<<<(S + 127) / 128, 128, 0, st>>>(c, s, w, ord_off, M, S, out);
    return cudaGetLastError();
}

cudaError_t launch_init_checks(int S, double *dprev, int *grow, double *leak, double *bal,
                               double *leak_out, double *phimin, double *sums, int *minkey,
                               cudaStream_t st)
{
    init_checks_kernel<<<(S + 255) / 256, 256, 0, st>>>(S, dprev, grow, leak, bal, leak_out,
                                                        phimin, sums, minkey);
    return cudaGetLastError();
}

}  // namespace romk
