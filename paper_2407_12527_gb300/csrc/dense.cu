// dense.cu -- the dense scattering source (K3, K4) for kernels that are not
// closed by a few angular moments (Henyey-Greenstein, or any kernel on demand).
//
// With the weights and the discrete kernel of eq. (wl),
//   S_l(z) = sigma_S(z) sum_l' A[l][l'] psi_l'(z) + q(z),   A[l][l'] = w_l' P(u_l', u_l),
// (eq. equ_random), optionally with each row of A divided by its sum (Remark,
// Sec. 3.1).  P(u', u) = G(u' . u) with G the linear kernel 1 + g mu (eq.
// anisotropic kernel) or Henyey-Greenstein (1 - g^2) / (1 + g^2 - 2 g mu)^{3/2};
// X-Y ordinates lie on the upper hemisphere and, unless the raw form is asked
// for, P is the mirror average 1/2 [G(cc' + ss' + zz') + G(cc' + ss' - zz')].
//
// K3 (pmat_kernel) builds A per sample in FP64 and rounds it to FP32, once per
// solve.  K4 (dense_source_kernel) is, per sample, the product of the M x M
// matrix A with the M x cells matrix of cell values psi, an FP32 SIMT GEMM
// (128 x 128 output tile per CTA, 8 x 8 per thread, double-buffered shared
// memory), with the sigma_S / q epilogue fused.
#include <math.h>

#include "rom_internal.cuh"

namespace romk {
namespace {

__device__ __forceinline__ double phase(int kind, double g, double mu)
{
    if (kind == 1) return 1.0 + g * mu;  // linear
    if (kind == 2) {                     // Henyey-Greenstein
        const double x = 1.0 + g * g - 2.0 * g * mu;
        return (1.0 - g * g) / (x * sqrt(x));
    }
    return 1.0;  // isotropic
}

__device__ __forceinline__ double kernel_P(const PmatArgs &a, long long lp, long long l)
{
    const double inplane = a.c[lp] * a.c[l] + a.s[lp] * a.s[l];
    const double zz = a.z[lp] * a.z[l];
    if (a.raw) return phase(a.kind, a.g, inplane + zz);
    return 0.5 * (phase(a.kind, a.g, inplane + zz) + phase(a.kind, a.g, inplane - zz));
}

// One block per row l of one sample: A[l][l'] = w_l' P(u_l', u_l) (/ row sum).
__global__ void __launch_bounds__(256) pmat_kernel(const PmatArgs a)
{
    const int s = blockIdx.y, l = blockIdx.x;
    const int M = a.M[s];
    if (l >= M) return;
    const long long o = a.ord_off[s];
    double sum = 0.0;
    for (int lp = threadIdx.x; lp < M; lp += blockDim.x) sum += a.w[o + lp] * kernel_P(a, o + lp, o + l);
    __shared__ double red[32];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, d);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
    __syncthreads();
    double tot = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
    const double scale = a.normalize ? 1.0 / tot : 1.0;
    float *row = a.A + a.a_off[s] + (long long)l * M;
    for (int lp = threadIdx.x; lp < M; lp += blockDim.x)
        row[lp] = (float)(a.w[o + lp] * kernel_P(a, o + lp, o + l) * scale);
}

constexpr int BM = 128, BN = 128, BK = 8;

__global__ void __launch_bounds__(256) dense_source_kernel(const DenseArgs a)
{
    const int s = blockIdx.z;
    if (!a.active[s]) return;
    const int M = a.M[s];
    const int m0 = blockIdx.y * BM;
    if (m0 >= M) return;
    const long long n0 = (long long)blockIdx.x * BN;
    const long long cells = a.cells;
    const long long o = a.ord_off[s];
    const float *A = a.A + a.a_off[s];
    const float *B = a.psi + o * cells;

    __shared__ __align__(16) float As[2][BK][BM];
    __shared__ __align__(16) float Bs[2][BK][BN];
    const int t = threadIdx.x;
    const int tx = t & 15, ty = t >> 4;
    // loader coordinates: A tile (BM x BK) as 4 consecutive k of one row; B tile
    // (BK x BN) as one float4 of one row
    const int ai = t >> 1, ak = (t & 1) * 4;
    const int bk = t >> 5, bj = (t & 31) * 4;

    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    float ra[4];
    float4 rb;
    auto gload = [&](int k0) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int m = m0 + ai, k = k0 + ak + e;
            ra[e] = (m < M && k < M) ? A[(long long)m * M + k] : 0.f;
        }
        const int k = k0 + bk;
        const long long n = n0 + bj;
        rb = (k < M && n < cells) ? *reinterpret_cast<const float4 *>(B + (long long)k * cells + n)
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
    };
    auto sstore = [&](int buf) {
#pragma unroll
        for (int e = 0; e < 4; ++e) As[buf][ak + e][ai] = ra[e];
        *reinterpret_cast<float4 *>(&Bs[buf][bk][bj]) = rb;
    };

    gload(0);
    sstore(0);
    __syncthreads();
    int buf = 0;
    for (int k0 = 0; k0 < M; k0 += BK) {
        const bool more = k0 + BK < M;
        if (more) gload(k0 + BK);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][kk][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][kk][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][64 + tx * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        if (more) {
            sstore(buf ^ 1);
            __syncthreads();
            buf ^= 1;
        }
    }

    // epilogue: S = sigma_S * (A psi) + q
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        const long long n = n0 + half * 64 + tx * 4;
        if (n >= cells) continue;
        const float4 ss = *reinterpret_cast<const float4 *>(a.sigma_s + n);
        const float4 qq = *reinterpret_cast<const float4 *>(a.q + n);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
            if (m >= M) continue;
            *reinterpret_cast<float4 *>(a.src + (o + m) * cells + n) =
                make_float4(fmaf(ss.x, acc[i][half * 4 + 0], qq.x),
                            fmaf(ss.y, acc[i][half * 4 + 1], qq.y),
                            fmaf(ss.z, acc[i][half * 4 + 2], qq.z),
                            fmaf(ss.w, acc[i][half * 4 + 3], qq.w));
        }
    }
}

// src[o][cell] = q[cell] for every ordinate (psi^0 = 0).
__global__ void dense_init_kernel(const float *q, long long cells, long long m_total, float *src)
{
    const long long n4 = cells / 4 * m_total;
    const float4 *q4 = reinterpret_cast<const float4 *>(q);
    float4 *s4 = reinterpret_cast<float4 *>(src);
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n4;
         v += (long long)gridDim.x * blockDim.x)
        s4[v] = q4[v % (cells / 4)];
}

}  // namespace

cudaError_t launch_pmat(const PmatArgs &a, int max_m, cudaStream_t st)
{
    if (a.S <= 0 || max_m <= 0) return cudaSuccess;
    pmat_kernel<<<dim3(max_m, a.S), 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_dense_source(const DenseArgs &a, int max_m, cudaStream_t st)
{
    if (a.S <= 0 || max_m <= 0) return cudaSuccess;
    const dim3 grid((unsigned)((a.cells + BN - 1) / BN), (unsigned)((max_m + BM - 1) / BM), a.S);
    dense_source_kernel<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_dense_init(const float *q, long long cells, long long m_total, float *src,
                              cudaStream_t st)
{
    const long long n4 = cells / 4 * m_total;
    long long b = (n4 + 255) / 256;
    if (b > 8192) b = 8192;
    if (b < 1) b = 1;
    dense_init_kernel<<<(unsigned)b, 256, 0, st>>>(q, cells, m_total, src);
    return cudaGetLastError();
}

}  // namespace romk
