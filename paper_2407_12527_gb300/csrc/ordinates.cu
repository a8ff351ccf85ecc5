// ordinates.cu -- ordinate sets (step a1 of the hot path).
//
// Device: the random ordinate sets of Sec. 3.1 / Sec. 4.2 (K7).  For sample s
// the first quadrant of the (zeta, theta) rectangle [0,1] x [0, pi/2] is split
// into n_zeta x n_theta equal cells (zeta nodes (n_zeta - i + 1)/n_zeta,
// theta nodes (j - 1) pi / (2 n_theta)); one point is drawn uniformly in each
// cell, (c, s) = sqrt(1 - zeta^2)(cos theta, sin theta), and the other three
// quadrants follow from the reflections of eq. (2Dordinates_symmetry), which
// for (c, s) are the sign changes (-c, s), (-c, -s), (c, -s).  Weights are
// |S_l| / |S| = 1 / (4 n_zeta n_theta) (eq. wl).  3D sets add the mirror image
// (c, s, -zeta) of each of those 4 m points (the lower hemisphere), weights
// 1 / (8 n_zeta n_theta).  The uniform numbers come from
// SplitMix64 (Steele, Lea & Flood 2014): the n-th output of seed k is
// mix(k + (n + 1) * 0x9E3779B97F4A7C15), its top 53 bits scaled by 2^-53.
//
// Host: the deterministic sets of Appendix A (2D uniform, eq. uniform2D; 2D
// Gaussian), and a product Gauss-Legendre set, with Legendre roots found by
// Newton's method on the three-term recurrence.
#include <math.h>

#include <vector>

#include "rom_internal.cuh"

namespace romk {
namespace {

__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed,
                                                            unsigned long long n)
{
    unsigned long long z = seed + (n + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double u01(unsigned long long seed, unsigned long long n)
{
    return (double)(splitmix64_at(seed, n) >> 11) * 0x1.0p-53;
}

__global__ void ordgen_kernel(const OrdGenArgs A)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= A.total_cells) return;
    int lo = 0, hi = A.n_samples;  // first_cell[lo] <= tid < first_cell[lo + 1]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (A.first_cell[mid] <= tid) lo = mid;
        else hi = mid;
    }
    const int s = lo;
    const int l0 = tid - A.first_cell[s];
    const int nz = A.nz[s], nt = A.nt[s], m = nz * nt;
    const int i = l0 / nt + 1, j = l0 % nt + 1;  // cell (i, j), 1-based
    const unsigned long long ctr =
        ((unsigned long long)(unsigned)(A.first_sample + s) << 32) | ((unsigned long long)l0 << 1);
    const double uz = u01(A.seed, ctr), ut = u01(A.seed, ctr | 1ull);
    const double pi = 3.14159265358979323846;
    const double z_lo = (double)(nz - i) / nz, z_hi = (double)(nz - i + 1) / nz;
    const double t_lo = (double)(j - 1) * pi / (2.0 * nt), t_hi = (double)j * pi / (2.0 * nt);
    const double zeta = z_lo + uz * (z_hi - z_lo);
    const double theta = t_lo + ut * (t_hi - t_lo);
    const double rho = sqrt(1.0 - zeta * zeta);
    double sn, cs;
    sincos(theta, &sn, &cs);
    const double c = rho * cs, sv = rho * sn, w = 1.0 / ((A.octants ? 8.0 : 4.0) * m);
    const long long base = A.ord_off[s] + l0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        if (q >= 4 && !A.octants) break;
        const double cq = (q == 1 || q == 2 || q == 5 || q == 6) ? -c : c;
        const double sq = ((q & 3) >= 2) ? -sv : sv;
        const double zq = q >= 4 ? -zeta : zeta;  // 3D: the mirror image in zeta
        const long long o = base + (long long)q * m;
        A.c64[o] = cq;
        A.s64[o] = sq;
        A.z64[o] = zq;
        A.w64[o] = w;
        A.c32[o] = (float)cq;
        A.s32[o] = (float)sq;
        A.z32[o] = (float)zq;
        A.w32[o] = (float)w;
    }
}

// Positive roots (descending) of the Legendre polynomial P_n and P_n' there.
void legendre_pos_roots(int n, std::vector<double> &x, std::vector<double> &dp)
{
    x.clear();
    dp.clear();
    const double pi = 3.14159265358979323846;
    for (int k = 1; k <= n / 2; ++k) {
        double r = cos(pi * (k - 0.25) / (n + 0.5));
        double d = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = r;
            for (int l = 1; l < n; ++l) {
                const double p2 = ((2.0 * l + 1.0) * r * p1 - l * p0) / (l + 1.0);
                p0 = p1;
                p1 = p2;
            }
            d = n * (r * p1 - p0) / (r * r - 1.0);
            const double step = p1 / d;
            r -= step;
            if (fabs(step) < 1e-16) break;
        }
        double p0 = 1.0, p1 = r;  // derivative at the converged root
        for (int l = 1; l < n; ++l) {
            const double p2 = ((2.0 * l + 1.0) * r * p1 - l * p0) / (l + 1.0);
            p0 = p1;
            p1 = p2;
        }
        d = n * (r * p1 - p0) / (r * r - 1.0);
        x.push_back(r);
        dp.push_back(d);
    }
}

}  // namespace

cudaError_t launch_ordgen(const OrdGenArgs &a, cudaStream_t st)
{
    if (a.total_cells <= 0) return cudaSuccess;
    ordgen_kernel<<<(a.total_cells + 127) / 128, 128, 0, st>>>(a);
    return cudaGetLastError();
}

// Fill (c, s, zeta, w) of a deterministic set; returns M or -1 on bad arguments.
int host_quadrature(int kind, int n1, int n2, std::vector<double> &c, std::vector<double> &s,
                    std::vector<double> &z, std::vector<double> &w)
{
    const double pi = 3.14159265358979323846;
    c.clear();
    s.clear();
    z.clear();
    w.clear();
    std::vector<double> qz, qt, qw;  // first quadrant (zeta, theta, weight)
    if (kind == 0) {                 // 2D uniform, eq. (uniform2D)
        if (n1 < 1 || n1 > 4096) return -1;
        const int N = n1;
        for (int i = 1; i <= N; ++i)
            for (int j = 1; j <= N; ++j) {
                qz.push_back((2.0 * N - 2.0 * i + 1.0) / (2.0 * N));
                qt.push_back((2.0 * j - 1.0) * pi / (4.0 * N));
                qw.push_back(1.0 / (4.0 * N * N));
            }
    } else if (kind == 1) {  // 2D Gaussian, Appendix A
        if (n1 < 1 || n1 > 1000) return -1;
        const int N = n1;
        std::vector<double> r, d;
        legendre_pos_roots(2 * N, r, d);
        for (int i = 1; i <= N; ++i) {
            const double zi = r[i - 1];
            const double wi = 1.0 / (2.0 * i * (1.0 - zi * zi) * d[i - 1] * d[i - 1]);
            for (int j = 1; j <= i; ++j) {
                qz.push_back(zi);
                qt.push_back((2.0 * j - 1.0) * pi / (4.0 * i));
                qw.push_back(wi);
            }
        }
    } else if (kind == 2) {  // product Gauss-Legendre x equally spaced azimuths
        if (n1 < 1 || n2 < 1 || n1 > 1000 || n2 > 100000) return -1;
        std::vector<double> r, d;
        legendre_pos_roots(2 * n1, r, d);
        for (int i = 0; i < n1; ++i) {
            const double wi = 2.0 / ((1.0 - r[i] * r[i]) * d[i] * d[i]);  // Gauss-Legendre weight
            const double rho = sqrt(1.0 - r[i] * r[i]);
            for (int j = 1; j <= n2; ++j) {
                const double th = (2.0 * j - 1.0) * pi / n2;
                c.push_back(rho * cos(th));
                s.push_back(rho * sin(th));
                z.push_back(r[i]);
                w.push_back(wi / n2);
            }
        }
        return (int)c.size();
    } else {
        return -1;
    }
    const int m = (int)qz.size();
    c.resize(4 * m);
    s.resize(4 * m);
    z.resize(4 * m);
    w.resize(4 * m);
    for (int l = 0; l < m; ++l) {
        const double rho = sqrt(1.0 - qz[l] * qz[l]);
        const double cc = rho * cos(qt[l]), ss = rho * sin(qt[l]);
        for (int q = 0; q < 4; ++q) {
            const int o = l + q * m;
            c[o] = (q == 1 || q == 2) ? -cc : cc;
            s[o] = (q >= 2) ? -ss : ss;
            z[o] = qz[l];
            w[o] = qw[l];
        }
    }
    return 4 * m;
}

}  // namespace romk
