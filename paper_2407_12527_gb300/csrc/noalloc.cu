// noalloc.cu -- rom_sweep_xy_noalloc: one transport sweep that allocates no
// device memory.
//
// Some callers cannot call cudaMalloc: plug-ins whose host application owns
// all device memory through its own pool and forbids other allocations, or
// real-time code paths where an allocation (and the implicit device
// synchronisation it may bring) is not allowed.  For them this entry point runs the sweep kernel of the library with
// its scratch memory -- padded copies of the inputs and the per-sample moment
// accumulators -- placed in one fixed-size array in the library's own
// device memory instead of in buffers it would allocate.
//
// The array below is a file-scope __device__ variable: every GPU that loads
// this library holds its kNoallocScratchBytes until the process exits, whether
// or not the entry point is called.  Host code must not use the name of the
// array as a pointer (on the host it is only a stand-in symbol); the device
// address is obtained once per device with cudaGetSymbolAddress, on the first
// call made with that device current, and cached for the life of the process.
// Because of that one-time set-up, make the first call on each device before
// any stream capture; after cudaDeviceReset the cached address is stale, so the
// entry point must not be used again on a reset device.  The small tables are
// staged in a static host table and copied with cudaMemcpyAsync from pageable
// memory, which returns only once the source bytes have been taken, so the next
// call may overwrite the table.
//
// All calls on a device share the array and it keeps the contents of the last
// call.  Nothing in it has to start at zero: every call overwrites (or clears)
// each byte it later reads.  Calls whose work overlaps on the GPU (different streams, or
// different host threads) race on the array and give wrong results; serialise
// them.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "../../include/rom.h"
#include "rom_internal.cuh"

namespace {

constexpr size_t kNoallocScratchBytes = (size_t)ROM_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;
constexpr int kMaxItems = 4096;
constexpr int kMaxOrdinates = 8192;
constexpr int kMaxSamples = 1024;
constexpr int kG = 2;  // ordinates per sweep work item

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_mu;
void *g_scratch_addr[kMaxDevices];

// Host staging of the small tables (guarded by g_mu; copied before return).
struct HostTables {
    romk::SweepItem items[kMaxItems];
    int active[kMaxSamples];
    float c[kMaxOrdinates], s[kMaxOrdinates], w[kMaxOrdinates];
};
HostTables g_host;

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

int report(char *errbuf, size_t len, int code, const char *msg, long long a = 0, long long b = 0)
{
    if (errbuf && len > 0) snprintf(errbuf, len, msg, a, b);
    return code;
}

// [J][I] -> [J][NXP] copies of sigma_T (padding 1) and of every sample's source (padding 0).
__global__ void noalloc_pad_kernel(const float *sigma_t, const float *src, int S, int I, int J,
                                   int NXP, float *st_pad, float *src_pad)
{
    const long long cells = (long long)J * NXP;
    const long long n = (long long)(S + 1) * cells;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        const long long a = v / cells, r = v - a * cells;
        const long long j = r / NXP, i = r - j * NXP;
        if (a == 0) st_pad[r] = i < I ? sigma_t[j * I + i] : 1.f;
        else src_pad[(a - 1) * cells + r] = i < I ? src[(a - 1) * (long long)J * I + j * I + i] : 0.f;
    }
}

// phi[s][j][i] = the moments the work items of sample s added to its accumulator.
__global__ void noalloc_unpad_kernel(const float *part, int S, int I, int J, int NXP, float *phi)
{
    const long long cells = (long long)J * NXP;
    const long long n = (long long)S * J * I;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        const long long s = v / ((long long)J * I), r = v - s * J * I;
        const long long j = r / I, i = r - j * I;
        phi[v] = part[s * cells + j * NXP + i];
    }
}

int blocks(long long n) { return (int)std::min<long long>(4096, std::max<long long>(1, (n + 255) / 256)); }

}  // namespace

extern "C" int rom_sweep_xy_noalloc(void *cuda_stream, int I, int J, double dx, double dy,
                                    int scheme, const float *sigma_t, int n_samples,
                                    const int32_t *m_per_sample, const double *dirs,
                                    const double *weights, const float *src, float *phi,
                                    char *errbuf, size_t errbuf_len)
{
    if (errbuf && errbuf_len) errbuf[0] = '\0';
    if (I < 1 || J < 1 || n_samples < 1 || !sigma_t || !src || !phi || !m_per_sample || !dirs ||
        !weights)
        return report(errbuf, errbuf_len, ROM_ERR_INVALID_ARG,
                      "need I, J, n_samples >= 1 and non-NULL arrays");
    if (!(dx > 0.0) || !(dy > 0.0) || (scheme != ROM_SCHEME_DD && scheme != ROM_SCHEME_STEP))
        return report(errbuf, errbuf_len, ROM_ERR_INVALID_ARG, "need dx, dy > 0 and a known scheme");
    if (I > 32 * romk::kMaxWarps * romk::kCols)
        return report(errbuf, errbuf_len, ROM_ERR_INVALID_ARG, "I = %lld exceeds %lld", I,
                      32 * romk::kMaxWarps * romk::kCols);
    if (n_samples > kMaxSamples)
        return report(errbuf, errbuf_len, ROM_ERR_INVALID_ARG, "%lld samples exceed the limit %lld",
                      n_samples, kMaxSamples);
    long long mtot = 0;
    for (int s = 0; s < n_samples; ++s) {
        if (m_per_sample[s] < 1)
            return report(errbuf, errbuf_len, ROM_ERR_INVALID_ARG, "sample %lld has no ordinates", s);
        mtot += m_per_sample[s];
    }
    if (mtot > kMaxOrdinates)
        return report(errbuf, errbuf_len, ROM_ERR_INVALID_ARG,
                      "%lld ordinates exceed the limit %lld", mtot, kMaxOrdinates);
    for (long long o = 0; o < mtot; ++o) {
        const double c = dirs[3 * o], sv = dirs[3 * o + 1], z = dirs[3 * o + 2];
        if (!(weights[o] > 0.0) || !isfinite(weights[o]) || !(fabs(c * c + sv * sv + z * z - 1.0) <= 1e-6))
            return report(errbuf, errbuf_len, ROM_ERR_INVALID_ARG,
                          "ordinate %lld: need a unit direction and a positive weight", o);
    }

    std::lock_guard<std::mutex> lock(g_mu);
    // work items: up to kG ordinates of one quadrant of one sample, samples in order
    int n_items = 0;
    long long off = 0;
    for (int s = 0; s < n_samples; ++s) {
        g_host.active[s] = 1;
        for (int code = 0; code < 4; ++code) {
            romk::SweepItem cur{};
            cur.n = 0;
            for (int l = 0; l < m_per_sample[s]; ++l) {
                const long long o = off + l;
                const int q = (dirs[3 * o] < 0.0 ? 1 : 0) | (dirs[3 * o + 1] < 0.0 ? 2 : 0);
                if (q != code) continue;
                if (cur.n == kG) {
                    if (n_items >= kMaxItems)
                        return report(errbuf, errbuf_len, ROM_ERR_INVALID_ARG,
                                      "more than %lld work items", kMaxItems);
                    g_host.items[n_items++] = cur;
                    cur = romk::SweepItem{};
                }
                cur.sample = s;
                cur.quad = code;
                cur.ord[cur.n++] = (int)o;
            }
            if (cur.n > 0) {
                for (int t = cur.n; t < romk::kMaxG; ++t) cur.ord[t] = cur.ord[0];
                if (n_items >= kMaxItems)
                    return report(errbuf, errbuf_len, ROM_ERR_INVALID_ARG,
                                  "more than %lld work items", kMaxItems);
                g_host.items[n_items++] = cur;
            }
        }
        off += m_per_sample[s];
    }
    for (long long o = 0; o < mtot; ++o) {
        g_host.c[o] = (float)dirs[3 * o];
        g_host.s[o] = (float)dirs[3 * o + 1];
        g_host.w[o] = (float)weights[o];
    }

    // scratch layout (each region 256-byte aligned)
    const int NXP = (I + romk::kCols - 1) / romk::kCols * romk::kCols;
    const size_t cells = (size_t)J * NXP;
    size_t o_st = 0;
    size_t o_src = o_st + align256(cells * 4);
    size_t o_part = o_src + align256((size_t)n_samples * cells * 4);
    size_t o_items = o_part + align256((size_t)n_samples * cells * 4);
    size_t o_active = o_items + align256((size_t)n_items * sizeof(romk::SweepItem));
    size_t o_c = o_active + align256((size_t)n_samples * sizeof(int));
    size_t o_s = o_c + align256((size_t)mtot * 4);
    size_t o_w = o_s + align256((size_t)mtot * 4);
    const size_t need = o_w + align256((size_t)mtot * 4);
    if (need > kNoallocScratchBytes)
        return report(errbuf, errbuf_len, ROM_ERR_INVALID_ARG,
                      "problem needs %lld bytes of scratch; the fixed maximum is %lld bytes",
                      (long long)need, (long long)kNoallocScratchBytes);

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return report(errbuf, errbuf_len, ROM_ERR_CUDA, "no usable current CUDA device");
    if (!g_scratch_addr[dev]) {  // one-time set-up on this device
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return report(errbuf, errbuf_len, ROM_ERR_CUDA,
                          "cudaGetSymbolAddress of the scratch array failed");
        }
        g_scratch_addr[dev] = p;
    }
    unsigned char *base = (unsigned char *)g_scratch_addr[dev];
    cudaStream_t st = (cudaStream_t)cuda_stream;

#define NA_CK(call)                                                                           \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return report(errbuf, errbuf_len, ROM_ERR_CUDA, "CUDA error %lld in " #call,       \
                          (long long)e_);                                                     \
    } while (0)

    NA_CK(cudaMemcpyAsync(base + o_items, g_host.items, n_items * sizeof(romk::SweepItem),
                          cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemcpyAsync(base + o_active, g_host.active, n_samples * sizeof(int),
                          cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemcpyAsync(base + o_c, g_host.c, mtot * 4, cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemcpyAsync(base + o_s, g_host.s, mtot * 4, cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemcpyAsync(base + o_w, g_host.w, mtot * 4, cudaMemcpyHostToDevice, st));

    float *st_pad = (float *)(base + o_st), *src_pad = (float *)(base + o_src);
    float *part = (float *)(base + o_part);
    NA_CK(cudaMemsetAsync(part, 0, (size_t)n_samples * cells * 4, st));  // the sweep adds into it
    noalloc_pad_kernel<<<blocks((long long)(n_samples + 1) * cells), 256, 0, st>>>(
        sigma_t, src, n_samples, I, J, NXP, st_pad, src_pad);
    NA_CK(cudaGetLastError());

    romk::SweepArgs a{};
    a.I = I;
    a.J = J;
    a.NXP = NXP;
    a.inv_dx = (float)(1.0 / dx);
    a.inv_dy = (float)(1.0 / dy);
    a.sigma_t_homog = 1.f;
    a.sigma_t = st_pad;
    a.src = src_pad;
    a.part = part;
    a.items = (const romk::SweepItem *)(base + o_items);
    a.oc = (const float *)(base + o_c);
    a.os = (const float *)(base + o_s);
    a.ow = (const float *)(base + o_w);
    a.inflow = nullptr;
    a.inflow_stride = 0;
    a.active = (const int *)(base + o_active);
    a.cells = (long long)cells;
    const int L = (I + romk::kCols - 1) / romk::kCols;
    NA_CK(romk::launch_sweep2d(a, n_items, (L + 31) / 32, kG, scheme, false, 1, 4, st));
    noalloc_unpad_kernel<<<blocks((long long)n_samples * J * I), 256, 0, st>>>(part, n_samples, I,
                                                                               J, NXP, phi);
    NA_CK(cudaGetLastError());
#undef NA_CK
    return ROM_OK;
}
