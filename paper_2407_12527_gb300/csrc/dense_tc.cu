// dense_tc.cu -- the dense scattering source on the 5th-generation tensor cores
// (K4, tensor-core variant).
//
// Per sample s and ordinate l (eq. equ_random with the discrete kernel of eq. wl):
//   S_l(z) = sigma_S(z) sum_l' A[l][l'] psi_l'(z) + q(z),   A[l][l'] = w_l' P(u_l', u_l),
// i.e. the product D = A Psi of the M x M operator with the M x cells matrix of
// cell values, followed by the sigma_S / q epilogue.  M <= 128.
//
// Precision: split BF16.  Each FP32 value v is carried as v_hi = v rounded to
// the nearest BF16 (ties away from zero) and v_lo = bf16_rn(v - v_hi) (16
// significant bits in all), written that way by the sweep (psi, as one 32-byte
// sector [8 hi | 8 lo] per 8 cells) and by pmat_split_kernel (A).  Read as one
// BF16 matrix, a row of psi is B' = [Psi_hi | Psi_lo] interleaved by 8 cells,
// twice as wide; the tensor cores compute A_hi B' + A_lo B' (FP32 accumulate in
// tensor memory, N = 256 per 128 cells) and the epilogue adds the hi and lo
// columns of each cell: D = (A_hi + A_lo)(Psi_hi + Psi_lo).
//
// GB300 mapping: one persistent CTA per SM walks a contiguous range of the
// (sample, 128-cell tile) units of the samples still iterating (every CTA
// lists those samples the same way, so the work stays balanced as samples
// finish).  Warp 0 (one lane) is the TMA producer: the sample's A_hi / A_lo
// (K-major, two 64-column boxes each) once per sample and, per unit, the
// 128 x 256 B' tile (MN-major, four 64-column boxes) into a two-stage ring, all
// with the 128-byte swizzle.  Warp 1 owns the tensor memory (two 128 x 256 FP32
// accumulators, all 512 columns) and one lane issues, per unit, 8 K-steps x 2
// tcgen05.mma (kind::f16, BF16 in, FP32 accumulate, M = 128, N = 256),
// committing to mbarriers that free the B' stage and hand the accumulator to
// the epilogue.  Warps 2-5 read the accumulator (tcgen05.ld,
// one TMEM lane per ordinate row), apply sigma_S and q (staged in shared memory
// one unit ahead) and store the FP32 sources.  Every mbarrier wait is bounded;
// on timeout the CTA raises an error flag, drains what it has in flight, frees
// its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "rom_internal.cuh"

namespace romk {
namespace {

constexpr int kTileN = 128;                  // cells per unit
constexpr int kMmaN = 2 * kTileN;            // B' columns per unit (hi and lo of each cell)
constexpr int kK = 128;                      // ordinates (rows of A, K of the product)
constexpr int kStages = 2;                   // Psi tile ring
constexpr uint32_t kBox = 128 * 64 * 2;      // bytes of one 64-wide, 128-high bf16 box (16 KB)
constexpr uint32_t kAbytes = 4 * kBox;       // A_hi + A_lo, two K-halves each (64 KB)
constexpr uint32_t kBbytes = 4 * kBox;       // B' = [Psi_hi | Psi_lo], four 64-column boxes (64 KB)
constexpr int kThreads = 6 * 32;
constexpr uint32_t kTmemCols = 512;          // two accumulators of 256 columns
constexpr unsigned kWaitTries = 1u << 22;
constexpr int kMaxSamples = 2048;            // samples a launch can list (DenseTcArgs::S)

struct TcBarriers {
    unsigned long long a_full, a_empty;
    unsigned long long b_full[kStages], b_empty[kStages];
    unsigned long long acc_full[2], acc_empty[2];
    uint32_t tmem_base;
    int abort_flag;
    float sq[2][2][kTileN];  // sigma_S and q of a unit's cells, per accumulator buffer
    int n_act;               // samples still iterating, and their indices in order
    int act[kMaxSamples];
};
// dynamic shared memory: [align pad][A 64 KB][B stage 0 64 KB][B stage 1 64 KB][barriers]
constexpr uint32_t kSmemBytes = 1024 + kAbytes + kStages * kBbytes + 12288;
static_assert(sizeof(TcBarriers) <= 12288, "barrier block");

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long *b, uint32_t count)
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
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *b, uint32_t bytes)
{
    asm volatile(
        "{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
            smem_u32(b)),
        "r"(bytes)
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *b, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity), "r"(1000u)
        : "memory");
    return ok != 0;
}
// Bounded wait of one thread; false on timeout.
__device__ __forceinline__ bool wait1(unsigned long long *b, uint32_t parity)
{
    for (unsigned i = 0; i < kWaitTries; ++i)
        if (mbar_try_wait(b, parity)) return true;
    return false;
}
// Bounded wait of a whole warp (lanes leave together).
__device__ __forceinline__ bool wait_warp(unsigned long long *b, uint32_t parity)
{
    for (unsigned i = 0; i < kWaitTries; ++i)
        if (__all_sync(0xffffffffu, mbar_try_wait(b, parity))) return true;
    return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, "
        "{%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor of tcgen05: start address, leading and stride
// byte offsets (16-byte units), descriptor version 1, layout (bits 61-63: 0 no
// swizzle, 2 128-byte swizzle).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo,
                                              uint32_t layout)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | ((uint64_t)layout << 61);
}

// Instruction descriptor, kind::f16: D FP32 (bits 4-5), A and B BF16 (bits 7-9,
// 10-12), A K-major (bit 15 clear), B MN-major (bit 16), N >> 3 (bits 17-22),
// M >> 4 (bits 24-28); M = 128, N = 256.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | (0u << 15) | (1u << 16) |
                            ((uint32_t)(kMmaN >> 3) << 17) | ((uint32_t)(kK >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(unsigned long long *bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// The CTA's contiguous range of units u = s * n_tiles + tile.
struct UnitRange {
    long long u0, u1;
};
__device__ __forceinline__ UnitRange unit_range(long long total)
{
    const long long per = (total + gridDim.x - 1) / gridDim.x;
    UnitRange r;
    r.u0 = min(total, (long long)blockIdx.x * per);
    r.u1 = min(total, r.u0 + per);
    return r;
}

__global__ void __launch_bounds__(kThreads, 1)
    dense_tc_kernel(const __grid_constant__ DenseTcMaps maps, const DenseTcArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned tiles (the 128-byte swizzle repeats every 8 rows of 128 B)
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char *const gbase = smem_raw + (base - raw);
    const uint32_t sA = base;
    const uint32_t sB = base + kAbytes;
    TcBarriers *bar = reinterpret_cast<TcBarriers *>(gbase + kAbytes + kStages * kBbytes);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_tiles = (int)((a.cells + kTileN - 1) / kTileN);

    if (warp == 2) {  // the samples still iterating, in order (the same list in every CTA)
        int n = 0;
        for (int s0 = 0; s0 < a.S; s0 += 32) {
            const bool on = s0 + lane < a.S && a.active[s0 + lane] != 0;
            const unsigned m = __ballot_sync(0xffffffffu, on);
            if (on) bar->act[n + __popc(m & ((1u << lane) - 1u))] = s0 + lane;
            n += __popc(m);
        }
        if (lane == 0) bar->n_act = n;
    }
    if (threadIdx.x == 0) {
        mbar_init(&bar->a_full, 1);
        mbar_init(&bar->a_empty, 1);
        for (int i = 0; i < kStages; ++i) {
            mbar_init(&bar->b_full[i], 1);
            mbar_init(&bar->b_empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&bar->acc_full[i], 1);
            mbar_init(&bar->acc_empty[i], 128);
        }
        bar->abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {  // tensor memory for the two accumulators
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&bar->tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = bar->tmem_base;
    // units u = k * n_tiles + tile over the k-th sample still iterating
    const UnitRange R = unit_range((long long)bar->n_act * n_tiles);
    const int *act = bar->act;

    if (warp == 0) {
        if (lane == 0) {  // ---------------------------------------------- TMA producer
            int prev_s = -1, n_a = 0;
            long long n_b = 0;
            for (long long u = R.u0; u < R.u1; ++u) {
                if (*(volatile int *)&bar->abort_flag) break;
                const int s = act[u / n_tiles], tile = (int)(u % n_tiles);
                if (s != prev_s) {
                    if (n_a > 0 && !wait1(&bar->a_empty, (uint32_t)(n_a - 1) & 1u)) {
                        atomicOr(a.err, 4);
                        bar->abort_flag = 1;
                        break;
                    }
                    mbar_expect_tx(&bar->a_full, kAbytes);
                    for (int kb = 0; kb < 2; ++kb) {
                        tma_load_2d(sA + kb * kBox, &maps.a_hi, 64 * kb, 128 * s, &bar->a_full);
                        tma_load_2d(sA + (2 + kb) * kBox, &maps.a_lo, 64 * kb, 128 * s,
                                    &bar->a_full);
                    }
                    ++n_a;
                    prev_s = s;
                }
                const int st = (int)(n_b % kStages);
                if (n_b >= kStages &&
                    !wait1(&bar->b_empty[st], (uint32_t)((n_b / kStages) - 1) & 1u)) {
                    atomicOr(a.err, 8);
                    bar->abort_flag = 1;
                    break;
                }
                mbar_expect_tx(&bar->b_full[st], kBbytes);
                const uint32_t dst = sB + st * kBbytes;
                const int row0 = (int)a.ord_off[s], x0 = tile * kTileN;
                // B' columns [2 x0, 2 x0 + 256) of the rows of sample s: four 64-wide boxes
                for (int nb = 0; nb < 4; ++nb)
                    tma_load_2d(dst + nb * kBox, &maps.b, 2 * x0 + 64 * nb, row0, &bar->b_full[st]);
                ++n_b;
            }
            // drain: the copies in flight complete before the CTA may leave
            for (long long k = n_b - kStages; k < n_b; ++k)
                if (k >= 0) wait1(&bar->b_full[k % kStages], (uint32_t)(k / kStages) & 1u);
            if (n_a > 0) wait1(&bar->a_full, (uint32_t)(n_a - 1) & 1u);
        }
    } else if (warp == 1) {
        if (lane == 0) {  // ---------------------------------------------- MMA issuer
            int prev_s = -1, n_a = 0;
            long long n_b = 0;
            for (long long u = R.u0; u < R.u1; ++u) {
                if (*(volatile int *)&bar->abort_flag) break;
                const int s = act[u / n_tiles];
                if (s != prev_s) {
                    if (!wait1(&bar->a_full, (uint32_t)n_a & 1u)) {
                        atomicOr(a.err, 16);
                        bar->abort_flag = 1;
                        break;
                    }
                    ++n_a;
                    prev_s = s;
                }
                const int st = (int)(n_b % kStages), acc = (int)(n_b & 1);
                if (!wait1(&bar->b_full[st], (uint32_t)(n_b / kStages) & 1u)) {
                    atomicOr(a.err, 32);
                    bar->abort_flag = 1;
                    break;
                }
                if (n_b >= 2 && !wait1(&bar->acc_empty[acc], (uint32_t)((n_b >> 1) - 1) & 1u)) {
                    atomicOr(a.err, 64);
                    bar->abort_flag = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + (uint32_t)acc * kMmaN;
                const uint32_t bb = sB + st * kBbytes;
#pragma unroll
                for (int ks = 0; ks < kK / 16; ++ks) {
                    // A: K-major, 128-byte rows of 64 k; the 16-wide K slice sits 32 B in
                    const uint32_t aoff = (ks >> 2) * kBox + (ks & 3) * 32;
                    const uint64_t a_hi = smem_desc(sA + aoff, 16, 1024, 2);
                    const uint64_t a_lo = smem_desc(sA + 2 * kBox + aoff, 16, 1024, 2);
                    // B': MN-major, 8-row (k) atoms of 1024 B; the next 64 columns at +16 KB
                    const uint64_t b = smem_desc(bb + ks * 2048, kBox, 1024, 2);
                    mma_bf16(d, a_hi, b, ks > 0 ? 1u : 0u);
                    mma_bf16(d, a_lo, b, 1u);
                }
                mma_commit(&bar->b_empty[st]);
                mma_commit(&bar->acc_full[acc]);
                // the last unit of this sample frees A for the producer
                if (u + 1 >= R.u1 || act[(u + 1) / n_tiles] != s) mma_commit(&bar->a_empty);
                ++n_b;
            }
            // the last products are complete before the tensor memory is freed
            if (n_b > 0) wait1(&bar->acc_full[(n_b - 1) & 1], (uint32_t)((n_b - 1) >> 1) & 1u);
        }
    } else {  // ------------------------------------------------------- epilogue (warps 2-5)
        // Each thread holds one TMEM lane (an ordinate row) and writes 128 cells of it.
        // sigma_S and q of a unit's 128 cells are staged in shared memory (one value
        // per thread, loaded one unit ahead) and read back as broadcasts.
        const int g = warp & 3;  // TMEM lane quarter this warp may access
        const int row = 32 * g + lane;
        const int et = threadIdx.x - 64;  // 0..127
        long long n_b = 0;
        auto fetch = [&](long long u, float &ssv, float &qv) {
            ssv = qv = 0.f;
            if (u < R.u1) {
                const long long n = (u % n_tiles) * kTileN + et;
                if (n < a.cells) {
                    ssv = a.sigma_s[n];
                    qv = a.q[n];
                }
            }
        };
        float ss_next, q_next;
        fetch(R.u0, ss_next, q_next);
        for (long long u = R.u0; u < R.u1; ++u) {
            const int s = act[u / n_tiles], tile = (int)(u % n_tiles);
            const int acc = (int)(n_b & 1);
            bar->sq[acc][0][et] = ss_next;
            bar->sq[acc][1][et] = q_next;
            asm volatile("bar.sync 1, 128;" ::: "memory");
            fetch(u + 1, ss_next, q_next);
            const bool ok = wait_warp(&bar->acc_full[acc], (uint32_t)(n_b >> 1) & 1u);
            // the four epilogue warps leave together or not at all (they share a named barrier)
            uint32_t any_fail;
            asm volatile(
                "{\n\t.reg .pred p, q;\n\tsetp.eq.u32 p, %1, 0;\n\t"
                "bar.red.or.pred q, 1, 128, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
                : "=r"(any_fail)
                : "r"(ok ? 1u : 0u)
                : "memory");
            if (any_fail) {
                if (lane == 0) atomicOr(a.err, 128);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int M = a.M[s];
            const long long n0 = (long long)tile * kTileN;
            float *dst = a.src + ((long long)a.ord_off[s] + row) * a.cells;
            const float *sss = bar->sq[acc][0], *sqq = bar->sq[acc][1];
            // columns 16 j .. 16 j + 7: the hi products of cells 8 j .. 8 j + 7,
            // columns 16 j + 8 .. 16 j + 15: their lo products
#pragma unroll 1
            for (int c = 0; c < kMmaN / 32; ++c) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(32 * g) << 16) + (uint32_t)acc * kMmaN + 32 * c, v);
                const long long nc = n0 + 16 * c;
                if (row < M && nc < a.cells) {
#pragma unroll
                    for (int q8 = 0; q8 < 2; ++q8) {
                        const long long n = nc + 8 * q8;
                        if (n < a.cells) {
                            float out[8];
#pragma unroll
                            for (int e = 0; e < 8; ++e) {
                                const int j = 16 * c + 8 * q8 + e;
                                out[e] = fmaf(sss[j], v[16 * q8 + e] + v[16 * q8 + 8 + e], sqq[j]);
                            }
                            stg8(dst + n, out);
                        }
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(&bar->acc_empty[acc]);
            ++n_b;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols)
                     : "memory");
    }
}

// A (FP32, M x M per sample) -> A_hi, A_lo (BF16, 128 x 128 per sample, zero padded).
__global__ void pmat_split_kernel(const float *A, const int *Ms, const long long *a_off, int S,
                                  __nv_bfloat16 *hi, __nv_bfloat16 *lo)
{
    const int s = blockIdx.x;
    if (s >= S) return;
    const int M = Ms[s];
    for (int i = threadIdx.x; i < kK * kK; i += blockDim.x) {
        const int l = i / kK, lp = i % kK;
        const float v = (l < M && lp < M) ? A[a_off[s] + (long long)l * M + lp] : 0.f;
        const uint32_t b = (__float_as_uint(v) + 0x8000u) & 0xFFFF0000u;
        const float vh = __uint_as_float(b);
        hi[(long long)s * kK * kK + i] = __ushort_as_bfloat16((unsigned short)(b >> 16));
        lo[(long long)s * kK * kK + i] = __float2bfloat16_rn(v - vh);
    }
}

using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                              const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                              const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn()
{
    static EncodeFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
        else
            (void)cudaGetLastError();
    }
    return fn;
}

// 2D BF16 map over [rows][cols] (cols contiguous), 64 x 128 boxes, 128-byte swizzle,
// zero fill outside the tensor.
bool make_map(CUtensorMap *m, const void *ptr, unsigned long long cols, unsigned long long rows)
{
    EncodeFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {cols * 2};
    const cuuint32_t box[2] = {64, 128};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

int dense_tc_max_m() { return kK; }
int dense_tc_max_samples() { return kMaxSamples; }

cudaError_t launch_pmat_split(const float *A, const int *M, const long long *a_off, int S,
                              void *hi, void *lo, cudaStream_t st)
{
    if (S <= 0) return cudaSuccess;
    pmat_split_kernel<<<S, 256, 0, st>>>(A, M, a_off, S, (__nv_bfloat16 *)hi, (__nv_bfloat16 *)lo);
    return cudaGetLastError();
}

cudaError_t make_dense_tc_maps(DenseTcMaps *maps, const void *a_hi, const void *a_lo, int S,
                               const void *psi_split, long long m_total, long long cells)
{
    if ((cells % 8) != 0 || m_total < 1 || S < 1) return cudaErrorInvalidValue;
    // the kernel's shared memory (set on the current device, outside any capture)
    cudaError_t e = cudaFuncSetAttribute(dense_tc_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    if (!make_map(&maps->a_hi, a_hi, kK, (unsigned long long)S * kK) ||
        !make_map(&maps->a_lo, a_lo, kK, (unsigned long long)S * kK) ||
        !make_map(&maps->b, psi_split, 2ull * (unsigned long long)cells,
                  (unsigned long long)m_total))
        return cudaErrorInvalidValue;
    return cudaSuccess;
}

cudaError_t launch_dense_tc(const DenseTcMaps &maps, const DenseTcArgs &a, int n_ctas,
                            cudaStream_t st)
{
    if (a.S <= 0 || n_ctas <= 0) return cudaSuccess;
    if (a.S > kMaxSamples) return cudaErrorInvalidValue;
    dense_tc_kernel<<<n_ctas, kThreads, kSmemBytes, st>>>(maps, a);
    return cudaGetLastError();
}

}  // namespace romk
