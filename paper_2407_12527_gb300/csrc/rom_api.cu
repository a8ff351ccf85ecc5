// rom_api.cu -- the C ABI of include/rom.h: context, problem setters, the
// source-iteration driver and result getters.  All arithmetic of the method
// runs in the kernels of sweep2d.cu, reduce.cu and ordinates.cu; this file
// validates arguments, lays data out in device memory and orders launches.
//
// Source iteration (Sec. 3.2, eq. psiexpansion), per sweep k:
//   sweep    (K1; K9 on 3D grids) every active sample: moments of
//                  L^{-1}(scatter(psi^{k-1}) + q)
//   combine  (K2)  phi^k per sample, next source, FP64 residual and balance sums
//   finalize (K5)  ||phi^k - phi^{k-1}|| / ||phi^k|| per sample, stop flags
// then the FP64 sample average (K6).  The loop runs either on the device (a
// CUDA graph whose conditional while-node repeats the three kernels until no
// sample is active; no host round trip per sweep) or on the host, reading the
// number of active samples every `check_every` sweeps.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "../../include/rom.h"
#include "rom_internal.cuh"

namespace romk {
int host_quadrature(int kind, int n1, int n2, std::vector<double> &c, std::vector<double> &s,
                    std::vector<double> &z, std::vector<double> &w);

}  // namespace romk

using romk::SweepItem;

namespace {

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
};

enum OrdSource { ORD_NONE = 0, ORD_EXPLICIT = 1, ORD_SEED = 2 };

}  // namespace

struct rom_ctx {
    int device = 0;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    std::string err;
    rom_options opt{};

    // grid (dim 3: K planes; cell arrays are [K][J][NXP], rows = J * K)
    bool grid_set = false;
    int dim = 2;
    int I = 0, J = 0, K = 1, NXP = 0;
    long long rows = 0;
    double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
    bool homog = false;
    float sigma_t_homog = 1.f;
    DevBuf sigt, sigs, q;

    // inflow (host copies; uploaded at solve time)
    std::vector<double> inflow_iso[6];
    std::vector<double> inflow_ord[6];
    bool inflow_dirty = true;
    DevBuf inflow_dev;
    bool inflow_any = false;
    long long inflow_stride = 0;

    // ordinates
    int ord_source = ORD_NONE;
    int S = 0;
    long long Mtot = 0;
    std::vector<int> M;            // per sample
    std::vector<long long> off;    // first ordinate per sample
    std::vector<unsigned char> quad;  // explicit sets: octant code per ordinate (bits c<0, s<0, z<0)
    bool seed_octants = false;        // seeded sets: 3D (8 m points) or X-Y (4 m)
    DevBuf c64, s64, z64, w64, c32, s32, z32, w32;

    // kernel
    int kernel_kind = ROM_KERNEL_ISO;
    double g = 0.0;
    int kernel_flags = 0;

    // work items
    bool items_dirty = true;
    int G_used = 0;
    int H_used = 4;   // X-Y sweep: rows a lane advances per wavefront step
    int tuned_g = 0;  // measured choice (tile_g = -1), valid while the layout is unchanged
    int tuned_h = 0;  // rows per step of that choice
    // per-sample tables of the balance: first ordinate and count, weight sums
    DevBuf otab, ordsum;
    // several X-Y grids in one context (rom_set_grids_xy; n_grids = 0: one grid):
    // the first grid_samples[0] samples are on grid 0, and so on
    int n_grids = 0;
    std::vector<romk::GridDesc> grids;
    std::vector<int> grid_samples;
    std::vector<long long> avg_off;  // first value of each grid's average in avg / sum
    long long coef_cells = 0;        // cells of the concatenated coefficient arrays
    std::vector<int> sgrid;          // grid of each sample
    std::vector<long long> soff;     // first float of each sample's [MOM][cells] block
    long long state_floats = 0;      // floats of one per-sample state array (all samples)
    long long max_cells = 0;         // largest grid's J * NXP
    DevBuf gdesc, sgrid_dev, soff_dev, sdA_dev;
    // per-sample divergence and balance state: dprev, grow, leak (added by the
    // sweep), bal / leak_out / phimin (last sweep); the X-Y sweep's wait flag
    DevBuf dprev, grow, leak, bal, leak_out, phimin, sweep_err;
    std::vector<double> h_bal, h_leak, h_phimin;
    std::vector<SweepItem> items;
    DevBuf items_dev;
    float *h_stage = nullptr;  // pinned host staging of rom_set_grid (reused; the call syncs)
    size_t h_stage_cap = 0;
    // 3D: CTA item lists (one octant each) and the tile hand-off buffers
    std::vector<int> cta_begin, cta_list;
    DevBuf cta_begin_dev, cta_list_dev, xface, yface, err3;
    // 3D diagonal storage: sigma_T [2], source and flux [2][S], sigma_S and q (family 0);
    // phi is kept in family 0 as well ([S][sk.cells])
    DevBuf sig3, src3, acc3, ss3, q3;
    int n_ctas3 = 0, nwarps3 = 1, n_tx = 1, n_ty = 1;

    // dense scattering operator (mode 0); tensor-core variant: split BF16 psi and A
    DevBuf psi, src_ord, Amat, dtab, psi_split, a_hi, a_lo, tc_err;
    bool pmat_dirty = true;
    romk::DenseTcMaps tc_maps;
    const void *tc_map_ptrs[3] = {nullptr, nullptr, nullptr};
    long long tc_map_cells = 0, tc_map_mtot = 0;
    int tc_map_S = 0;

    // iteration state
    int MOM = 1;  // 1 isotropic moments, 3 linear moments, 0 dense operator
    int chunks = 1;
    DevBuf phi, src, part, sums, minkey, active, iters, flags, resid, n_active, avg, sum, tmp;
    bool solved = false;
    std::vector<int> h_iters;
    std::vector<double> h_resid;

    // device-side loop
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    bool graph_valid = false;

    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<cudaEvent_t> kev;  // sweep-kernel timing events (time_kernels = 1)
    long long launches = 0;
    int sm_count = 152;
};

namespace {

int fail(rom_ctx *c, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(ctx, ROM_ERR_CUDA, "%s failed: %s (%s:%d)", #call,                    \
                        cudaGetErrorString(e_), __FILE__, __LINE__);                          \
    } while (0)

int ensure(rom_ctx *ctx, DevBuf &b, size_t bytes)
{
    if (bytes == 0) bytes = 256;
    if (b.cap >= bytes) return ROM_OK;
    if (b.p) {
        cudaError_t e = cudaFree(b.p);
        b.p = nullptr;
        b.cap = 0;
        if (e != cudaSuccess) return fail(ctx, ROM_ERR_CUDA, "cudaFree: %s", cudaGetErrorString(e));
    }
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        b.p = nullptr;
        (void)cudaGetLastError();
        return fail(ctx, ROM_ERR_OOM, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
    }
    b.cap = bytes;
    return ROM_OK;
}

int ensure_host_stage(rom_ctx *ctx, size_t bytes)
{
    if (ctx->h_stage_cap >= bytes) return ROM_OK;
    if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    ctx->h_stage = nullptr;
    ctx->h_stage_cap = 0;
    void *p = nullptr;
    cudaError_t e = cudaMallocHost(&p, bytes);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(ctx, ROM_ERR_OOM, "cudaMallocHost(%zu bytes): %s", bytes, cudaGetErrorString(e));
    }
    ctx->h_stage = (float *)p;
    ctx->h_stage_cap = bytes;
    return ROM_OK;
}

void release(DevBuf &b)
{
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
}

void invalidate_graph(rom_ctx *ctx)
{
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    if (ctx->graph) cudaGraphDestroy(ctx->graph);
    ctx->graph_exec = nullptr;
    ctx->graph = nullptr;
    ctx->graph_valid = false;
}

void reset_ordinate_dependents(rom_ctx *ctx)
{
    ctx->pmat_dirty = true;
    ctx->tuned_g = 0;
    ctx->tuned_h = 0;
    for (int f = 0; f < 6; ++f) ctx->inflow_ord[f].clear();
    ctx->inflow_dirty = true;
    ctx->items_dirty = true;
    ctx->solved = false;
    invalidate_graph(ctx);
}

int n_faces(const rom_ctx *ctx) { return ctx->dim == 3 ? 6 : 4; }

// cells of a face: 2D x faces J, y faces I; 3D x faces K*J, y faces K*I, z faces J*I
long long face_cells(const rom_ctx *ctx, int face)
{
    const long long K = ctx->dim == 3 ? ctx->K : 1;
    if (face < 2) return K * ctx->J;
    if (face < 4) return K * ctx->I;
    return (long long)ctx->J * ctx->I;
}

long long face_offset(const rom_ctx *ctx, int face)
{
    long long o = 0;
    for (int f = 0; f < face; ++f) o += face_cells(ctx, f);
    return o;
}

long long n_cells(const rom_ctx *ctx) { return (long long)ctx->I * ctx->J * ctx->K; }
// cells of the coefficient arrays: [rows][NXP], or the grids' blocks of a batch
long long padded_cells(const rom_ctx *ctx)
{
    return ctx->n_grids > 0 ? ctx->coef_cells : ctx->rows * ctx->NXP;
}
bool batch(const rom_ctx *ctx) { return ctx->n_grids > 0; }
// values of the sample average (all grids' averages, one after the other, in a batch)
long long avg_cells(const rom_ctx *ctx)
{
    return ctx->n_grids > 0 ? ctx->avg_off[ctx->n_grids] : n_cells(ctx);
}
// cells of one sample's flux (its grid's, in a batch)
long long sample_cells(const rom_ctx *ctx, int s)
{
    if (!batch(ctx)) return n_cells(ctx);
    const romk::GridDesc &g = ctx->grids[ctx->sgrid[s]];
    return (long long)g.I * g.J;
}

// prev: the context held a valid grid before this call.  A grid of the same shape
// and extent keeps the work items, the tuned work-item size, the buffers and the
// captured graph (only the coefficient arrays change); any inflow is dropped.
int set_grid_common(rom_ctx *ctx, bool prev, int dim, const int64_t n[3], const double lo[3],
                    const double hi[3])
{
    if (dim != 2 && dim != 3) return fail(ctx, ROM_ERR_INVALID_ARG, "dim must be 2 or 3 (got %d)", dim);
    if (!n || !lo || !hi) return fail(ctx, ROM_ERR_INVALID_ARG, "n, lo, hi must not be NULL");
    if (n[0] < 1 || n[1] < 1 || (dim == 3 && n[2] < 1))
        return fail(ctx, ROM_ERR_INVALID_ARG, "grid sizes must be >= 1");
    if (dim == 2 && n[0] > 32 * romk::kMaxWarps * romk::kCols)
        return fail(ctx, ROM_ERR_INVALID_ARG, "I = %lld exceeds %d", (long long)n[0],
                    32 * romk::kMaxWarps * romk::kCols);
    if (dim == 3 && (n[0] > 4096 || n[1] > 4096 || n[2] > 4096))
        return fail(ctx, ROM_ERR_INVALID_ARG, "3D grid sizes are limited to 4096 per axis");
    if (n[1] > (1 << 24)) return fail(ctx, ROM_ERR_INVALID_ARG, "J too large");
    for (int d = 0; d < dim; ++d)
        if (!(hi[d] > lo[d]) || !isfinite(lo[d]) || !isfinite(hi[d]))
            return fail(ctx, ROM_ERR_INVALID_ARG, "need hi > lo (finite)");
    const bool was_batch = batch(ctx);
    ctx->n_grids = 0;  // one grid from here on
    bool same = prev && !was_batch && ctx->dim == dim && ctx->I == (int)n[0] && ctx->J == (int)n[1] &&
                ctx->K == (dim == 3 ? (int)n[2] : 1);
    for (int d = 0; d < 3 && same; ++d)
        same = ctx->lo[d] == (d < dim ? lo[d] : 0.0) && ctx->hi[d] == (d < dim ? hi[d] : 1.0);
    ctx->dim = dim;
    ctx->I = (int)n[0];
    ctx->J = (int)n[1];
    ctx->K = dim == 3 ? (int)n[2] : 1;
    ctx->rows = (long long)ctx->J * ctx->K;
    ctx->NXP = (ctx->I + romk::kCols - 1) / romk::kCols * romk::kCols;
    for (int d = 0; d < 3; ++d) {
        ctx->lo[d] = d < dim ? lo[d] : 0.0;
        ctx->hi[d] = d < dim ? hi[d] : 1.0;
    }
    bool had_inflow = false;
    for (int f = 0; f < 6; ++f) {
        had_inflow |= !ctx->inflow_iso[f].empty() || !ctx->inflow_ord[f].empty();
        ctx->inflow_iso[f].clear();
        ctx->inflow_ord[f].clear();
    }
    ctx->solved = false;
    if (!same) {
        ctx->inflow_dirty = true;
        ctx->items_dirty = true;
        ctx->tuned_g = 0;
        ctx->tuned_h = 0;
        invalidate_graph(ctx);
    } else if (had_inflow) {
        ctx->inflow_dirty = true;  // re-uploaded (as vacuum) by the next solve
    }
    const size_t bytes = (size_t)padded_cells(ctx) * sizeof(float);
    int rc;
    if ((rc = ensure(ctx, ctx->sigt, bytes)) || (rc = ensure(ctx, ctx->sigs, bytes)) ||
        (rc = ensure(ctx, ctx->q, bytes)))
        return rc;
    return ROM_OK;
}

// Uniform sigma_T selects the sweep variant and enters its arguments: a change
// re-tunes the work-item size and rebuilds the graph.
void set_homog(rom_ctx *ctx, bool homog, float sigma_t)
{
    if (homog != ctx->homog || sigma_t != ctx->sigma_t_homog) {
        ctx->tuned_g = 0;
        ctx->tuned_h = 0;
        ctx->items_dirty = true;
        invalidate_graph(ctx);
    }
    ctx->homog = homog;
    ctx->sigma_t_homog = sigma_t;
}

// The sweep adds each sample's moments to one accumulator (vector reductions in
// L2; the combine reads and clears it) rather than storing per-item partials for
// the combine to sum: per-item partials would be cells x ordinates in 3D and GB
// in the dense mode, and in the X-Y moment modes the accumulator measured 19%
// faster per source iteration (the sweep writes less, the combine reads one
// array).  The price is the order of the additions, which follows the timing.
// 3D keeps its accumulators (and source, sigma_T) in diagonal storage, not in part;
// the X-Y moment modes keep theirs in part, in sheared storage.

// 1: isotropic moment, 3: linear-kernel moments, 0: dense operator
int source_mode(const rom_ctx *ctx)
{
    if (ctx->opt.dense_source) return 0;
    if (ctx->kernel_kind == ROM_KERNEL_ISO) return 1;
    if (ctx->kernel_kind == ROM_KERNEL_LINEAR && ctx->kernel_flags == 0) return 3;
    return 0;
}

// rows per wavefront step of the X-Y sweep: forced by the option, else the autotuned
// value (moment modes), else 4; 1 is the one-row kernel (sweep2d_row.cuh)
int choose_rows(const rom_ctx *ctx)
{
    if (ctx->dim != 2) return 4;
    if (source_mode(ctx) == 0) {  // dense operator mode: the 4-row or the one-row kernel
        if (ctx->opt.rows_per_step == 1) return 1;
        if (ctx->opt.tile_g == -1 && ctx->tuned_h > 0) return ctx->tuned_h;
        return 4;
    }
    if (ctx->opt.rows_per_step == 1 || ctx->opt.rows_per_step == 2 || ctx->opt.rows_per_step == 4)
        return ctx->opt.rows_per_step;
    if (ctx->opt.tile_g == -1 && ctx->tuned_h > 0) return ctx->tuned_h;
    return 4;
}

// X-Y moment modes: the particle balance is formed from the sweep's leakage and
// the combine's partial sums
bool has_balance(const rom_ctx *ctx) { return ctx->dim == 2 && source_mode(ctx) != 0; }

int choose_g(const rom_ctx *ctx)
{
    if (ctx->dim == 3) return ctx->opt.tile_g == 1 ? 1 : 2;
    const int cap = source_mode(ctx) == 0 ? 2 : 4;  // dense mode: registers for 2 ordinates
    if (ctx->opt.tile_g == 1 || ctx->opt.tile_g == 2 || ctx->opt.tile_g == 4)
        return std::min(ctx->opt.tile_g, cap);
    if (ctx->opt.tile_g == -1 && ctx->tuned_g > 0) return std::min(ctx->tuned_g, cap);
    // largest G that still gives at least two work items per SM
    for (int G : {4, 2}) {
        if (G > cap) continue;
        long long n = 0;
        for (int s = 0; s < ctx->S; ++s) n += 4 * ((ctx->M[s] / 4 + G - 1) / G);
        if (n >= 2LL * ctx->sm_count) return G;
    }
    return 1;
}

// 3D: work items of G = 2 ordinates of one sample and octant (1 with tile_g =
// 1); CTAs take strided lists of the items of one octant (consecutive CTAs of
// an octant work on neighbouring items, hence on the same few samples at a
// time); CTAs per octant in proportion to its items.
int build_items3(rom_ctx *ctx)
{
    const int G = ctx->opt.tile_g == 1 ? 1 : 2;
    ctx->G_used = G;
    ctx->items.clear();
    std::vector<int> byo[8];
    for (int s = 0; s < ctx->S; ++s) {
        std::vector<int> ords[8];
        for (int l = 0; l < ctx->M[s]; ++l) {
            const long long o = ctx->off[s] + l;
            int code;
            if (ctx->ord_source == ORD_SEED) {
                // generated blocks of m: (+,+), (-,+), (-,-), (+,-), then (3D) the same with zeta < 0
                const int m = ctx->M[s] / (ctx->seed_octants ? 8 : 4);
                const int qd = l / m;
                const int q4 = qd & 3;
                code = (q4 == 0 ? 0 : q4 == 1 ? 1 : q4 == 2 ? 3 : 2) | (qd >= 4 ? 4 : 0);
            } else {
                code = ctx->quad[o];
            }
            ords[code].push_back((int)o);
        }
        for (int code = 0; code < 8; ++code)
            for (size_t k = 0; k < ords[code].size(); k += G) {
                SweepItem it{};
                it.sample = s;
                it.quad = code;
                it.n = (int)std::min<size_t>(G, ords[code].size() - k);
                for (int t = 0; t < romk::kMaxG; ++t)
                    it.ord[t] = ords[code][k + (t < it.n ? t : 0)];
                byo[code].push_back((int)ctx->items.size());
                ctx->items.push_back(it);
            }
    }
    const long long total = (long long)ctx->items.size();
    const int L = (ctx->I + romk::kCols - 1) / romk::kCols;
    const int strips = romk::sweep3d_tile_cols() / romk::kCols;
    ctx->nwarps3 = std::min(strips, L);
    ctx->n_tx = (L + strips - 1) / strips;
    ctx->n_ty = (ctx->J + 127) / 128;
    const int grid = ctx->sm_count * romk::sweep3d_ctas_per_sm(ctx->nwarps3, G);
    ctx->cta_begin.assign(1, 0);
    ctx->cta_list.clear();
    for (int code = 0; code < 8; ++code) {
        const std::vector<int> &v = byo[code];
        if (v.empty()) continue;
        long long P = std::max<long long>(1, (long long)llround((double)grid * v.size() / total));
        P = std::min<long long>(P, (long long)v.size());
        P = std::max<long long>(P, ((long long)v.size() + romk::kMaxCtaItems3 - 1) / romk::kMaxCtaItems3);
        for (long long b = 0; b < P; ++b) {
            for (long long k = b; k < (long long)v.size(); k += P) ctx->cta_list.push_back(v[k]);
            ctx->cta_begin.push_back((int)ctx->cta_list.size());
        }
    }
    ctx->n_ctas3 = (int)ctx->cta_begin.size() - 1;
    int rc;
    if ((rc = ensure(ctx, ctx->items_dev, ctx->items.size() * sizeof(SweepItem))) ||
        (rc = ensure(ctx, ctx->cta_begin_dev, ctx->cta_begin.size() * sizeof(int))) ||
        (rc = ensure(ctx, ctx->cta_list_dev, ctx->cta_list.size() * sizeof(int))) ||
        (rc = ensure(ctx, ctx->err3, sizeof(int))))
        return rc;
    if (ctx->n_tx > 1 &&
        (rc = ensure(ctx, ctx->xface, (size_t)total * G * ctx->K * ctx->J * sizeof(float))))
        return rc;
    if (ctx->n_ty > 1 &&
        (rc = ensure(ctx, ctx->yface, (size_t)total * G * ctx->K * ctx->NXP * sizeof(float))))
        return rc;
    if (!ctx->items.empty())
        CK(cudaMemcpyAsync(ctx->items_dev.p, ctx->items.data(), ctx->items.size() * sizeof(SweepItem),
                           cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->cta_begin_dev.p, ctx->cta_begin.data(),
                       ctx->cta_begin.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    if (!ctx->cta_list.empty())
        CK(cudaMemcpyAsync(ctx->cta_list_dev.p, ctx->cta_list.data(),
                           ctx->cta_list.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->items_dirty = false;
    return ROM_OK;
}

// Batches of several grids: the grid and state offset of every sample and the
// device tables of the grids (GridDesc), samples (grid, offset) and cell areas.
int build_batch_tables(rom_ctx *ctx)
{
    long long tot = 0;
    for (int p = 0; p < ctx->n_grids; ++p) tot += ctx->grid_samples[p];
    if (tot != ctx->S)
        return fail(ctx, ROM_ERR_STATE,
                    "the grids hold %lld samples, the ordinate sets %d: set them to agree", tot,
                    ctx->S);
    const int MOM = ctx->MOM == 0 ? 1 : ctx->MOM;
    ctx->sgrid.assign(ctx->S, 0);
    ctx->soff.assign(ctx->S, 0);
    std::vector<double> sdA(ctx->S);
    long long off = 0;
    int s = 0;
    for (int p = 0; p < ctx->n_grids; ++p)
        for (int k = 0; k < ctx->grid_samples[p]; ++k, ++s) {
            const romk::GridDesc &g = ctx->grids[p];
            ctx->sgrid[s] = p;
            ctx->soff[s] = off;
            off += (long long)MOM * g.cells;
            sdA[s] = (double)g.dx * g.dy;
        }
    ctx->state_floats = off;
    int rc;
    if ((rc = ensure(ctx, ctx->gdesc, ctx->grids.size() * sizeof(romk::GridDesc))) ||
        (rc = ensure(ctx, ctx->sgrid_dev, ctx->S * sizeof(int))) ||
        (rc = ensure(ctx, ctx->soff_dev, ctx->S * sizeof(long long))) ||
        (rc = ensure(ctx, ctx->sdA_dev, ctx->S * sizeof(double))))
        return rc;
    CK(cudaMemcpyAsync(ctx->gdesc.p, ctx->grids.data(), ctx->grids.size() * sizeof(romk::GridDesc),
                       cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->sgrid_dev.p, ctx->sgrid.data(), ctx->S * sizeof(int),
                       cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->soff_dev.p, ctx->soff.data(), ctx->S * sizeof(long long),
                       cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->sdA_dev.p, sdA.data(), ctx->S * sizeof(double),
                       cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));  // the host vectors may change before the next use
    return ROM_OK;
}

int build_items(rom_ctx *ctx)
{
    if (ctx->dim == 3) return build_items3(ctx);
    if (batch(ctx)) {
        int rc = build_batch_tables(ctx);
        if (rc) return rc;
    }
    const int G = choose_g(ctx);
    ctx->G_used = G;
    ctx->H_used = choose_rows(ctx);
    ctx->items.clear();
    std::vector<int> byq[4];
    for (int s = 0; s < ctx->S; ++s) {
        for (int qd = 0; qd < 4; ++qd) byq[qd].clear();
        if (ctx->ord_source == ORD_SEED) {
            const int nblk = ctx->seed_octants ? 8 : 4;
            const int m = ctx->M[s] / nblk;
            for (int qd = 0; qd < nblk; ++qd)
                for (int l = 0; l < m; ++l) {
                    // quadrant blocks of the generated set: (+,+), (-,+), (-,-), (+,-)
                    // (3D sets repeat them with zeta < 0; X-Y sweeps ignore zeta)
                    const int q4 = qd & 3;
                    const int code = q4 == 0 ? 0 : q4 == 1 ? 1 : q4 == 2 ? 3 : 2;
                    byq[code].push_back((int)(ctx->off[s] + (long long)qd * m + l));
                }
        } else {
            for (int l = 0; l < ctx->M[s]; ++l) {
                const long long o = ctx->off[s] + l;
                byq[ctx->quad[o] & 3].push_back((int)o);
            }
        }
        for (int code = 0; code < 4; ++code) {
            const std::vector<int> &v = byq[code];
            for (size_t k = 0; k < v.size(); k += G) {
                SweepItem it{};
                it.sample = s;
                it.quad = code;
                it.n = (int)std::min<size_t>(G, v.size() - k);
                for (int t = 0; t < romk::kMaxG; ++t) it.ord[t] = t < it.n ? v[k + t] : v[k];
                it.grid = batch(ctx) ? ctx->sgrid[s] : 0;
                ctx->items.push_back(it);
            }
        }
    }
    int rc;
    if ((rc = ensure(ctx, ctx->items_dev, ctx->items.size() * sizeof(SweepItem)))) return rc;
    if (!ctx->items.empty())
        CK(cudaMemcpyAsync(ctx->items_dev.p, ctx->items.data(), ctx->items.size() * sizeof(SweepItem),
                           cudaMemcpyHostToDevice, ctx->stream));
    // first ordinate and count per sample ([S] long long, [S] int), for the
    // per-sample weight sums of the balance
    const size_t tb = (size_t)ctx->S * (sizeof(long long) + sizeof(int));
    if ((rc = ensure(ctx, ctx->otab, tb))) return rc;
    std::vector<unsigned char> h(tb);
    memcpy(h.data(), ctx->off.data(), ctx->S * sizeof(long long));
    memcpy(h.data() + ctx->S * sizeof(long long), ctx->M.data(), ctx->S * sizeof(int));
    CK(cudaMemcpyAsync(ctx->otab.p, h.data(), tb, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));  // host vectors may change before the next use
    ctx->items_dirty = false;
    return ROM_OK;
}

int upload_inflow(rom_ctx *ctx)
{
    bool any_ord = false, any_iso = false;
    const int NF = n_faces(ctx);
    for (int f = 0; f < NF; ++f) {
        any_ord |= !ctx->inflow_ord[f].empty();
        any_iso |= !ctx->inflow_iso[f].empty();
    }
    const long long nface = face_offset(ctx, NF);
    ctx->inflow_any = any_ord || any_iso;
    if (!ctx->inflow_any) {
        ctx->inflow_dirty = false;
        return ROM_OK;
    }
    const long long rows = any_ord ? ctx->Mtot : 1;
    ctx->inflow_stride = any_ord ? nface : 0;
    std::vector<float> h((size_t)(rows * nface), 0.f);
    for (long long o = 0; o < rows; ++o)
        for (int f = 0; f < NF; ++f) {
            const long long nf = face_cells(ctx, f), fo = face_offset(ctx, f);
            for (long long k = 0; k < nf; ++k) {
                double v = 0.0;
                if (!ctx->inflow_ord[f].empty()) v = ctx->inflow_ord[f][(size_t)o * nf + k];
                else if (!ctx->inflow_iso[f].empty()) v = ctx->inflow_iso[f][k];
                h[(size_t)(o * nface + fo + k)] = (float)v;
            }
        }
    int rc = ensure(ctx, ctx->inflow_dev, h.size() * sizeof(float));
    if (rc) return rc;
    CK(cudaMemcpyAsync(ctx->inflow_dev.p, h.data(), h.size() * sizeof(float),
                       cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->inflow_dirty = false;
    return ROM_OK;
}

romk::SweepArgs sweep_args(const rom_ctx *ctx)
{
    romk::SweepArgs a{};
    a.I = ctx->I;
    a.J = ctx->J;
    a.NXP = ctx->NXP;
    a.inv_dx = (float)(ctx->I / (ctx->hi[0] - ctx->lo[0]));
    a.inv_dy = (float)(ctx->J / (ctx->hi[1] - ctx->lo[1]));
    a.sigma_t_homog = ctx->sigma_t_homog;
    a.sigma_t = (const float *)ctx->sigt.p;
    a.src = (const float *)ctx->src.p;
    a.part = (float *)ctx->part.p;
    a.items = (const SweepItem *)ctx->items_dev.p;
    a.oc = (const float *)ctx->c32.p;
    a.os = (const float *)ctx->s32.p;
    a.ow = (const float *)ctx->w32.p;
    a.inflow = ctx->inflow_any ? (const float *)ctx->inflow_dev.p : nullptr;
    a.inflow_stride = ctx->inflow_stride;
    a.active = (const int *)ctx->active.p;
    a.cells = (long long)ctx->J * ctx->NXP;
    if (batch(ctx)) {
        a.grids = (const romk::GridDesc *)ctx->gdesc.p;
        a.soff = (const long long *)ctx->soff_dev.p;
    }
    a.leak = has_balance(ctx) ? (double *)ctx->leak.p : nullptr;
    a.dx = (float)((ctx->hi[0] - ctx->lo[0]) / ctx->I);
    a.dy = (float)((ctx->hi[1] - ctx->lo[1]) / ctx->J);
    a.err = (int *)ctx->sweep_err.p;
    a.wait_ns = (unsigned long long)(ctx->opt.wait_timeout_ms * 1e6);
    a.stall = ctx->opt.test_stall_waits;
    if (ctx->MOM == 0) {
        a.src = (const float *)ctx->src_ord.p;
        if (ctx->opt.dense_precision == 1) {
            a.psi_split = (uint32_t *)ctx->psi_split.p;
        } else {
            a.psi = (float *)ctx->psi.p;
        }
    }
    return a;
}

romk::Sweep3Args sweep3_args(const rom_ctx *ctx)
{
    romk::Sweep3Args a{};
    a.I = ctx->I;
    a.J = ctx->J;
    a.K = ctx->K;
    a.NXP = ctx->NXP;
    a.inv_dx = (float)(ctx->I / (ctx->hi[0] - ctx->lo[0]));
    a.inv_dy = (float)(ctx->J / (ctx->hi[1] - ctx->lo[1]));
    a.inv_dz = (float)(ctx->K / (ctx->hi[2] - ctx->lo[2]));
    a.sk = romk::make_skew3(ctx->J, ctx->K, ctx->NXP);
    a.sigma_t = (const float *)ctx->sig3.p;
    a.src = (const float *)ctx->src3.p;
    a.phi = (float *)ctx->acc3.p;
    a.S = ctx->S;
    a.items = (const SweepItem *)ctx->items_dev.p;
    a.cta_begin = (const int *)ctx->cta_begin_dev.p;
    a.cta_list = (const int *)ctx->cta_list_dev.p;
    a.oc = (const float *)ctx->c32.p;
    a.os = (const float *)ctx->s32.p;
    a.oz = (const float *)ctx->z32.p;
    a.ow = (const float *)ctx->w32.p;
    a.inflow = ctx->inflow_any ? (const float *)ctx->inflow_dev.p : nullptr;
    a.inflow_stride = ctx->inflow_stride;
    a.active = (const int *)ctx->active.p;
    a.cells = padded_cells(ctx);
    a.n_tx = ctx->n_tx;
    a.n_ty = ctx->n_ty;
    a.xface = (float *)ctx->xface.p;
    a.yface = (float *)ctx->yface.p;
    a.err = (int *)ctx->err3.p;
    a.wait_ns = (unsigned long long)(ctx->opt.wait_timeout_ms * 1e6);
    a.stall = ctx->opt.test_stall_waits;
    return a;
}

int max_m(const rom_ctx *ctx)
{
    int m = 0;
    for (int v : ctx->M) m = std::max(m, v);
    return m;
}

// device tables of the dense operator: M [S] int, ord_off [S], a_off [S] (long long)
struct DenseTab {
    const int *M;
    const long long *ord_off, *a_off;
};

DenseTab dense_tab(const rom_ctx *ctx)
{
    const unsigned char *b = (const unsigned char *)ctx->dtab.p;
    const size_t S = ctx->S;
    DenseTab t;
    t.ord_off = (const long long *)b;
    t.a_off = (const long long *)(b + S * 8);
    t.M = (const int *)(b + S * 16);
    return t;
}

romk::DenseArgs dense_args(const rom_ctx *ctx)
{
    const DenseTab t = dense_tab(ctx);
    romk::DenseArgs d{};
    d.S = ctx->S;
    d.M = t.M;
    d.ord_off = t.ord_off;
    d.a_off = t.a_off;
    d.A = (const float *)ctx->Amat.p;
    d.psi = (const float *)ctx->psi.p;
    d.src = (float *)ctx->src_ord.p;
    d.sigma_s = (const float *)ctx->sigs.p;
    d.q = (const float *)ctx->q.p;
    d.cells = (long long)ctx->J * ctx->NXP;
    d.active = (const int *)ctx->active.p;
    return d;
}

// Buffers, tables and the operator A of the dense mode (A once per ordinate set).
int prepare_dense(rom_ctx *ctx)
{
    const long long cells = (long long)ctx->J * ctx->NXP;
    const bool tc = ctx->opt.dense_precision == 1;
    int rc;
    if (tc && max_m(ctx) > romk::dense_tc_max_m())
        return fail(ctx, ROM_ERR_UNSUPPORTED,
                    "dense_precision = 1 (tensor cores) needs at most %d ordinates per sample",
                    romk::dense_tc_max_m());
    if (tc && ctx->S > romk::dense_tc_max_samples())
        return fail(ctx, ROM_ERR_UNSUPPORTED,
                    "dense_precision = 1 (tensor cores) takes at most %d samples per context",
                    romk::dense_tc_max_samples());
    if ((rc = ensure(ctx, ctx->src_ord, (size_t)ctx->Mtot * cells * sizeof(float)))) return rc;
    if (tc) {
        const size_t split = (size_t)ctx->Mtot * cells * 4;  // BF16 hi + lo
        const size_t ab = (size_t)ctx->S * 128 * 128 * 2;
        if ((rc = ensure(ctx, ctx->psi_split, split)) || (rc = ensure(ctx, ctx->a_hi, ab)) ||
            (rc = ensure(ctx, ctx->a_lo, ab)) || (rc = ensure(ctx, ctx->tc_err, sizeof(int))))
            return rc;
        const void *ptrs[3] = {ctx->a_hi.p, ctx->a_lo.p, ctx->psi_split.p};
        if (memcmp(ptrs, ctx->tc_map_ptrs, sizeof ptrs) != 0 || ctx->tc_map_cells != cells ||
            ctx->tc_map_mtot != ctx->Mtot || ctx->tc_map_S != ctx->S) {
            CK(romk::make_dense_tc_maps(&ctx->tc_maps, ctx->a_hi.p, ctx->a_lo.p, ctx->S,
                                        ctx->psi_split.p, ctx->Mtot, cells));
            memcpy(ctx->tc_map_ptrs, ptrs, sizeof ptrs);
            ctx->tc_map_cells = cells;
            ctx->tc_map_mtot = ctx->Mtot;
            ctx->tc_map_S = ctx->S;
            invalidate_graph(ctx);
        }
    } else if ((rc = ensure(ctx, ctx->psi, (size_t)ctx->Mtot * cells * sizeof(float)))) {
        return rc;
    }
    if (!ctx->pmat_dirty) return ROM_OK;
    std::vector<long long> a_off(ctx->S);
    long long asz = 0;
    for (int s = 0; s < ctx->S; ++s) {
        a_off[s] = asz;
        asz += (long long)ctx->M[s] * ctx->M[s];
    }
    const size_t tb = (size_t)ctx->S * 20;
    if ((rc = ensure(ctx, ctx->Amat, (size_t)asz * sizeof(float))) || (rc = ensure(ctx, ctx->dtab, tb)))
        return rc;
    std::vector<unsigned char> h(tb);
    memcpy(h.data(), ctx->off.data(), ctx->S * 8);
    memcpy(h.data() + ctx->S * 8, a_off.data(), ctx->S * 8);
    memcpy(h.data() + ctx->S * 16, ctx->M.data(), ctx->S * 4);
    CK(cudaMemcpyAsync(ctx->dtab.p, h.data(), tb, cudaMemcpyHostToDevice, ctx->stream));
    const DenseTab t = dense_tab(ctx);
    romk::PmatArgs pa{};
    pa.S = ctx->S;
    pa.M = t.M;
    pa.ord_off = t.ord_off;
    pa.a_off = t.a_off;
    pa.c = (const double *)ctx->c64.p;
    pa.s = (const double *)ctx->s64.p;
    pa.z = (const double *)ctx->z64.p;
    pa.w = (const double *)ctx->w64.p;
    pa.kind = ctx->kernel_kind;
    pa.g = ctx->g;
    pa.raw = (ctx->kernel_flags & ROM_KERNEL_FLAG_RAW) ? 1 : 0;
    pa.normalize = (ctx->kernel_flags & ROM_KERNEL_FLAG_NORMALIZE) ? 1 : 0;
    pa.A = (float *)ctx->Amat.p;
    CK(romk::launch_pmat(pa, max_m(ctx), ctx->stream));
    ++ctx->launches;
    if (tc) {  // A -> A_hi, A_lo (BF16, 128 x 128 per sample, zero padded)
        CK(romk::launch_pmat_split((const float *)ctx->Amat.p, t.M, t.a_off, ctx->S, ctx->a_hi.p,
                                   ctx->a_lo.p, ctx->stream));
        ++ctx->launches;
    }
    CK(cudaStreamSynchronize(ctx->stream));  // the host table dies with this call
    ctx->pmat_dirty = false;
    return ROM_OK;
}

// One X-Y sweep launch with work items of G ordinates and H rows per step: one CTA
// per item, as many warps as the widest grid needs.
cudaError_t launch_xy_sweep(const rom_ctx *ctx, const romk::SweepArgs &sa, int G, int H,
                            cudaStream_t st)
{
    const int L = (ctx->I + romk::kCols - 1) / romk::kCols;
    const int nwarps = (L + 31) / 32;
    if (H == 1) {
        if (batch(ctx))
            return romk::launch_sweep2d_row_batch(sa, (int)ctx->items.size(), nwarps, G,
                                                  ctx->opt.scheme, ctx->MOM, st);
        return romk::launch_sweep2d_row(sa, (int)ctx->items.size(), nwarps, G, ctx->opt.scheme,
                                        ctx->homog, ctx->MOM, st);
    }
    if (batch(ctx))
        return romk::launch_sweep2d_batch(sa, (int)ctx->items.size(), nwarps, G, ctx->opt.scheme,
                                          ctx->MOM, H, st);
    return romk::launch_sweep2d(sa, (int)ctx->items.size(), nwarps, G, ctx->opt.scheme,
                                ctx->homog, ctx->MOM, H, st);
}

int launches_per_iteration(const rom_ctx *ctx)
{
    if (ctx->dim == 3) return ctx->n_tx * ctx->n_ty + 2;
    return ctx->MOM == 0 ? 4 : 3;
}

// One source-iteration sweep: K1 (K9 per tile in 3D) + K2 (+ K4 in dense mode) + K5.
int enqueue_iteration(rom_ctx *ctx, cudaStream_t st, bool use_cond, cudaGraphConditionalHandle h,
                      cudaEvent_t k0 = nullptr, cudaEvent_t k1 = nullptr,
                      cudaEvent_t k2 = nullptr, cudaEvent_t k3 = nullptr)
{
    if (k0) CK(cudaEventRecord(k0, st));
    if (ctx->dim == 3) {
        romk::Sweep3Args a3 = sweep3_args(ctx);
        for (int ty = 0; ty < ctx->n_ty; ++ty)
            for (int tx = 0; tx < ctx->n_tx; ++tx) {
                a3.tile_x = tx;
                a3.tile_y = ty;
                CK(romk::launch_sweep3d(a3, ctx->n_ctas3, ctx->nwarps3, ctx->G_used,
                                        ctx->opt.scheme, st));
            }
    } else {
        CK(launch_xy_sweep(ctx, sweep_args(ctx), ctx->G_used, ctx->H_used, st));
    }
    if (k1) CK(cudaEventRecord(k1, st));
    romk::CombineArgs ca{};
    ca.S = ctx->S;
    ca.I = ctx->I;
    ca.NXP = ctx->NXP;
    ca.MOM = ctx->MOM == 0 ? 1 : ctx->MOM;
    // about four combine blocks per SM over the whole launch (the launcher evens out
    // the passes per thread)
    ca.chunks = (int)std::max<long long>(1, (4LL * ctx->sm_count + ctx->S - 1) / ctx->S);
    ca.cells = padded_cells(ctx);
    ca.g = (float)ctx->g;
    ca.acc = (float *)ctx->part.p;
    ca.phi = (float *)ctx->phi.p;
    ca.src = (float *)ctx->src.p;
    ca.sigma_s = (const float *)ctx->sigs.p;
    ca.q = (const float *)ctx->q.p;
    ca.active = (const int *)ctx->active.p;
    ca.sums = (double *)ctx->sums.p;
    ca.minkey = (int *)ctx->minkey.p;
    ca.balance = has_balance(ctx) ? 1 : 0;
    ca.sigma_t = ctx->homog ? nullptr : (const float *)ctx->sigt.p;
    ca.sigma_t_homog = ctx->sigma_t_homog;
    if (batch(ctx)) {
        ca.grids = (const romk::GridDesc *)ctx->gdesc.p;
        ca.sgrid = (const int *)ctx->sgrid_dev.p;
        ca.soff = (const long long *)ctx->soff_dev.p;
        ca.cells = ctx->max_cells;
    }
    if (ctx->dim == 3) {
        romk::Combine3Args c3{};
        c3.S = ctx->S;
        c3.chunks = ctx->chunks;
        c3.sk = romk::make_skew3(ctx->J, ctx->K, ctx->NXP);
        c3.acc = (float *)ctx->acc3.p;
        c3.src = (float *)ctx->src3.p;
        c3.phi = (float *)ctx->phi.p;
        c3.sigma_s = (const float *)ctx->ss3.p;
        c3.q = (const float *)ctx->q3.p;
        c3.active = (const int *)ctx->active.p;
        c3.sums = (double *)ctx->sums.p;
        c3.minkey = (int *)ctx->minkey.p;
        c3.I = ctx->I;
        CK(romk::launch_combine3(c3, st));
    } else {
        CK(romk::launch_combine(ca, st));
    }
    if (ctx->MOM == 0) {
        if (k2) CK(cudaEventRecord(k2, st));
        if (ctx->opt.dense_precision == 1) {
            const romk::DenseArgs d = dense_args(ctx);
            romk::DenseTcArgs ta{};
            ta.S = ctx->S;
            ta.M = d.M;
            ta.ord_off = d.ord_off;
            ta.cells = d.cells;
            ta.sigma_s = d.sigma_s;
            ta.q = d.q;
            ta.src = d.src;
            ta.active = d.active;
            ta.err = (int *)ctx->tc_err.p;
            CK(romk::launch_dense_tc(ctx->tc_maps, ta, ctx->sm_count, st));
        } else {
            CK(romk::launch_dense_source(dense_args(ctx), max_m(ctx), st));
        }
        if (k3) CK(cudaEventRecord(k3, st));
    }
    romk::FinalizeArgs fa{};
    fa.S = ctx->S;
    fa.chunks = ctx->chunks;
    fa.fixed_iters = ctx->opt.fixed_iters;
    fa.max_iter = ctx->opt.max_iter;
    fa.tol = ctx->opt.tol;
    fa.sums = (double *)ctx->sums.p;
    fa.minkey = (int *)ctx->minkey.p;
    fa.active = (int *)ctx->active.p;
    fa.iters = (int *)ctx->iters.p;
    fa.flags = (int *)ctx->flags.p;
    fa.resid = (double *)ctx->resid.p;
    fa.diverge_window = ctx->opt.diverge_window;
    fa.dprev = (double *)ctx->dprev.p;
    fa.grow = (int *)ctx->grow.p;
    fa.balance = has_balance(ctx) ? 1 : 0;
    fa.leak = (double *)ctx->leak.p;
    fa.dA = (ctx->hi[0] - ctx->lo[0]) / ctx->I * (ctx->hi[1] - ctx->lo[1]) / ctx->J;
    fa.sdA = batch(ctx) ? (const double *)ctx->sdA_dev.p : nullptr;
    fa.ordsum = (const double *)ctx->ordsum.p;
    fa.bal_out = (double *)ctx->bal.p;
    fa.leak_out = (double *)ctx->leak_out.p;
    fa.phimin_out = (double *)ctx->phimin.p;
    fa.n_active = (int *)ctx->n_active.p;
    fa.use_cond = use_cond ? 1 : 0;
    fa.cond = h;
    CK(romk::launch_finalize(fa, st));
    return ROM_OK;
}

int ensure_state(rom_ctx *ctx);
int init_state(rom_ctx *ctx);

// tile_g = -1: time the sweep kernel of every candidate work-item size G and
// rows per wavefront step H (1 and 2 only in the moment modes) on the current
// problem (three sweeps after one warm-up, from the initial source) and keep the
// fastest.
int autotune_g(rom_ctx *ctx)
{
    const int cap = source_mode(ctx) == 0 ? 2 : 4;
    float best_ms = 0.f;
    int best = 0, best_h = 4, rc;
    const bool dense = source_mode(ctx) == 0;
    // 0: every H (dense operator mode: 1 and 4; 2 there means 4)
    const int want_h = dense && ctx->opt.rows_per_step == 2 ? 4 : ctx->opt.rows_per_step;
    for (int cand = 0; cand < 9; ++cand) {
        const int G = 1 << (cand / 3), H = 1 << (cand % 3);  // H = 1, 2, 4
        if (G > cap || (want_h != 0 && H != want_h) || (dense && H == 2)) continue;
        ctx->opt.tile_g = G;
        if ((rc = build_items(ctx))) return rc;
        if ((rc = ensure_state(ctx))) return rc;  // phi, sources, accumulators
        if ((rc = init_state(ctx))) return rc;
        const romk::SweepArgs sa = sweep_args(ctx);
        for (int rep = 0; rep < 4; ++rep) {
            if (rep == 1) CK(cudaEventRecord(ctx->ev0, ctx->stream));
            CK(launch_xy_sweep(ctx, sa, G, H, ctx->stream));
            ++ctx->launches;
        }
        CK(cudaEventRecord(ctx->ev1, ctx->stream));
        CK(cudaEventSynchronize(ctx->ev1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
        if (best == 0 || ms < best_ms) {
            best = G;
            best_h = H;
            best_ms = ms;
        }
    }
    ctx->opt.tile_g = -1;
    ctx->tuned_g = best;
    ctx->tuned_h = best_h;
    ctx->items_dirty = true;
    return ROM_OK;
}

// Per-sample state arrays of the current layout -- phi, the source moments and
// the sweep's accumulators in row-major (dense operator mode), sheared (X-Y
// moment modes) or diagonal (3D) storage -- and the sheared coefficient copies.
int ensure_state(rom_ctx *ctx)
{
    int rc;
    const int MOM = ctx->MOM == 0 ? 1 : ctx->MOM;
    const size_t S = ctx->S;
    if (ctx->dim == 3) {
        const romk::Skew3 sk = romk::make_skew3(ctx->J, ctx->K, ctx->NXP);
        if (sk.cells >= (1LL << 31))
            return fail(ctx, ROM_ERR_UNSUPPORTED, "3D grid too large for one sample's arrays");
        const size_t b = (size_t)sk.cells * sizeof(float);
        if ((rc = ensure(ctx, ctx->sig3, 2 * b)) || (rc = ensure(ctx, ctx->src3, 2 * S * b)) ||
            (rc = ensure(ctx, ctx->acc3, 2 * S * b)) || (rc = ensure(ctx, ctx->ss3, b)) ||
            (rc = ensure(ctx, ctx->q3, b)) || (rc = ensure(ctx, ctx->phi, S * b)))
            return rc;
        return ROM_OK;
    }
    // [S][MOM][J][NXP], or each sample's [MOM][J_p][NXP_p] block of its grid
    const size_t b = (batch(ctx) ? (size_t)ctx->state_floats
                                 : S * MOM * (size_t)padded_cells(ctx)) * sizeof(float);
    if ((rc = ensure(ctx, ctx->phi, b)) || (rc = ensure(ctx, ctx->src, b)) ||
        (rc = ensure(ctx, ctx->part, b)))
        return rc;
    return ROM_OK;
}

// Device state of a new solve, on the context stream: phi^0 = 0, the first
// source q (psi^0 = 0), cleared accumulators and error words, every sample
// active, the coefficient copies of the layout, the divergence and balance
// state, and the per-sample weight sums of the balance.
int init_state(rom_ctx *ctx)
{
    const int MOM = ctx->MOM == 0 ? 1 : ctx->MOM;
    const long long cells = padded_cells(ctx);
    cudaStream_t st = ctx->stream;
    if (ctx->MOM == 0 && ctx->opt.dense_precision == 1)
        CK(cudaMemsetAsync(ctx->tc_err.p, 0, sizeof(int), st));
    CK(cudaMemsetAsync(ctx->sweep_err.p, 0, sizeof(int), st));
    if (ctx->dim == 3) {
        // diagonal storage: sigma_T (both families), the first source q of every
        // sample, sigma_S and q for the combine (family 0), cleared accumulators, phi = 0
        const romk::Skew3 sk = romk::make_skew3(ctx->J, ctx->K, ctx->NXP);
        CK(cudaMemsetAsync(ctx->err3.p, 0, sizeof(int), st));
        CK(cudaMemsetAsync(ctx->acc3.p, 0, 2 * (size_t)ctx->S * sk.cells * sizeof(float), st));
        CK(romk::launch_skew3_scatter((const float *)ctx->sigt.p, sk, ctx->NXP, 2, 1,
                                      (float *)ctx->sig3.p, st));
        CK(romk::launch_skew3_scatter((const float *)ctx->q.p, sk, ctx->NXP, 2, ctx->S,
                                      (float *)ctx->src3.p, st));
        CK(romk::launch_skew3_scatter((const float *)ctx->sigs.p, sk, ctx->NXP, 1, 1,
                                      (float *)ctx->ss3.p, st));
        CK(romk::launch_skew3_scatter((const float *)ctx->q.p, sk, ctx->NXP, 1, 1,
                                      (float *)ctx->q3.p, st));
        ctx->launches += 4;
        CK(romk::launch_init_state(ctx->S, 1, sk.cells, nullptr, (float *)ctx->phi.p, nullptr,
                                   (int *)ctx->active.p, (int *)ctx->iters.p, (int *)ctx->flags.p,
                                   (double *)ctx->resid.p, st));
    } else if (batch(ctx)) {
        CK(cudaMemsetAsync(ctx->part.p, 0, (size_t)ctx->state_floats * sizeof(float), st));
        CK(romk::launch_init_state(ctx->S, MOM, 0, nullptr, nullptr, nullptr, (int *)ctx->active.p,
                                   (int *)ctx->iters.p, (int *)ctx->flags.p,
                                   (double *)ctx->resid.p, st));
        CK(romk::launch_init_grids(ctx->S, MOM, (const romk::GridDesc *)ctx->gdesc.p,
                                   (const int *)ctx->sgrid_dev.p, (const long long *)ctx->soff_dev.p,
                                   (int)ctx->max_cells, (const float *)ctx->q.p,
                                   (float *)ctx->phi.p, (float *)ctx->src.p, st));
        ++ctx->launches;
    } else {
        // the sweep accumulates into part; the combine clears it
        CK(cudaMemsetAsync(ctx->part.p, 0, (size_t)ctx->S * MOM * cells * sizeof(float), st));
        CK(romk::launch_init_state(ctx->S, MOM, cells, (const float *)ctx->q.p,
                                   (float *)ctx->phi.p, (float *)ctx->src.p, (int *)ctx->active.p,
                                   (int *)ctx->iters.p, (int *)ctx->flags.p,
                                   (double *)ctx->resid.p, st));
    }
    ++ctx->launches;
    if (ctx->MOM == 0) {  // psi^0 = 0: every ordinate's first source is q
        CK(romk::launch_dense_init((const float *)ctx->q.p, cells, ctx->Mtot,
                                   (float *)ctx->src_ord.p, st));
        ++ctx->launches;
    }
    CK(romk::launch_init_checks(ctx->S, (double *)ctx->dprev.p, (int *)ctx->grow.p,
                                (double *)ctx->leak.p, (double *)ctx->bal.p,
                                (double *)ctx->leak_out.p, (double *)ctx->phimin.p,
                                (double *)ctx->sums.p, (int *)ctx->minkey.p, st));
    ++ctx->launches;
    if (has_balance(ctx)) {
        const unsigned char *ot = (const unsigned char *)ctx->otab.p;
        CK(romk::launch_ordsum((const double *)ctx->c64.p, (const double *)ctx->s64.p,
                               (const double *)ctx->w64.p, (const long long *)ot,
                               (const int *)(ot + ctx->S * sizeof(long long)), ctx->S,
                               (double *)ctx->ordsum.p, st));
        ++ctx->launches;
    }
    return ROM_OK;
}

int build_graph(rom_ctx *ctx)
{
    invalidate_graph(ctx);
    CK(cudaGraphCreate(&ctx->graph, 0));
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, ctx->graph, 1, cudaGraphCondAssignDefault));
    // the struct has a union with a deleted default constructor: zero raw storage
    alignas(cudaGraphNodeParams) unsigned char np_raw[sizeof(cudaGraphNodeParams)];
    memset(np_raw, 0, sizeof np_raw);
    cudaGraphNodeParams &np = *reinterpret_cast<cudaGraphNodeParams *>(np_raw);
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, ctx->graph, nullptr, nullptr, 0, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    // capture on the context's private stream (capturable even when the user
    // stream is the legacy default stream)
    CK(cudaStreamBeginCaptureToGraph(ctx->own_stream, body, nullptr, nullptr, 0,
                                     cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_iteration(ctx, ctx->own_stream, true, h);
    cudaGraph_t captured = nullptr;
    cudaError_t e = cudaStreamEndCapture(ctx->own_stream, &captured);
    if (rc) return rc;
    if (e != cudaSuccess)
        return fail(ctx, ROM_ERR_CUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
    CK(cudaGraphInstantiate(&ctx->graph_exec, ctx->graph, 0));
    ctx->graph_valid = true;
    return ROM_OK;
}

}  // namespace

// =========================================================== public ABI

extern "C" {

const char *rom_version(void) { return "rom-gb300 0.1.0 (sm_103a)"; }

void rom_default_options(rom_options *opt)
{
    if (!opt) return;
    memset(opt, 0, sizeof *opt);
    opt->scheme = ROM_SCHEME_DD;
    opt->max_iter = 10000;
    opt->tol = 1e-6;
    opt->fixed_iters = 0;
    opt->check_every = 0;
    opt->tile_g = 0;
    opt->time_kernels = 0;
    opt->dense_source = 0;
    opt->dense_precision = 0;
    opt->rows_per_step = 0;
    opt->diverge_window = 16;
    opt->wait_timeout_ms = 2000.0;
    opt->test_stall_waits = 0;
}

int rom_create(rom_ctx **out, int cuda_device)
{
    if (!out) return ROM_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cuda_device < 0 || cuda_device >= ndev) {
        (void)cudaGetLastError();
        return ROM_ERR_INVALID_ARG;
    }
    rom_ctx *ctx = new (std::nothrow) rom_ctx();
    if (!ctx) return ROM_ERR_OOM;
    ctx->device = cuda_device;
    rom_default_options(&ctx->opt);
    if (cudaSetDevice(cuda_device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&ctx->ev0) != cudaSuccess || cudaEventCreate(&ctx->ev1) != cudaSuccess) {
        (void)cudaGetLastError();
        rom_destroy(ctx);
        return ROM_ERR_CUDA;
    }
    ctx->stream = ctx->own_stream;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, cuda_device) == cudaSuccess &&
        sms > 0)
        ctx->sm_count = sms;
    *out = ctx;
    return ROM_OK;
}

void rom_destroy(rom_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    invalidate_graph(ctx);
    DevBuf *bufs[] = {&ctx->sigt, &ctx->sigs, &ctx->q, &ctx->inflow_dev, &ctx->c64, &ctx->s64,
                      &ctx->z64, &ctx->w64, &ctx->c32, &ctx->s32, &ctx->w32, &ctx->items_dev,
                      &ctx->phi, &ctx->src, &ctx->part, &ctx->sums, &ctx->minkey,
                      &ctx->active, &ctx->iters, &ctx->flags, &ctx->resid, &ctx->n_active,
                      &ctx->avg, &ctx->sum, &ctx->tmp, &ctx->psi, &ctx->src_ord, &ctx->Amat,
                      &ctx->dtab, &ctx->z32, &ctx->cta_begin_dev, &ctx->cta_list_dev,
                      &ctx->xface, &ctx->yface, &ctx->err3, &ctx->sig3, &ctx->src3,
                      &ctx->acc3, &ctx->ss3, &ctx->q3, &ctx->psi_split,
                      &ctx->a_hi, &ctx->a_lo, &ctx->tc_err, &ctx->otab, &ctx->ordsum,
                      &ctx->dprev, &ctx->grow,
                      &ctx->leak, &ctx->bal, &ctx->leak_out, &ctx->phimin, &ctx->sweep_err,
                      &ctx->gdesc, &ctx->sgrid_dev, &ctx->soff_dev, &ctx->sdA_dev};
    for (DevBuf *b : bufs) release(*b);
    if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    for (cudaEvent_t e : ctx->kev) cudaEventDestroy(e);
    if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
    delete ctx;
}

const char *rom_last_error(const rom_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int rom_set_stream(rom_ctx *ctx, void *cuda_stream)
{
    if (!ctx) return ROM_ERR_INVALID_ARG;
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->stream = cuda_stream ? (cudaStream_t)cuda_stream : ctx->own_stream;
    return ROM_OK;
}

int rom_set_options(rom_ctx *ctx, const rom_options *opt)
{
    if (!ctx || !opt) return fail(ctx, ROM_ERR_INVALID_ARG, "NULL argument");
    if (opt->scheme != ROM_SCHEME_DD && opt->scheme != ROM_SCHEME_STEP)
        return fail(ctx, ROM_ERR_INVALID_ARG, "unknown scheme %d", opt->scheme);
    if (opt->fixed_iters < 0) return fail(ctx, ROM_ERR_INVALID_ARG, "fixed_iters < 0");
    if (opt->fixed_iters == 0 && (opt->max_iter < 1 || !(opt->tol > 0.0)))
        return fail(ctx, ROM_ERR_INVALID_ARG, "need max_iter >= 1 and tol > 0");
    if (opt->check_every < 0) return fail(ctx, ROM_ERR_INVALID_ARG, "check_every < 0");
    if (opt->time_kernels != 0 && opt->time_kernels != 1)
        return fail(ctx, ROM_ERR_INVALID_ARG, "time_kernels must be 0 or 1");
    if (opt->tile_g != 0 && opt->tile_g != 1 && opt->tile_g != 2 && opt->tile_g != 4 &&
        opt->tile_g != -1)
        return fail(ctx, ROM_ERR_INVALID_ARG, "tile_g must be -1, 0, 1, 2 or 4");
    if (opt->dense_source != 0 && opt->dense_source != 1)
        return fail(ctx, ROM_ERR_INVALID_ARG, "dense_source must be 0 or 1");
    if (opt->dense_precision != 0 && opt->dense_precision != 1)
        return fail(ctx, ROM_ERR_INVALID_ARG, "dense_precision must be 0 or 1");
    if (opt->rows_per_step != 0 && opt->rows_per_step != 1 && opt->rows_per_step != 2 &&
        opt->rows_per_step != 4)
        return fail(ctx, ROM_ERR_INVALID_ARG, "rows_per_step must be 0, 1, 2 or 4");
    if (opt->diverge_window < 0) return fail(ctx, ROM_ERR_INVALID_ARG, "diverge_window < 0");
    if (!(opt->wait_timeout_ms > 0.0) || !(opt->wait_timeout_ms <= 6e5))
        return fail(ctx, ROM_ERR_INVALID_ARG, "wait_timeout_ms must be in (0, 600000]");
    if (opt->test_stall_waits != 0 && opt->test_stall_waits != 1)
        return fail(ctx, ROM_ERR_INVALID_ARG, "test_stall_waits must be 0 or 1");
    if (opt->tile_g != ctx->opt.tile_g || opt->dense_source != ctx->opt.dense_source ||
        opt->dense_precision != ctx->opt.dense_precision ||
        opt->rows_per_step != ctx->opt.rows_per_step) {
        ctx->items_dirty = true;
        ctx->pmat_dirty = true;
    }
    ctx->opt = *opt;
    invalidate_graph(ctx);
    return ROM_OK;
}

int rom_set_grid(rom_ctx *ctx, int dim, const int64_t n[3], const double lo[3], const double hi[3],
                 const double *sigma_t, const double *sigma_s, const double *q)
{
    if (!ctx) return ROM_ERR_INVALID_ARG;
    if (!sigma_t || !sigma_s || !q) return fail(ctx, ROM_ERR_INVALID_ARG, "NULL coefficient array");
    CK(cudaSetDevice(ctx->device));
    const bool prev = ctx->grid_set;
    ctx->grid_set = false;
    int rc = set_grid_common(ctx, prev, dim, n, lo, hi);
    if (rc) return rc;
    const int I = ctx->I, NXP = ctx->NXP;
    const long long J = ctx->rows;  // 3D: the K * J rows of [K][J][I]
    const size_t plane = (size_t)J * NXP;
    if ((rc = ensure_host_stage(ctx, 3 * plane * sizeof(float)))) return rc;
    // one pass: check the hypotheses, convert to FP32, pad the rows, track min/max
    // sigma_T; the pinned staging buffer makes the three copies plain DMA
    float *hs = ctx->h_stage, *hss = hs + plane, *hq = hss + plane;
    double mn = sigma_t[0], mx = sigma_t[0];
    for (long long j = 0; j < J; ++j) {
        const double *a = sigma_t + j * I, *b = sigma_s + j * I, *c = q + j * I;
        float *da = hs + j * NXP, *db = hss + j * NXP, *dc = hq + j * NXP;
        for (int i = 0; i < I; ++i) {
            const double x = a[i], y = b[i], z = c[i];
            if (!(isfinite(x) && isfinite(y) && isfinite(z) && y >= 0.0 && y < x && z >= 0.0))
                return fail(ctx, ROM_ERR_INVALID_ARG,
                            "cell %lld: need 0 <= sigma_S < sigma_T and q >= 0 (got %g, %g, %g)",
                            j * I + i, x, y, z);
            da[i] = (float)x;
            db[i] = (float)y;
            dc[i] = (float)z;
            mn = std::min(mn, x);
            mx = std::max(mx, x);
        }
        for (int i = I; i < NXP; ++i) {
            da[i] = 1.f;
            db[i] = 0.f;
            dc[i] = 0.f;
        }
    }
    set_homog(ctx, (float)mn == (float)mx, (float)mn);
    const size_t bytes = plane * sizeof(float);
    CK(cudaMemcpyAsync(ctx->sigt.p, hs, bytes, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->sigs.p, hss, bytes, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->q.p, hq, bytes, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->grid_set = true;
    return ROM_OK;
}

int rom_set_grid_device(rom_ctx *ctx, int dim, const int64_t n[3], const double lo[3],
                        const double hi[3], const float *sigma_t, const float *sigma_s,
                        const float *q)
{
    if (!ctx) return ROM_ERR_INVALID_ARG;
    if (!sigma_t || !sigma_s || !q) return fail(ctx, ROM_ERR_INVALID_ARG, "NULL coefficient array");
    CK(cudaSetDevice(ctx->device));
    const bool prev = ctx->grid_set;
    ctx->grid_set = false;
    int rc = set_grid_common(ctx, prev, dim, n, lo, hi);
    if (rc) return rc;
    if ((rc = ensure(ctx, ctx->tmp, 4 * sizeof(unsigned int)))) return rc;
    unsigned int init[3] = {0x7f800000u, 0u, 0u};  // +inf bits, 0, 0
    CK(cudaMemcpyAsync(ctx->tmp.p, init, sizeof init, cudaMemcpyHostToDevice, ctx->stream));
    CK(romk::launch_pad_grid(sigma_t, sigma_s, q, ctx->I, (int)ctx->rows, ctx->NXP, (float *)ctx->sigt.p,
                             (float *)ctx->sigs.p, (float *)ctx->q.p, (unsigned int *)ctx->tmp.p,
                             ctx->stream));
    ++ctx->launches;
    unsigned int st[3];
    CK(cudaMemcpyAsync(st, ctx->tmp.p, sizeof st, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (st[2] != 0)
        return fail(ctx, ROM_ERR_INVALID_ARG,
                    "%u cells violate 0 <= sigma_S < sigma_T, q >= 0 (or are not finite)", st[2]);
    float mn, mx;
    memcpy(&mn, &st[0], sizeof mn);
    memcpy(&mx, &st[1], sizeof mx);
    set_homog(ctx, mn == mx, mn);
    ctx->grid_set = true;
    return ROM_OK;
}

int rom_set_grids_xy(rom_ctx *ctx, int n_grids, const int64_t *n, const double *lo,
                     const double *hi, const double *sigma_t, const double *sigma_s,
                     const double *q, const int32_t *samples_per_grid)
{
    if (!ctx) return ROM_ERR_INVALID_ARG;
    if (n_grids < 1) return fail(ctx, ROM_ERR_INVALID_ARG, "n_grids must be >= 1");
    if (!n || !lo || !hi || !sigma_t || !sigma_s || !q || !samples_per_grid)
        return fail(ctx, ROM_ERR_INVALID_ARG, "NULL argument");
    CK(cudaSetDevice(ctx->device));
    ctx->grid_set = false;
    std::vector<romk::GridDesc> grids(n_grids);
    std::vector<long long> avg_off(n_grids + 1, 0), in_off(n_grids + 1, 0);
    long long off = 0, max_cells = 0;
    int max_i = 0, max_j = 0;
    for (int p = 0; p < n_grids; ++p) {
        const long long I = n[2 * p], J = n[2 * p + 1];
        if (I < 1 || J < 1) return fail(ctx, ROM_ERR_INVALID_ARG, "grid %d: sizes must be >= 1", p);
        if (I > 32 * romk::kMaxWarps * romk::kCols || J > (1 << 24))
            return fail(ctx, ROM_ERR_INVALID_ARG, "grid %d: %lld x %lld is too large", p, I, J);
        for (int d = 0; d < 2; ++d)
            if (!(hi[2 * p + d] > lo[2 * p + d]) || !isfinite(lo[2 * p + d]) ||
                !isfinite(hi[2 * p + d]))
                return fail(ctx, ROM_ERR_INVALID_ARG, "grid %d: need hi > lo (finite)", p);
        if (samples_per_grid[p] < 1)
            return fail(ctx, ROM_ERR_INVALID_ARG, "grid %d: samples_per_grid must be >= 1", p);
        romk::GridDesc &g = grids[p];
        g.I = (int)I;
        g.J = (int)J;
        g.NXP = (int)((I + romk::kCols - 1) / romk::kCols * romk::kCols);
        const double wx = hi[2 * p] - lo[2 * p], wy = hi[2 * p + 1] - lo[2 * p + 1];
        g.inv_dx = (float)(I / wx);
        g.inv_dy = (float)(J / wy);
        g.dx = (float)(wx / I);
        g.dy = (float)(wy / J);
        g.off = off;
        g.cells = J * g.NXP;
        off += g.cells;
        max_cells = std::max(max_cells, g.cells);
        max_i = std::max(max_i, g.I);
        max_j = std::max(max_j, g.J);
        avg_off[p + 1] = avg_off[p] + I * J;
        in_off[p + 1] = in_off[p] + I * J;
    }
    int rc;
    if ((rc = ensure_host_stage(ctx, 3 * (size_t)off * sizeof(float)))) return rc;
    float *hs = ctx->h_stage, *hss = hs + off, *hq = hss + off;
    for (int p = 0; p < n_grids; ++p) {
        const romk::GridDesc &g = grids[p];
        for (long long j = 0; j < g.J; ++j) {
            const long long src = in_off[p] + j * g.I, dst = g.off + j * g.NXP;
            for (int i = 0; i < g.I; ++i) {
                const double x = sigma_t[src + i], y = sigma_s[src + i], z = q[src + i];
                if (!(isfinite(x) && isfinite(y) && isfinite(z) && y >= 0.0 && y < x && z >= 0.0))
                    return fail(ctx, ROM_ERR_INVALID_ARG,
                                "grid %d, cell %lld: need 0 <= sigma_S < sigma_T and q >= 0 "
                                "(got %g, %g, %g)", p, j * g.I + i, x, y, z);
                hs[dst + i] = (float)x;
                hss[dst + i] = (float)y;
                hq[dst + i] = (float)z;
            }
            for (int i = g.I; i < g.NXP; ++i) {
                hs[dst + i] = 1.f;
                hss[dst + i] = 0.f;
                hq[dst + i] = 0.f;
            }
        }
    }
    // the context's own grid fields hold the largest extents (the sweep's block
    // width); the per-grid sizes travel in the grid table
    ctx->n_grids = 0;
    ctx->dim = 2;
    ctx->I = max_i;
    ctx->J = max_j;
    ctx->K = 1;
    ctx->rows = max_j;
    ctx->NXP = (max_i + romk::kCols - 1) / romk::kCols * romk::kCols;
    for (int d = 0; d < 3; ++d) {
        ctx->lo[d] = d < 2 ? lo[d] : 0.0;
        ctx->hi[d] = d < 2 ? hi[d] : 1.0;
    }
    for (int f = 0; f < 6; ++f) {
        ctx->inflow_iso[f].clear();
        ctx->inflow_ord[f].clear();
    }
    ctx->grids = grids;
    ctx->grid_samples.assign(samples_per_grid, samples_per_grid + n_grids);
    ctx->avg_off = avg_off;
    ctx->coef_cells = off;
    ctx->max_cells = max_cells;
    ctx->n_grids = n_grids;
    ctx->solved = false;
    ctx->inflow_dirty = true;
    ctx->items_dirty = true;
    ctx->tuned_g = 0;
    ctx->tuned_h = 0;
    invalidate_graph(ctx);
    set_homog(ctx, false, 1.f);  // sigma_T is read per cell (the grids' blocks)
    const size_t bytes = (size_t)off * sizeof(float);
    if ((rc = ensure(ctx, ctx->sigt, bytes)) || (rc = ensure(ctx, ctx->sigs, bytes)) ||
        (rc = ensure(ctx, ctx->q, bytes)))
        return rc;
    CK(cudaMemcpyAsync(ctx->sigt.p, hs, bytes, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->sigs.p, hss, bytes, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->q.p, hq, bytes, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->grid_set = true;
    return ROM_OK;
}

int rom_set_inflow_isotropic(rom_ctx *ctx, int face, const double *psi_face)
{
    if (!ctx) return ROM_ERR_INVALID_ARG;
    if (!ctx->grid_set) return fail(ctx, ROM_ERR_STATE, "set the grid first");
    if (batch(ctx)) return fail(ctx, ROM_ERR_UNSUPPORTED, "several grids: vacuum boundaries only");
    if (face < 0 || face >= n_faces(ctx))
        return fail(ctx, ROM_ERR_INVALID_ARG, "face must be 0..%d", n_faces(ctx) - 1);
    ctx->inflow_iso[face].clear();
    ctx->inflow_ord[face].clear();
    if (psi_face) {
        const long long nf = face_cells(ctx, face);
        for (long long k = 0; k < nf; ++k)
            if (!(psi_face[k] >= 0.0) || !isfinite(psi_face[k]))
                return fail(ctx, ROM_ERR_INVALID_ARG, "inflow must be finite and >= 0");
        ctx->inflow_iso[face].assign(psi_face, psi_face + nf);
    }
    ctx->inflow_dirty = true;
    ctx->solved = false;
    return ROM_OK;
}

int rom_set_inflow_ordinates(rom_ctx *ctx, int face, const double *psi)
{
    if (!ctx) return ROM_ERR_INVALID_ARG;
    if (!ctx->grid_set) return fail(ctx, ROM_ERR_STATE, "set the grid first");
    if (ctx->ord_source == ORD_NONE) return fail(ctx, ROM_ERR_STATE, "set the ordinates first");
    if (batch(ctx)) return fail(ctx, ROM_ERR_UNSUPPORTED, "several grids: vacuum boundaries only");
    if (face < 0 || face >= n_faces(ctx))
        return fail(ctx, ROM_ERR_INVALID_ARG, "face must be 0..%d", n_faces(ctx) - 1);
    ctx->inflow_iso[face].clear();
    ctx->inflow_ord[face].clear();
    if (psi) {
        const size_t n = (size_t)ctx->Mtot * face_cells(ctx, face);
        for (size_t k = 0; k < n; ++k)
            if (!(psi[k] >= 0.0) || !isfinite(psi[k]))
                return fail(ctx, ROM_ERR_INVALID_ARG, "inflow must be finite and >= 0");
        ctx->inflow_ord[face].assign(psi, psi + n);
    }
    ctx->inflow_dirty = true;
    ctx->solved = false;
    return ROM_OK;
}

int rom_set_ordinates(rom_ctx *ctx, int n_samples, const int32_t *m_per_sample,
                      const double *dirs, const double *weights)
{
    if (!ctx) return ROM_ERR_INVALID_ARG;
    if (n_samples < 1 || !m_per_sample || !dirs || !weights)
        return fail(ctx, ROM_ERR_INVALID_ARG, "need n_samples >= 1 and non-NULL arrays");
    CK(cudaSetDevice(ctx->device));
    long long tot = 0;
    for (int s = 0; s < n_samples; ++s) {
        if (m_per_sample[s] < 1)
            return fail(ctx, ROM_ERR_INVALID_ARG, "sample %d has %d ordinates", s, m_per_sample[s]);
        tot += m_per_sample[s];
    }
    if (tot > (1LL << 30)) return fail(ctx, ROM_ERR_INVALID_ARG, "too many ordinates");
    for (long long o = 0; o < tot; ++o) {
        const double c = dirs[3 * o], s = dirs[3 * o + 1], z = dirs[3 * o + 2], w = weights[o];
        if (!(isfinite(c) && isfinite(s) && isfinite(z) && isfinite(w)) || !(w > 0.0) ||
            fabs(c * c + s * s + z * z - 1.0) > 1e-6)
            return fail(ctx, ROM_ERR_INVALID_ARG,
                        "ordinate %lld: need |u| = 1 and weight > 0 (got %g %g %g, %g)", o, c, s,
                        z, w);
    }
    ctx->S = n_samples;
    ctx->Mtot = tot;
    ctx->M.assign(m_per_sample, m_per_sample + n_samples);
    ctx->off.resize(n_samples);
    long long acc = 0;
    for (int s = 0; s < n_samples; ++s) {
        ctx->off[s] = acc;
        acc += ctx->M[s];
    }
    ctx->quad.resize(tot);
    std::vector<double> c(tot), s(tot), z(tot), w(tot);
    std::vector<float> cf(tot), sf(tot), zf(tot), wf(tot);
    for (long long o = 0; o < tot; ++o) {
        c[o] = dirs[3 * o];
        s[o] = dirs[3 * o + 1];
        z[o] = dirs[3 * o + 2];
        w[o] = weights[o];
        cf[o] = (float)c[o];
        sf[o] = (float)s[o];
        zf[o] = (float)z[o];
        wf[o] = (float)w[o];
        ctx->quad[o] =
            (unsigned char)((c[o] < 0.0 ? 1 : 0) | (s[o] < 0.0 ? 2 : 0) | (z[o] < 0.0 ? 4 : 0));
    }
    int rc;
    const size_t b8 = tot * sizeof(double), b4 = tot * sizeof(float);
    if ((rc = ensure(ctx, ctx->c64, b8)) || (rc = ensure(ctx, ctx->s64, b8)) ||
        (rc = ensure(ctx, ctx->z64, b8)) || (rc = ensure(ctx, ctx->w64, b8)) ||
        (rc = ensure(ctx, ctx->c32, b4)) || (rc = ensure(ctx, ctx->s32, b4)) ||
        (rc = ensure(ctx, ctx->z32, b4)) || (rc = ensure(ctx, ctx->w32, b4)))
        return rc;
    CK(cudaMemcpyAsync(ctx->c64.p, c.data(), b8, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->s64.p, s.data(), b8, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->z64.p, z.data(), b8, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->w64.p, w.data(), b8, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->c32.p, cf.data(), b4, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->s32.p, sf.data(), b4, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->z32.p, zf.data(), b4, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->w32.p, wf.data(), b4, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->ord_source = ORD_EXPLICIT;
    ctx->seed_octants = false;
    reset_ordinate_dependents(ctx);
    return ROM_OK;
}

}  // extern "C"

namespace {

int set_ordinates_seeded(rom_ctx *ctx, uint64_t seed, int first_sample, int n_samples,
                         const int32_t *n_zeta, const int32_t *n_theta, bool octants)
{
    if (!ctx) return ROM_ERR_INVALID_ARG;
    if (n_samples < 1 || first_sample < 0 || !n_zeta || !n_theta)
        return fail(ctx, ROM_ERR_INVALID_ARG, "need n_samples >= 1, first_sample >= 0, arrays");
    if ((long long)first_sample + n_samples > (1LL << 31))
        return fail(ctx, ROM_ERR_INVALID_ARG, "sample index out of range");
    CK(cudaSetDevice(ctx->device));
    const bool same_layout =
        ctx->ord_source == ORD_SEED && ctx->S == n_samples && ctx->seed_octants == octants;
    const int per_cell = octants ? 8 : 4;
    std::vector<int> nz(n_zeta, n_zeta + n_samples), nt(n_theta, n_theta + n_samples);
    std::vector<int> first_cell(n_samples + 1, 0);
    std::vector<long long> off(n_samples);
    std::vector<int> M(n_samples);
    long long tot = 0;
    for (int s = 0; s < n_samples; ++s) {
        if (nz[s] < 1 || nt[s] < 1 || (long long)nz[s] * nt[s] > (1 << 24))
            return fail(ctx, ROM_ERR_INVALID_ARG, "sample %d: bad partition %d x %d", s, nz[s],
                        nt[s]);
        const int m = nz[s] * nt[s];
        first_cell[s + 1] = first_cell[s] + m;
        off[s] = tot;
        M[s] = per_cell * m;
        tot += (long long)per_cell * m;
        if (first_cell[s + 1] > (1 << 30)) return fail(ctx, ROM_ERR_INVALID_ARG, "too many cells");
    }
    bool layout_same = same_layout && ctx->M == M;
    ctx->S = n_samples;
    ctx->Mtot = tot;
    ctx->M = M;
    ctx->off = off;
    int rc;
    const size_t b8 = tot * sizeof(double), b4 = tot * sizeof(float);
    if ((rc = ensure(ctx, ctx->c64, b8)) || (rc = ensure(ctx, ctx->s64, b8)) ||
        (rc = ensure(ctx, ctx->z64, b8)) || (rc = ensure(ctx, ctx->w64, b8)) ||
        (rc = ensure(ctx, ctx->c32, b4)) || (rc = ensure(ctx, ctx->s32, b4)) ||
        (rc = ensure(ctx, ctx->z32, b4)) || (rc = ensure(ctx, ctx->w32, b4)))
        return rc;
    // small per-sample tables packed into one device buffer
    const size_t tb = (size_t)n_samples * (2 * sizeof(int) + sizeof(long long)) +
                      (size_t)(n_samples + 1) * sizeof(int) + 64;
    if ((rc = ensure(ctx, ctx->tmp, tb))) return rc;
    std::vector<unsigned char> packed(tb, 0);
    size_t p = 0;
    const size_t o_off = p;
    memcpy(packed.data() + p, off.data(), n_samples * sizeof(long long));
    p += n_samples * sizeof(long long);
    const size_t o_nz = p;
    memcpy(packed.data() + p, nz.data(), n_samples * sizeof(int));
    p += n_samples * sizeof(int);
    const size_t o_nt = p;
    memcpy(packed.data() + p, nt.data(), n_samples * sizeof(int));
    p += n_samples * sizeof(int);
    const size_t o_fc = p;
    memcpy(packed.data() + p, first_cell.data(), (n_samples + 1) * sizeof(int));
    CK(cudaMemcpyAsync(ctx->tmp.p, packed.data(), tb, cudaMemcpyHostToDevice, ctx->stream));
    romk::OrdGenArgs a{};
    unsigned char *base = (unsigned char *)ctx->tmp.p;
    a.seed = seed;
    a.n_samples = n_samples;
    a.nz = (const int *)(base + o_nz);
    a.nt = (const int *)(base + o_nt);
    a.first_cell = (const int *)(base + o_fc);
    a.ord_off = (const long long *)(base + o_off);
    a.first_sample = first_sample;
    a.total_cells = first_cell[n_samples];
    a.octants = octants ? 1 : 0;
    a.c64 = (double *)ctx->c64.p;
    a.s64 = (double *)ctx->s64.p;
    a.z64 = (double *)ctx->z64.p;
    a.w64 = (double *)ctx->w64.p;
    a.c32 = (float *)ctx->c32.p;
    a.s32 = (float *)ctx->s32.p;
    a.z32 = (float *)ctx->z32.p;
    a.w32 = (float *)ctx->w32.p;
    CK(romk::launch_ordgen(a, ctx->stream));
    ++ctx->launches;
    CK(cudaStreamSynchronize(ctx->stream));  // the packed host table dies with this call
    ctx->ord_source = ORD_SEED;
    ctx->seed_octants = octants;
    if (layout_same) {
        // same sample layout: work items, buffers and the captured graph stay valid;
        // the dense operator belongs to the old ordinates, and so does per-ordinate inflow
        bool had_ord_inflow = false;
        for (int f = 0; f < 6; ++f) {
            had_ord_inflow |= !ctx->inflow_ord[f].empty();
            ctx->inflow_ord[f].clear();
        }
        if (had_ord_inflow) ctx->inflow_dirty = true;
        ctx->pmat_dirty = true;
        ctx->solved = false;
    } else {
        reset_ordinate_dependents(ctx);
    }
    return ROM_OK;
}

}  // namespace

extern "C" {

int rom_set_ordinates_seed_offset(rom_ctx *ctx, uint64_t seed, int first_sample, int n_samples,
                                  const int32_t *n_zeta, const int32_t *n_theta)
{
    return set_ordinates_seeded(ctx, seed, first_sample, n_samples, n_zeta, n_theta, false);
}

int rom_set_ordinates_seed_xyz(rom_ctx *ctx, uint64_t seed, int first_sample, int n_samples,
                               const int32_t *n_zeta, const int32_t *n_theta)
{
    return set_ordinates_seeded(ctx, seed, first_sample, n_samples, n_zeta, n_theta, true);
}

int rom_set_ordinates_seed(rom_ctx *ctx, uint64_t seed, int n_samples, const int32_t *n_zeta,
                           const int32_t *n_theta)
{
    return rom_set_ordinates_seed_offset(ctx, seed, 0, n_samples, n_zeta, n_theta);
}

int rom_quadrature_xy(int kind, int n1, int n2, double *dirs, double *weights, int32_t *m_out)
{
    std::vector<double> c, s, z, w;
    const int M = romk::host_quadrature(kind, n1, n2, c, s, z, w);
    if (M < 1) return ROM_ERR_INVALID_ARG;
    if (m_out) *m_out = M;
    if (dirs)
        for (int o = 0; o < M; ++o) {
            dirs[3 * o] = c[o];
            dirs[3 * o + 1] = s[o];
            dirs[3 * o + 2] = z[o];
        }
    if (weights)
        for (int o = 0; o < M; ++o) weights[o] = w[o];
    return ROM_OK;
}

int rom_set_quadrature(rom_ctx *ctx, int kind, int n1, int n2)
{
    if (!ctx) return ROM_ERR_INVALID_ARG;
    std::vector<double> c, s, z, w;
    const int M = romk::host_quadrature(kind, n1, n2, c, s, z, w);
    if (M < 1) return fail(ctx, ROM_ERR_INVALID_ARG, "bad quadrature (%d, %d, %d)", kind, n1, n2);
    std::vector<double> dirs(3 * (size_t)M);
    for (int o = 0; o < M; ++o) {
        dirs[3 * o] = c[o];
        dirs[3 * o + 1] = s[o];
        dirs[3 * o + 2] = z[o];
    }
    const int32_t m = M;
    return rom_set_ordinates(ctx, 1, &m, dirs.data(), w.data());
}

int rom_get_ordinates(rom_ctx *ctx, double *dirs, double *weights)
{
    if (!ctx) return ROM_ERR_INVALID_ARG;
    if (ctx->ord_source == ORD_NONE) return fail(ctx, ROM_ERR_STATE, "no ordinates set");
    CK(cudaSetDevice(ctx->device));
    const long long n = ctx->Mtot;
    std::vector<double> c(n), s(n), z(n);
    CK(cudaMemcpyAsync(c.data(), ctx->c64.p, n * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(s.data(), ctx->s64.p, n * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(z.data(), ctx->z64.p, n * 8, cudaMemcpyDeviceToHost, ctx->stream));
    if (weights)
        CK(cudaMemcpyAsync(weights, ctx->w64.p, n * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (dirs)
        for (long long o = 0; o < n; ++o) {
            dirs[3 * o] = c[o];
            dirs[3 * o + 1] = s[o];
            dirs[3 * o + 2] = z[o];
        }
    return ROM_OK;
}

int rom_set_kernel(rom_ctx *ctx, int kind, double g, int flags)
{
    if (!ctx) return ROM_ERR_INVALID_ARG;
    if (kind < ROM_KERNEL_ISO || kind > ROM_KERNEL_HG)
        return fail(ctx, ROM_ERR_INVALID_ARG, "unknown kernel %d", kind);
    if (!(g > -1.0 && g < 1.0)) return fail(ctx, ROM_ERR_INVALID_ARG, "need -1 < g < 1");
    if (flags & ~(ROM_KERNEL_FLAG_NORMALIZE | ROM_KERNEL_FLAG_RAW))
        return fail(ctx, ROM_ERR_INVALID_ARG, "unknown kernel flags");
    ctx->kernel_kind = kind;
    ctx->g = kind == ROM_KERNEL_ISO ? 0.0 : g;
    ctx->kernel_flags = flags;
    ctx->pmat_dirty = true;
    ctx->tuned_g = 0;
    ctx->tuned_h = 0;
    ctx->items_dirty = true;
    ctx->solved = false;
    invalidate_graph(ctx);
    return ROM_OK;
}

int rom_solve(rom_ctx *ctx, rom_stats *stats_out)
{
    if (!ctx) return ROM_ERR_INVALID_ARG;
    if (!ctx->grid_set) return fail(ctx, ROM_ERR_STATE, "set the grid first");
    if (ctx->ord_source == ORD_NONE) return fail(ctx, ROM_ERR_STATE, "set the ordinates first");
    CK(cudaSetDevice(ctx->device));
    int rc;
    const long long cells = batch(ctx) ? ctx->max_cells : padded_cells(ctx);
    const int mode = source_mode(ctx);
    const int MOM = mode == 0 ? 1 : mode;  // moments kept per sample
    if (batch(ctx) && mode == 0)
        return fail(ctx, ROM_ERR_UNSUPPORTED,
                    "several grids support the moment modes only (isotropic or linear kernel)");
    if (ctx->dim == 3 && mode != 1)
        return fail(ctx, ROM_ERR_UNSUPPORTED,
                    "3D grids support the isotropic kernel with angular moments only");
    if (mode != ctx->MOM) {
        ctx->MOM = mode;
        ctx->items_dirty = true;
        invalidate_graph(ctx);
    }
    if (ctx->items_dirty) {
        if ((rc = build_items(ctx))) return rc;
        invalidate_graph(ctx);
    }
    if (ctx->inflow_dirty) {
        if ((rc = upload_inflow(ctx))) return rc;
        invalidate_graph(ctx);
    }
    // residual chunks of the 3D combine: blocks of 256 threads per sample, each
    // thread taking one or more 8-cell sectors; about 16 blocks per SM in all, so
    // that large grids stream many sectors per thread instead of paying the block's
    // reduction per sector (the X-Y combine sizes its own grid)
    const long long max_chunks = std::max<long long>(1, (cells / 8 + 255) / 256);
    const long long want = std::max<long long>(1, (16LL * ctx->sm_count + ctx->S - 1) / ctx->S);
    const int chunks = (int)std::min(max_chunks, want);
    if (chunks != ctx->chunks) invalidate_graph(ctx);
    ctx->chunks = chunks;
    const size_t nI = (size_t)avg_cells(ctx);
    void *before[] = {ctx->phi.p,  ctx->src.p,  ctx->part.p,  ctx->sums.p, ctx->minkey.p, ctx->active.p,
                      ctx->sig3.p, ctx->src3.p, ctx->acc3.p,  ctx->ss3.p,      ctx->q3.p,
                      ctx->ordsum.p, ctx->dprev.p,
                      ctx->grow.p, ctx->leak.p, ctx->bal.p, ctx->leak_out.p, ctx->phimin.p,
                      ctx->sweep_err.p, ctx->otab.p};
    if ((rc = ensure(ctx, ctx->sums, (size_t)ctx->S * romk::kNP * sizeof(double))) ||
        (rc = ensure(ctx, ctx->minkey, (size_t)ctx->S * sizeof(int))) ||
        (rc = ensure(ctx, ctx->active, ctx->S * sizeof(int))) ||
        (rc = ensure(ctx, ctx->iters, ctx->S * sizeof(int))) ||
        (rc = ensure(ctx, ctx->flags, ctx->S * sizeof(int))) ||
        (rc = ensure(ctx, ctx->resid, ctx->S * sizeof(double))) ||
        (rc = ensure(ctx, ctx->dprev, ctx->S * sizeof(double))) ||
        (rc = ensure(ctx, ctx->grow, ctx->S * sizeof(int))) ||
        (rc = ensure(ctx, ctx->leak, ctx->S * sizeof(double))) ||
        (rc = ensure(ctx, ctx->bal, ctx->S * sizeof(double))) ||
        (rc = ensure(ctx, ctx->leak_out, ctx->S * sizeof(double))) ||
        (rc = ensure(ctx, ctx->phimin, ctx->S * sizeof(double))) ||
        (rc = ensure(ctx, ctx->ordsum, (size_t)ctx->S * 3 * sizeof(double))) ||
        (rc = ensure(ctx, ctx->sweep_err, sizeof(int))) ||
        (rc = ensure(ctx, ctx->n_active, sizeof(int))) ||
        (rc = ensure(ctx, ctx->avg, nI * sizeof(double))) ||
        (rc = ensure(ctx, ctx->sum, nI * sizeof(double))))
        return rc;
    if (ctx->MOM == 0) {
        void *dense_before[] = {ctx->psi.p, ctx->src_ord.p, ctx->Amat.p, ctx->dtab.p};
        if ((rc = prepare_dense(ctx))) return rc;
        void *dense_after[] = {ctx->psi.p, ctx->src_ord.p, ctx->Amat.p, ctx->dtab.p};
        if (memcmp(dense_before, dense_after, sizeof dense_before) != 0) invalidate_graph(ctx);
    }
    if (ctx->dim == 2 && ctx->opt.tile_g == -1 && ctx->tuned_g == 0) {
        if ((rc = autotune_g(ctx))) return rc;
        if ((rc = build_items(ctx))) return rc;
        invalidate_graph(ctx);
    }
    if ((rc = ensure_state(ctx))) return rc;
    void *after[] = {ctx->phi.p,  ctx->src.p,  ctx->part.p,  ctx->sums.p, ctx->minkey.p, ctx->active.p,
                     ctx->sig3.p, ctx->src3.p, ctx->acc3.p,  ctx->ss3.p,      ctx->q3.p,
                     ctx->ordsum.p, ctx->dprev.p,
                     ctx->grow.p, ctx->leak.p, ctx->bal.p, ctx->leak_out.p, ctx->phimin.p,
                     ctx->sweep_err.p, ctx->otab.p};
    if (memcmp(before, after, sizeof before) != 0) invalidate_graph(ctx);

    const long long launches0 = ctx->launches;
    CK(cudaEventRecord(ctx->ev0, ctx->stream));
    if ((rc = init_state(ctx))) return rc;
    const int cap = ctx->opt.fixed_iters > 0 ? ctx->opt.fixed_iters : ctx->opt.max_iter;
    const bool timed = ctx->opt.time_kernels == 1;
    double sweep_ms = 0.0, source_ms = 0.0;
    long long sweep_launches = 0, source_launches = 0;
    const bool device_loop = ctx->opt.check_every == 0 && !timed;
    if (device_loop) {
        if (!ctx->graph_valid && (rc = build_graph(ctx))) return rc;
        CK(cudaGraphLaunch(ctx->graph_exec, ctx->stream));
    } else {
        const int every = ctx->opt.check_every > 0 ? ctx->opt.check_every : 1;
        if (timed && ctx->kev.size() < 4 * (size_t)every) {
            while (ctx->kev.size() < 4 * (size_t)every) {
                cudaEvent_t e;
                CK(cudaEventCreate(&e));
                ctx->kev.push_back(e);
            }
        }
        int done = 0;
        while (done < cap) {
            const int n = std::min(every, cap - done);
            for (int k = 0; k < n; ++k) {
                cudaEvent_t k0 = timed ? ctx->kev[4 * k] : nullptr;
                cudaEvent_t k1 = timed ? ctx->kev[4 * k + 1] : nullptr;
                cudaEvent_t k2 = timed && ctx->MOM == 0 ? ctx->kev[4 * k + 2] : nullptr;
                cudaEvent_t k3 = timed && ctx->MOM == 0 ? ctx->kev[4 * k + 3] : nullptr;
                if ((rc = enqueue_iteration(ctx, ctx->stream, false, 0, k0, k1, k2, k3))) return rc;
                ctx->launches += launches_per_iteration(ctx);
            }
            done += n;
            int n_active = 0;
            CK(cudaMemcpyAsync(&n_active, ctx->n_active.p, sizeof(int), cudaMemcpyDeviceToHost,
                               ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
            if (timed)
                for (int k = 0; k < n; ++k) {
                    float ms = 0.f;
                    CK(cudaEventElapsedTime(&ms, ctx->kev[4 * k], ctx->kev[4 * k + 1]));
                    sweep_ms += ms;
                    ++sweep_launches;
                    if (ctx->MOM == 0) {
                        CK(cudaEventElapsedTime(&ms, ctx->kev[4 * k + 2], ctx->kev[4 * k + 3]));
                        source_ms += ms;
                        ++source_launches;
                    }
                }
            if (n_active == 0) break;
        }
    }
    if (ctx->dim == 3)
        CK(romk::launch_average3((const float *)ctx->phi.p, ctx->S,
                                 romk::make_skew3(ctx->J, ctx->K, ctx->NXP), ctx->I,
                                 (double *)ctx->avg.p, (double *)ctx->sum.p, ctx->stream));
    else if (batch(ctx)) {  // each grid's samples are consecutive [MOM][J_p][NXP_p] blocks
        int s0 = 0;
        for (int p = 0; p < ctx->n_grids; ++p) {
            const romk::GridDesc &g = ctx->grids[p];
            CK(romk::launch_average((const float *)ctx->phi.p + ctx->soff[s0],
                                    ctx->grid_samples[p], MOM, g.I, g.J, g.NXP,
                                    (double *)ctx->avg.p + ctx->avg_off[p],
                                    (double *)ctx->sum.p + ctx->avg_off[p], ctx->stream));
            s0 += ctx->grid_samples[p];
        }
        ctx->launches += ctx->n_grids - 1;
    } else
        CK(romk::launch_average((const float *)ctx->phi.p, ctx->S, MOM, ctx->I, (int)ctx->rows,
                                ctx->NXP, (double *)ctx->avg.p, (double *)ctx->sum.p,
                                ctx->stream));
    ++ctx->launches;
    CK(cudaEventRecord(ctx->ev1, ctx->stream));
    ctx->h_iters.assign(ctx->S, 0);
    ctx->h_resid.assign(ctx->S, 0.0);
    ctx->h_bal.assign(ctx->S, 0.0);
    ctx->h_leak.assign(ctx->S, 0.0);
    ctx->h_phimin.assign(ctx->S, 0.0);
    std::vector<int> flags(ctx->S, 0);
    int err3 = 0, tc_err = 0, sweep_err = 0;
    if (ctx->dim == 3)
        CK(cudaMemcpyAsync(&err3, ctx->err3.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(&sweep_err, ctx->sweep_err.p, sizeof(int), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaMemcpyAsync(ctx->h_bal.data(), ctx->bal.p, ctx->S * sizeof(double),
                       cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(ctx->h_leak.data(), ctx->leak_out.p, ctx->S * sizeof(double),
                       cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(ctx->h_phimin.data(), ctx->phimin.p, ctx->S * sizeof(double),
                       cudaMemcpyDeviceToHost, ctx->stream));
    if (ctx->MOM == 0 && ctx->opt.dense_precision == 1)
        CK(cudaMemcpyAsync(&tc_err, ctx->tc_err.p, sizeof(int), cudaMemcpyDeviceToHost,
                           ctx->stream));
    CK(cudaMemcpyAsync(ctx->h_iters.data(), ctx->iters.p, ctx->S * sizeof(int),
                       cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(ctx->h_resid.data(), ctx->resid.p, ctx->S * sizeof(double),
                       cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(flags.data(), ctx->flags.p, ctx->S * sizeof(int), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
    if (err3)
        return fail(ctx, ROM_ERR_TIMEOUT, "3D sweep: a wait between warps timed out (flags %d)",
                    err3);
    if (sweep_err)
        return fail(ctx, ROM_ERR_TIMEOUT, "X-Y sweep: a bounded wait ran out (flags %d)",
                    sweep_err);
    if (tc_err)
        return fail(ctx, ROM_ERR_TIMEOUT, "tensor-core dense source: a wait timed out (flags %d)",
                    tc_err);
    ctx->solved = true;

    rom_stats st{};
    st.n_samples = ctx->S;
    st.iterations_max = 0;
    st.iterations_min = ctx->S ? ctx->h_iters[0] : 0;
    int diverged = 0, growing = 0;
    st.balance_max = has_balance(ctx) ? 0.0 : NAN;
    st.phi_min = INFINITY;
    for (int s = 0; s < ctx->S; ++s) {
        const int it = ctx->h_iters[s];
        st.iterations_max = std::max(st.iterations_max, it);
        st.iterations_min = std::min(st.iterations_min, it);
        st.updates += (int64_t)sample_cells(ctx, s) * ctx->M[s] * it;
        const double r = ctx->h_resid[s];
        if (!(r <= st.residual_max)) st.residual_max = r;
        if (has_balance(ctx) && !(ctx->h_bal[s] <= st.balance_max)) st.balance_max = ctx->h_bal[s];
        st.phi_min = std::min(st.phi_min, ctx->h_phimin[s]);
        if (flags[s] & 3) {
            ++diverged;
            if (flags[s] & 2) ++growing;
        } else if (ctx->opt.fixed_iters == 0 && !(r < ctx->opt.tol)) {
            ++st.n_not_converged;
        }
    }
    st.gpu_ms = ms;
    st.sweep_ms = sweep_ms;
    st.sweep_launches = sweep_launches;
    st.source_ms = source_ms;
    st.source_launches = source_launches;
    st.tile_g = ctx->G_used;
    st.rows_per_step = ctx->dim == 2 ? ctx->H_used : 0;
    if (device_loop) ctx->launches += (long long)launches_per_iteration(ctx) * st.iterations_max;
    st.kernel_launches = ctx->launches - launches0;
    if (stats_out) *stats_out = st;
    if (diverged)
        return fail(ctx, ROM_ERR_DIVERGED,
                    "%d samples diverged (%d with a NaN/Inf residual, %d with a change that grew "
                    "for %d sweeps)",
                    diverged, diverged - growing, growing, ctx->opt.diverge_window);
    if (st.n_not_converged)
        return fail(ctx, ROM_ERR_NOT_CONVERGED, "%d samples did not reach tol %g in %d sweeps",
                    st.n_not_converged, ctx->opt.tol, ctx->opt.max_iter);
    return ROM_OK;
}

// phi of one sample -> out[n_cells] (device), from the layout its dimension keeps
cudaError_t extract_phi(rom_ctx *ctx, int sample, double *out)
{
    if (batch(ctx)) {
        const romk::GridDesc &g = ctx->grids[ctx->sgrid[sample]];
        return romk::launch_extract((const float *)ctx->phi.p + ctx->soff[sample], 0,
                                    ctx->MOM == 0 ? 1 : ctx->MOM, g.I, g.J, g.NXP, out,
                                    ctx->stream);
    }
    if (ctx->dim == 3)
        return romk::launch_extract3((const float *)ctx->phi.p, sample,
                                     romk::make_skew3(ctx->J, ctx->K, ctx->NXP), ctx->I, out,
                                     ctx->stream);
    return romk::launch_extract((const float *)ctx->phi.p, sample, ctx->MOM == 0 ? 1 : ctx->MOM,
                                ctx->I, (int)ctx->rows, ctx->NXP, out, ctx->stream);
}

int rom_get_scalar_flux(rom_ctx *ctx, int sample, double *out)
{
    if (!ctx || !out) return fail(ctx, ROM_ERR_INVALID_ARG, "NULL argument");
    if (!ctx->solved) return fail(ctx, ROM_ERR_STATE, "call rom_solve first");
    if (sample < -1 || sample >= ctx->S) return fail(ctx, ROM_ERR_INVALID_ARG, "bad sample %d", sample);
    if (sample == -1 && batch(ctx))
        return fail(ctx, ROM_ERR_INVALID_ARG,
                    "several grids: read each grid's average with rom_get_grid_average");
    CK(cudaSetDevice(ctx->device));
    const size_t nI = (size_t)(sample >= 0 ? sample_cells(ctx, sample) : n_cells(ctx));
    if (sample >= 0) {
        int rc = ensure(ctx, ctx->tmp, nI * sizeof(double));
        if (rc) return rc;
        CK(extract_phi(ctx, sample, (double *)ctx->tmp.p));
        ++ctx->launches;
        CK(cudaMemcpyAsync(out, ctx->tmp.p, nI * sizeof(double), cudaMemcpyDeviceToHost,
                           ctx->stream));
    } else {
        CK(cudaMemcpyAsync(out, ctx->avg.p, nI * sizeof(double), cudaMemcpyDeviceToHost,
                           ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return ROM_OK;
}

int rom_get_scalar_flux_device(rom_ctx *ctx, int sample, double *out)
{
    if (!ctx || !out) return fail(ctx, ROM_ERR_INVALID_ARG, "NULL argument");
    if (!ctx->solved) return fail(ctx, ROM_ERR_STATE, "call rom_solve first");
    if (sample < -1 || sample >= ctx->S) return fail(ctx, ROM_ERR_INVALID_ARG, "bad sample %d", sample);
    if (sample == -1 && batch(ctx))
        return fail(ctx, ROM_ERR_INVALID_ARG,
                    "several grids: read each grid's average with rom_get_grid_average");
    CK(cudaSetDevice(ctx->device));
    const size_t nI = (size_t)(sample >= 0 ? sample_cells(ctx, sample) : n_cells(ctx));
    if (sample >= 0) {
        CK(extract_phi(ctx, sample, out));
        ++ctx->launches;
    } else {
        CK(cudaMemcpyAsync(out, ctx->avg.p, nI * sizeof(double), cudaMemcpyDeviceToDevice,
                           ctx->stream));
    }
    return ROM_OK;
}

int rom_get_iterations(rom_ctx *ctx, int32_t *iters, double *residuals)
{
    if (!ctx) return ROM_ERR_INVALID_ARG;
    if (!ctx->solved) return fail(ctx, ROM_ERR_STATE, "call rom_solve first");
    for (int s = 0; s < ctx->S; ++s) {
        if (iters) iters[s] = ctx->h_iters[s];
        if (residuals) residuals[s] = ctx->h_resid[s];
    }
    return ROM_OK;
}

int rom_get_balance(rom_ctx *ctx, double *leakage, double *balance, double *phi_min)
{
    if (!ctx) return ROM_ERR_INVALID_ARG;
    if (!ctx->solved) return fail(ctx, ROM_ERR_STATE, "call rom_solve first");
    const bool have = has_balance(ctx);
    for (int s = 0; s < ctx->S; ++s) {
        if (leakage) leakage[s] = have ? ctx->h_leak[s] : NAN;
        if (balance) balance[s] = have ? ctx->h_bal[s] : NAN;
        if (phi_min) phi_min[s] = ctx->h_phimin[s];
    }
    return ROM_OK;
}

int rom_get_grid_average(rom_ctx *ctx, int grid, double *out)
{
    if (!ctx || !out) return fail(ctx, ROM_ERR_INVALID_ARG, "NULL argument");
    if (!ctx->solved) return fail(ctx, ROM_ERR_STATE, "call rom_solve first");
    const int n = batch(ctx) ? ctx->n_grids : 1;
    if (grid < 0 || grid >= n) return fail(ctx, ROM_ERR_INVALID_ARG, "bad grid %d", grid);
    CK(cudaSetDevice(ctx->device));
    const long long o = batch(ctx) ? ctx->avg_off[grid] : 0;
    const long long len = batch(ctx) ? ctx->avg_off[grid + 1] - o : n_cells(ctx);
    CK(cudaMemcpyAsync(out, (const double *)ctx->avg.p + o, (size_t)len * sizeof(double),
                       cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return ROM_OK;
}

int rom_get_partial_sum(rom_ctx *ctx, double *sum_out, int64_t *count_out)
{
    if (!ctx) return ROM_ERR_INVALID_ARG;
    if (!ctx->solved) return fail(ctx, ROM_ERR_STATE, "call rom_solve first");
    if (batch(ctx))
        return fail(ctx, ROM_ERR_UNSUPPORTED,
                    "several grids: the partial sums are per grid (rom_get_grid_average)");
    CK(cudaSetDevice(ctx->device));
    if (sum_out) {
        CK(cudaMemcpyAsync(sum_out, ctx->sum.p, (size_t)n_cells(ctx) * sizeof(double),
                           cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    if (count_out) *count_out = ctx->S;
    return ROM_OK;
}

}  // extern "C"
