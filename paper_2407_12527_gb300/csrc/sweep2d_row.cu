// sweep2d_row.cu -- the one-row-per-step X-Y sweep kernels (sweep2d_row.cuh) for
// one grid: the diamond-difference isotropic moment mode here, and the dispatch
// to the other translation units (sweep2d_row_step.cu: step scheme;
// sweep2d_row_m3.cu: linear-kernel moments; sweep2d_row_dense.cu: the dense
// operator mode; sweep2d_row_batch.cu: batches of several grids), which build in
// parallel.
#include "sweep2d_row.cuh"

namespace romk {

cudaError_t launch_sweep2d_row_step(const SweepArgs &a, int n_items, int nwarps, int G, bool homog,
                                    cudaStream_t st);
cudaError_t launch_sweep2d_row_m3(const SweepArgs &a, int n_items, int nwarps, int G, int scheme,
                                  bool homog, cudaStream_t st);
cudaError_t launch_sweep2d_row_dense(const SweepArgs &a, int n_items, int nwarps, int G,
                                     int scheme, bool homog, cudaStream_t st);

cudaError_t launch_sweep2d_row(const SweepArgs &a, int n_items, int nwarps, int G, int scheme,
                               bool homog, int mom, cudaStream_t st)
{
    if (mom == 3) return launch_sweep2d_row_m3(a, n_items, nwarps, G, scheme, homog, st);
    if (mom == 0) return launch_sweep2d_row_dense(a, n_items, nwarps, G, scheme, homog, st);
    if (mom != 1) return cudaErrorInvalidValue;
    if (scheme == 1) return launch_sweep2d_row_step(a, n_items, nwarps, G, homog, st);
    return row_launch<1, 0, false>(a, n_items, nwarps, G, homog, st);
}

}  // namespace romk
