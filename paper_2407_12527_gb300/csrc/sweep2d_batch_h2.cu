// sweep2d_batch_h2.cu -- the X-Y sweep kernels for batches of several grids
// (sweep2d_batch.cu) with H = 2 rows per wavefront step.
#define SWEEP2D_ROWS 2
#define SWEEP2D_WITH_DENSE 0
#define SWEEP2D_BATCH 1
#include "sweep2d_impl.cuh"

namespace romk {

cudaError_t launch_sweep2d_batch_rows2(const SweepArgs &a, int n_items, int nwarps, int G,
                                       int scheme, int mom, cudaStream_t st)
{
    return launch_rows(a, n_items, nwarps, G, scheme, false, mom, st);
}

}  // namespace romk
