// sweep2d_batch.cu -- the X-Y sweep kernels of sweep2d_impl.cuh for batches of
// several grids (SweepArgs::grids): each work item takes the sizes, cell widths
// and coefficient block of its sample's grid, and its sample's state starts at
// SweepArgs::soff; sigma_T is read per cell.  H = 4 rows per step; H = 2 is in
// sweep2d_batch_h2.cu.
#define SWEEP2D_ROWS 4
#define SWEEP2D_WITH_DENSE 0
#define SWEEP2D_BATCH 1
#include "sweep2d_impl.cuh"

namespace romk {

cudaError_t launch_sweep2d_batch_rows2(const SweepArgs &a, int n_items, int nwarps, int G,
                                       int scheme, int mom, cudaStream_t st);

cudaError_t launch_sweep2d_batch(const SweepArgs &a, int n_items, int nwarps, int G, int scheme,
                                 int mom, int rows, cudaStream_t st)
{
    if (rows == 2) return launch_sweep2d_batch_rows2(a, n_items, nwarps, G, scheme, mom, st);
    if (rows != 4) return cudaErrorInvalidValue;
    return launch_rows(a, n_items, nwarps, G, scheme, false, mom, st);
}

}  // namespace romk
