// sweep2d_row_batch.cu -- the one-row-per-step X-Y sweep (sweep2d_row.cuh) for
// batches of several grids (SweepArgs::grids): each work item takes its grid's
// sizes and coefficient block; sigma_T is read per cell; vacuum boundaries.
#include "sweep2d_row.cuh"

namespace romk {

cudaError_t launch_sweep2d_row_batch(const SweepArgs &a, int n_items, int nwarps, int G,
                                     int scheme, int mom, cudaStream_t st)
{
    if (mom == 1) {
        if (scheme == 1) return row_launch<1, 1, true>(a, n_items, nwarps, G, false, st);
        return row_launch<1, 0, true>(a, n_items, nwarps, G, false, st);
    }
    if (mom == 3) {
        if (scheme == 1) return row_launch<3, 1, true>(a, n_items, nwarps, G, false, st);
        return row_launch<3, 0, true>(a, n_items, nwarps, G, false, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace romk
