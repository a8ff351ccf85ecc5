// sweep2d_row_step.cu -- the one-row-per-step X-Y sweep (sweep2d_row.cuh) for one
// grid, step scheme, isotropic moment mode.
#include "sweep2d_row.cuh"

namespace romk {

cudaError_t launch_sweep2d_row_step(const SweepArgs &a, int n_items, int nwarps, int G, bool homog,
                                    cudaStream_t st)
{
    return row_launch<1, 1, false>(a, n_items, nwarps, G, homog, st);
}

}  // namespace romk
