// sweep2d_row_dense.cu -- the one-row-per-step X-Y sweep (sweep2d_row.cuh) for one
// grid in the dense operator mode: one source per ordinate in, psi of every
// ordinate out (FP32, or split BF16 for the tensor-core contraction), both schemes.
#include "sweep2d_row.cuh"

namespace romk {

cudaError_t launch_sweep2d_row_dense(const SweepArgs &a, int n_items, int nwarps, int G,
                                     int scheme, bool homog, cudaStream_t st)
{
    if (scheme == 1) return row_launch<0, 1, false>(a, n_items, nwarps, G, homog, st);
    return row_launch<0, 0, false>(a, n_items, nwarps, G, homog, st);
}

}  // namespace romk
