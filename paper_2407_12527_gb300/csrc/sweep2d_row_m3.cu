// sweep2d_row_m3.cu -- the one-row-per-step X-Y sweep (sweep2d_row.cuh) for one
// grid in the linear-kernel mode (three source and flux moments), both schemes.
#include "sweep2d_row.cuh"

namespace romk {

cudaError_t launch_sweep2d_row_m3(const SweepArgs &a, int n_items, int nwarps, int G, int scheme,
                                  bool homog, cudaStream_t st)
{
    if (scheme == 1) return row_launch<3, 1, false>(a, n_items, nwarps, G, homog, st);
    return row_launch<3, 0, false>(a, n_items, nwarps, G, homog, st);
}

}  // namespace romk
