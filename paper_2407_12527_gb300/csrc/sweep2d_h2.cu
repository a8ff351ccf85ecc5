// sweep2d_h2.cu -- the X-Y sweep kernels of sweep2d_impl.cuh for H = 2 rows per
// wavefront step (isotropic and linear-kernel moment modes).
#define SWEEP2D_ROWS 2
#define SWEEP2D_WITH_DENSE 0
#include "sweep2d_impl.cuh"

namespace romk {

cudaError_t launch_sweep2d_rows2(const SweepArgs &a, int n_items, int nwarps, int G, int scheme,
                                 bool homog, int mom, cudaStream_t st)
{
    return launch_rows(a, n_items, nwarps, G, scheme, homog, mom, st);
}

}  // namespace romk
