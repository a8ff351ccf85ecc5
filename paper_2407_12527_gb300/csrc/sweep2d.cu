// sweep2d.cu -- transport sweep of the discrete ordinate system (K1).
//
// One sweep solves, for every ordinate l of every active sample, the
// diamond-difference cell equations of eq. (equ_random) on the I x J grid
// (Sec. 2) in upwind order, given the scattering source of the previous source
// iteration, and adds the scalar-flux moments of each work item to its sample:
//   psi_c = (S_l + a psi_xin + b psi_yin) / (sigma_T + a + b),
//   DD:   a = 2|c|/dx, b = 2|s|/dy, psi_out = 2 psi_c - psi_in,
//   step: a =  |c|/dx, b =  |s|/dy, psi_out = psi_c,
//   phi += w_l psi_c   (and Jx += w_l c_l psi_c, Jy += w_l s_l psi_c).
//
// GB300 mapping.  A CTA sweeps one work item: up to G ordinates of one
// quadrant of one sample, i.e. ordinates that share the upwind order.  Lanes
// run along x: lane g owns the 8 cells [8g, 8g+8) of every row (one aligned
// 32-byte sector of FP32), and the CTA covers the full width with
// ceil(I/8) lanes.  The sweep advances along y in blocks of H rows; lane g
// processes block t - d at step t, where d is its distance in lanes from the
// inflow face, so the x-dependence (the upwind x-flux of H rows x G ordinates)
// passes one lane per step by a warp shuffle (shared memory plus one barrier
// per step between warps).  The y-dependence (8 columns x G ordinates) stays
// in registers across steps.  Each cell is visited once per ordinate group:
// source loads and moment reductions are full sectors, and the G ordinates and the
// H x 8 block give the instruction-level parallelism that hides the
// FMA -> MUL -> FMA chain of each cell.  Ordinates are processed in pairs with
// the packed FP32x2 instructions of sm_100+ (__ffma2_rn, __fmul2_rn), which
// halves the issue slots of the cell arithmetic.  The source rows of the next
// block are loaded one step ahead into registers.  No ordinate or cell values
// are stored (except psi in the dense mode): each item adds its moments to its
// sample's accumulator with vector reductions (red.global.add.v4.f32), which the
// combine reads and clears.  The order of those additions follows the timing of
// the items, so the last bits of phi can differ from run to run.
//
// The kernels live in sweep2d_impl.cuh; this unit compiles them for H = 4 rows
// per step (every source mode) and sweep2d_h2.cu for H = 2 (moment modes), the
// better shape for large batches, picked by the work-item autotuner.
#define SWEEP2D_ROWS 4
#define SWEEP2D_WITH_DENSE 1
#include "sweep2d_impl.cuh"

namespace romk {

cudaError_t launch_sweep2d(const SweepArgs &a, int n_items, int nwarps, int G, int scheme,
                           bool homog, int mom, int rows, cudaStream_t st)
{
    if (rows == 2) return launch_sweep2d_rows2(a, n_items, nwarps, G, scheme, homog, mom, st);
    if (rows != 4) return cudaErrorInvalidValue;
    return launch_rows(a, n_items, nwarps, G, scheme, homog, mom, st);
}

}  // namespace romk
