"""GPU checks beside the flux: the particle balance of the sweep, the minimum of
phi, divergence detection and the bounded waits between sweep warps.

The balance is the cell balance of eq. (equ_random) (diamond difference or step,
Sec. 2) multiplied by the cell area and summed over cells and ordinates: the
edge terms telescope to the net leakage L through the boundary, so
    L + sum sigma_T phi^k dA = sum_l w_l sum S_l^{k-1} dA
for the k-th sweep.  The oracle computes L from its FP64 boundary values; the
library accumulates it from the sweep's FP32 edges in FP64."""
import numpy as np
import pytest

from oracle import oracle as O
import rom_workloads as W
from parity_util import rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rom():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__
    __graft_entry__.build()
    from paper_2407_12527_gb300 import rom as R
    return R


def _ctx(R, I, J, bounds, st, ss, q, sets, inflow=None, per_ordinate=None, **opts):
    ctx = R.RomContext(0)
    ctx.set_grid(I, J, bounds, st, ss, q)
    ctx.set_ordinates([(o.c, o.s, o.zeta, o.w) for o in sets])
    off = [0, J, 2 * J, 2 * J + I, 2 * J + 2 * I]
    if inflow is not None:
        for f in range(4):
            ctx.set_inflow_isotropic(f, inflow[off[f]:off[f + 1]])
    if per_ordinate is not None:
        for f in range(4):
            ctx.set_inflow_ordinates(f, np.ascontiguousarray(per_ordinate[:, off[f]:off[f + 1]]))
    ctx.set_options(**opts)
    return ctx


@pytest.mark.parametrize("scheme", ["dd", "step"])
@pytest.mark.parametrize("inflow", ["vacuum", "isotropic", "per_ordinate"])
@pytest.mark.parametrize("grid", [(37, 29), (70, 9), (300, 41)], ids=["37x29", "70x9", "300x41"])
@pytest.mark.parametrize("tile_g", [1, 2, 4])
@pytest.mark.parametrize("rows", [4, 1])
def test_balance_and_leakage_match_oracle(rom, scheme, inflow, grid, tile_g, rows):
    """Ragged grids, random media, random inflow: the GPU's net leakage of the
    last sweep equals the oracle's (FP32 sweep against FP64), and its balance
    closes to FP32 rounding (blocked and one-row sweep kernels)."""
    I, J = grid
    bounds = (0.0, 1.3, -0.2, 0.9)
    st, ss, q = W.random_medium(I, J, seed=I + 7 * J)
    sets = [O.Ordinates(*W.random_directions(M, seed=200 + M, weights="random"))
            for M in (6, 11)]
    iso = W.random_inflow(I, J, seed=3) if inflow == "isotropic" else None
    per = W.random_inflow(I, J, seed=4, per_ordinate_M=17) if inflow == "per_ordinate" else None
    K = 5
    ctx = _ctx(rom, I, J, bounds, st, ss, q, sets, inflow=iso, per_ordinate=per,
               scheme=rom.SCHEME[scheme], fixed_iters=K, tile_g=tile_g, rows_per_step=rows)
    stats = ctx.solve()
    leak, bal, mn = ctx.balance()
    phi = np.stack([ctx.scalar_flux(k) for k in range(2)])
    ctx.close()
    if per is not None:
        ref = O.solve_xy(I, J, bounds, st, ss, q, sets, scheme=scheme, fixed_iters=K, inflow=per,
                         inflow_per_ordinate=True)
    else:
        ref = O.solve_xy(I, J, bounds, st, ss, q, sets, scheme=scheme, fixed_iters=K, inflow=iso)
    for k in range(2):
        assert rel(phi[k], ref["phi"][k]) < 1e-5
        scale = abs(ref["leak"][k]) + np.sum(st * ref["phi"][k]) * (1.3 / I) * (1.1 / J)
        assert abs(leak[k] - ref["leak"][k]) < 1e-5 * scale, k
        assert bal[k] < 1e-5, k
        assert mn[k] == pytest.approx(phi[k].min(), rel=1e-6, abs=1e-12)
    assert stats["balance_max"] == pytest.approx(bal.max())
    assert stats["phi_min"] == pytest.approx(mn.min())


@pytest.mark.parametrize("rows", [4, 1])
def test_balance_linear_kernel_and_seeded_sets(rom, rows):
    """Linear kernel (three source moments): sum_l w_l S_l = S0 sum w + S1x sum w c +
    S1y sum w s enters the balance; seeded ROM sets, converged solve."""
    p = W.example_2_1(I=50, J=44, g=0.9)
    ctx = rom.RomContext(0)
    ctx.set_grid(p.I, p.J, p.bounds, p.sigma_t, p.sigma_s, p.q)
    ctx.set_ordinates_seed(31, [2, 3], [2, 3])
    ctx.set_kernel("linear", 0.9)
    ctx.set_options(tol=1e-6, max_iter=300, rows_per_step=rows)
    stats = ctx.solve()
    leak, bal, mn = ctx.balance()
    ctx.close()
    sets = [O.rom_ordinates_xy(31, k, n, n) for k, n in enumerate((2, 3))]
    it = stats["iterations_max"]
    ref = O.solve_xy(p.I, p.J, p.bounds, p.sigma_t, p.sigma_s, p.q, sets, kernel="linear",
                     g=0.9, fixed_iters=it)
    assert np.all(bal < 1e-5)
    for k in range(2):
        assert leak[k] == pytest.approx(ref["leak"][k], rel=2e-5)


def test_balance_not_computed_in_dense_mode(rom):
    I, J = 24, 20
    ctx = rom.RomContext(0)
    ctx.set_grid(I, J, (0, 1, 0, 1), 1.0, 0.5, 1.0)
    ctx.set_ordinates_seed(3, [2], [2])
    ctx.set_kernel("hg", 0.5)
    ctx.set_options(fixed_iters=3)
    stats = ctx.solve()
    leak, bal, mn = ctx.balance()
    ctx.close()
    assert np.isnan(stats["balance_max"]) and np.isnan(bal[0]) and np.isnan(leak[0])
    assert np.isfinite(mn[0]) and mn[0] >= 0.0


def _divergent_problem():
    """Unnormalised Henyey-Greenstein kernel with g = 0.9 (Remark, Sec. 3.1): with
    16 ordinates the operator w_l' P(u_l', u_l) has row sums far above 1 (the
    diagonal alone is w G(1) / 2 ~ 6), and sigma_S / sigma_T = 0.99 on a domain
    8 mean free paths wide keeps the leakage small, so the spectral radius of the
    source iteration is > 1."""
    I = J = 32
    return I, J, (0.0, 8.0, 0.0, 8.0), 1.0, 0.99, 1.0


def test_divergence_detected(rom):
    I, J, bounds, st, ss, q = _divergent_problem()
    ctx = rom.RomContext(0)
    ctx.set_grid(I, J, bounds, st, ss, q)
    ctx.set_ordinates_seed(5, [2], [2])
    ctx.set_kernel("hg", 0.9)
    ctx.set_options(tol=1e-6, max_iter=500, diverge_window=8)
    with pytest.raises(rom.RomError) as e:
        ctx.solve()
    assert e.value.code == -5
    it, res = ctx.iterations()
    assert 8 <= it[0] < 100 and res[0] > 1e-3
    # the same problem row-normalised (Remark, Sec. 3.1) converges on the same context
    ctx.set_kernel("hg", 0.9, rom.KERNEL_FLAG_NORMALIZE)
    ctx.set_options(tol=1e-6, max_iter=5000)
    ctx.solve()
    ctx.close()


@pytest.mark.parametrize("case", ["xy", "xy_one_warp", "xy_one_row", "3d"])
def test_bounded_waits_report_timeout(rom, case):
    """test_stall_waits makes every sweep warp wait on an mbarrier that nothing
    completes; with a 5 ms bound the sweep gives up, raises its error word and
    returns, rom_solve reports ROM_ERR_TIMEOUT, and the context solves normally
    afterwards."""
    ctx = rom.RomContext(0)
    if case == "3d":
        I = J = K = 16
        ctx.set_grid3(I, J, K, (0, 1, 0, 1, 0, 1), 1.0, 0.5, 1.0)
        ctx.set_ordinates_seed_xyz(3, [1], [1])
    else:
        I, J = (300, 40) if case == "xy" else (40, 30)
        ctx.set_grid(I, J, (0, 1, 0, 1), 1.0, 0.5, 1.0)
        ctx.set_ordinates_seed(3, [1], [2])
    rows = 1 if case == "xy_one_row" else 0
    ctx.set_options(fixed_iters=2, test_stall_waits=1, wait_timeout_ms=5.0, check_every=1,
                    rows_per_step=rows)
    with pytest.raises(rom.RomError) as e:
        ctx.solve()
    assert e.value.code == -8
    ctx.set_options(fixed_iters=2)
    ctx.solve()
    phi = ctx.scalar_flux(0)
    ctx.close()
    assert np.all(np.isfinite(phi)) and phi.max() > 0.0
