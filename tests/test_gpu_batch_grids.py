"""GPU parity for batches whose samples sit on different X-Y grids.

The ROM samples are independent discrete-ordinate solves (Sec. 3.1), so one
batch may hold samples of several problems: grids of different sizes, extents
and media, each with its own ordinate count.  Every sample is checked against
the FP64 oracle run on that sample's own grid with the same ordinate array
(relative l2 and largest-cell error within 1e-5, as in the other parity
tests), and each grid's sample average (Sec. 4.1) against the average of the
oracle's samples.
"""
import numpy as np
import pytest

from oracle import oracle as O
import rom_workloads as W
from parity_util import rel

pytestmark = pytest.mark.gpu

TOL = 1e-5

# (I, J, bounds): ragged tiles, a grid two warps wide, one column, one row; then
# taller grids on which the one-row sweep reaches its unchecked middle steps
GRIDS = [
    (37, 29, (0.0, 1.3, -0.2, 0.9)),
    (300, 23, (-1.0, 2.0, 0.0, 0.5)),
    (64, 20, (0.0, 1.0, 0.0, 0.4)),
    (1, 9, (0.0, 0.1, 0.0, 1.0)),
    (11, 1, (0.0, 1.0, 0.0, 0.1)),
    (256, 70, (0.0, 1.0, 0.0, 0.3)),   # one warp wide: its second warp idle in the batch
    (300, 64, (0.0, 1.2, 0.0, 0.25)),  # two warps, the second with idle lanes
    (40, 80, (0.0, 0.5, 0.0, 1.0)),    # one warp, most lanes idle
]


@pytest.fixture(scope="module")
def rom():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__
    __graft_entry__.build()
    from paper_2407_12527_gb300 import rom as R
    return R


def make_batch(grid_ids, per_grid, seed0):
    """Media per grid and random ordinate sets with uneven M per sample."""
    grids, sets = [], []
    rng = np.random.default_rng(seed0)
    for p, gi in enumerate(grid_ids):
        I, J, bounds = GRIDS[gi]
        st, ss, q = W.random_medium(I, J, seed=seed0 + 17 * p)
        grids.append((I, J, bounds, st, ss, q))
        for k in range(per_grid[p]):
            M = int(rng.choice([3, 5, 8, 12, 16]))
            sets.append(O.Ordinates(*W.random_directions(M, seed=seed0 + 100 * p + k,
                                                         weights="random")))
    return grids, sets


def solve_batch(R, grids, per_grid, sets=None, seed=None, nz=None, nt=None, kernel="iso", g=0.0,
                **opts):
    ctx = R.RomContext(0)
    ctx.set_grids(grids, per_grid)
    if sets is not None:
        ctx.set_ordinates([(o.c, o.s, o.zeta, o.w) for o in sets])
    else:
        ctx.set_ordinates_seed(seed, nz, nt)
    if kernel != "iso":
        ctx.set_kernel(kernel, g)
    ctx.set_options(**opts)
    stats = ctx.solve()
    n = ctx.n_samples
    phi = [ctx.scalar_flux(k) for k in range(n)]
    avg = [ctx.grid_average(p) for p in range(len(grids))]
    it, res = ctx.iterations()
    leak, bal, mn = ctx.balance()
    ctx.close()
    return {"phi": phi, "avg": avg, "iters": it, "resid": res, "stats": stats, "leak": leak,
            "bal": bal, "min": mn}


def oracle_batch(grids, per_grid, sets, **kw):
    """The oracle on each grid with that grid's samples: phi list and per-grid leak."""
    phi, leak, iters = [], [], []
    s0 = 0
    for p, (I, J, bounds, st, ss, q) in enumerate(grids):
        ref = O.solve_xy(I, J, bounds, st, ss, q, sets[s0:s0 + per_grid[p]], **kw)
        phi += list(ref["phi"])
        leak += list(ref["leak"])
        iters += list(ref["iters"])
        s0 += per_grid[p]
    return phi, np.array(leak), np.array(iters)


@pytest.mark.parametrize("scheme", ["dd", "step"])
@pytest.mark.parametrize("tile_g", [2, 4])
def test_mixed_tall_grids_one_row_sweep(rom, scheme, tile_g):
    """One launch over grids one and two warps wide (a whole warp idle on the
    narrower ones) with enough rows for the unchecked middle steps."""
    per_grid = [2, 2, 2]
    grids, sets = make_batch([5, 6, 7], per_grid, seed0=700)
    K = 3
    gpu = solve_batch(rom, grids, per_grid, sets=sets, scheme=rom.SCHEME[scheme], fixed_iters=K,
                      rows_per_step=1, tile_g=tile_g)
    ref_phi, _, _ = oracle_batch(grids, per_grid, sets, scheme=scheme, fixed_iters=K)
    for k in range(len(sets)):
        assert rel(gpu["phi"][k], ref_phi[k]) < TOL, k
    s0 = 0
    for p in range(3):
        want = O.rom_average(np.stack(ref_phi[s0:s0 + per_grid[p]]))
        assert rel(gpu["avg"][p], want) < TOL, p
        s0 += per_grid[p]


@pytest.mark.parametrize("scheme", ["dd", "step"])
@pytest.mark.parametrize("rows", [4, 2, 1])
@pytest.mark.parametrize("tile_g", [1, 2, 4])
def test_mixed_grids_fixed_k_parity(rom, scheme, rows, tile_g):
    """Three grids (ragged, two warps wide, exact tiles) with uneven M per sample."""
    per_grid = [2, 3, 2]
    grids, sets = make_batch([0, 1, 2], per_grid, seed0=400)
    K = 4
    gpu = solve_batch(rom, grids, per_grid, sets=sets, scheme=rom.SCHEME[scheme], fixed_iters=K,
                      rows_per_step=rows, tile_g=tile_g)
    ref_phi, ref_leak, _ = oracle_batch(grids, per_grid, sets, scheme=scheme, fixed_iters=K)
    for k in range(len(sets)):
        assert gpu["phi"][k].shape == ref_phi[k].shape, k
        assert rel(gpu["phi"][k], ref_phi[k]) < TOL, k
    assert list(gpu["iters"]) == [K] * len(sets)
    assert gpu["stats"]["tile_g"] == tile_g and gpu["stats"]["rows_per_step"] == rows
    # updates counted on each sample's own grid
    upd = sum(K * g[0] * g[1] * len(s.c) for g, s in
              zip([grids[p] for p in range(3) for _ in range(per_grid[p])], sets))
    assert gpu["stats"]["updates"] == upd
    # net leakage of the last sweep against the oracle's (FP32 against FP64)
    owners = [grids[p] for p in range(3) for _ in range(per_grid[p])]
    for k, (I, J, b, st, ss, q) in enumerate(owners):
        dA = (b[1] - b[0]) / I * (b[3] - b[2]) / J
        scale = abs(ref_leak[k]) + np.sum(st * ref_phi[k]) * dA
        assert abs(gpu["leak"][k] - ref_leak[k]) < 1e-5 * scale, k
        assert gpu["bal"][k] < 1e-5, k


def test_degenerate_grids_in_one_batch(rom):
    """One-column and one-row grids next to a two-warp grid."""
    per_grid = [1, 2, 1]
    grids, sets = make_batch([3, 1, 4], per_grid, seed0=77)
    gpu = solve_batch(rom, grids, per_grid, sets=sets, fixed_iters=5)
    ref_phi, _, _ = oracle_batch(grids, per_grid, sets, fixed_iters=5)
    for k in range(len(sets)):
        assert rel(gpu["phi"][k], ref_phi[k]) < TOL, k


@pytest.mark.parametrize("rows", [4, 1])
@pytest.mark.parametrize("kernel", ["iso", "linear"])
def test_mixed_grids_converged_average_and_balance(rom, kernel, rows):
    """Seeded ROM sets of uneven size, converged solves: per-sample flux, each
    grid's sample average, and the particle balance of the last sweep."""
    per_grid = [3, 2]
    grids, _ = make_batch([0, 2], per_grid, seed0=9)
    nz, nt = [1, 2, 2, 1, 3], [2, 2, 3, 4, 3]
    g = 0.7 if kernel == "linear" else 0.0
    gpu = solve_batch(rom, grids, per_grid, seed=31, nz=nz, nt=nt, kernel=kernel, g=g, tol=1e-6,
                      max_iter=500, rows_per_step=rows)
    sets = [O.rom_ordinates_xy(31, k, nz[k], nt[k]) for k in range(5)]
    ref_phi, ref_leak, ref_it = oracle_batch(grids, per_grid, sets, kernel=kernel, g=g, tol=1e-12)
    for k in range(5):
        assert rel(gpu["phi"][k], ref_phi[k]) < TOL, k
    s0 = 0
    for p in range(2):
        ref_avg = O.rom_average(np.stack(ref_phi[s0:s0 + per_grid[p]]))
        assert gpu["avg"][p].shape == ref_avg.shape
        assert rel(gpu["avg"][p], ref_avg) < TOL, p
        s0 += per_grid[p]
    assert np.all(gpu["bal"] < 1e-5)
    for k in range(5):
        assert gpu["min"][k] == pytest.approx(gpu["phi"][k].min(), rel=1e-6, abs=1e-12)


def test_mixed_grids_autotuned_and_graph_vs_host_loop(rom):
    """The autotuned work-item shape and the host-driven loop give the same fluxes."""
    per_grid = [2, 2]
    grids, sets = make_batch([1, 0], per_grid, seed0=5)
    a = solve_batch(rom, grids, per_grid, sets=sets, tile_g=-1, tol=1e-6)
    b = solve_batch(rom, grids, per_grid, sets=sets, tile_g=2, check_every=1, tol=1e-6)
    ref_phi, _, _ = oracle_batch(grids, per_grid, sets, tol=1e-12)
    for k in range(4):
        assert rel(a["phi"][k], ref_phi[k]) < TOL, k
        assert rel(b["phi"][k], ref_phi[k]) < TOL, k
    assert list(a["iters"]) == list(b["iters"])


def test_mixed_grids_refusals_and_return_to_one_grid(rom):
    """Wrong sample counts, inflow, the dense operator and the whole-batch average are
    refused; rom_set_grid then brings the context back to one grid."""
    per_grid = [2, 1]
    grids, sets = make_batch([0, 2], per_grid, seed0=3)
    ctx = rom.RomContext(0)
    try:
        ctx.set_grids(grids, per_grid)
        ctx.set_ordinates([(o.c, o.s, o.zeta, o.w) for o in sets[:2]])
        with pytest.raises(rom.RomError) as e:
            ctx.solve()
        assert e.value.code == -6  # ROM_ERR_STATE
        ctx.set_ordinates([(o.c, o.s, o.zeta, o.w) for o in sets])
        with pytest.raises(rom.RomError) as e:
            ctx.set_inflow_isotropic(0, np.ones(29))
        assert e.value.code == -7  # ROM_ERR_UNSUPPORTED
        ctx.set_kernel("hg", 0.5)
        with pytest.raises(rom.RomError) as e:
            ctx.solve()
        assert e.value.code == -7  # ROM_ERR_UNSUPPORTED
        ctx.set_kernel("iso")
        ctx.set_options(fixed_iters=3)
        ctx.solve()
        with pytest.raises(rom.RomError):
            ctx.scalar_flux(-1)
        with pytest.raises(rom.RomError):
            ctx.grid_average(2)
        with pytest.raises(rom.RomError):
            ctx.partial_sum()
        # invalid grids: zero size, hi <= lo, sigma_S >= sigma_T, no samples
        bad = [(0, 5, (0, 1, 0, 1), 1.0, 0.5, 1.0)]
        with pytest.raises(rom.RomError):
            ctx.set_grids(bad, [1])
        bad = [(4, 5, (0, 1, 1, 1), 1.0, 0.5, 1.0)]
        with pytest.raises(rom.RomError):
            ctx.set_grids(bad, [1])
        bad = [(4, 5, (0, 1, 0, 1), 1.0, 1.0, 1.0)]
        with pytest.raises(rom.RomError):
            ctx.set_grids(bad, [1])
        with pytest.raises(rom.RomError):
            ctx.set_grids(grids, [2, 0])
        # back to one grid on the same context
        I, J, bounds, st, ss, q = grids[0]
        ctx.set_grid(I, J, bounds, st, ss, q)
        ctx.set_ordinates([(o.c, o.s, o.zeta, o.w) for o in sets[:2]])
        ctx.set_options(fixed_iters=3)
        ctx.solve()
        ref = O.solve_xy(I, J, bounds, st, ss, q, sets[:2], fixed_iters=3)
        for k in range(2):
            assert rel(ctx.scalar_flux(k), ref["phi"][k]) < TOL
        assert rel(ctx.scalar_flux(-1), O.rom_average(ref["phi"])) < TOL
    finally:
        ctx.close()


def test_one_grid_batch_equals_single_grid(rom):
    """A batch of one grid gives the single-grid solve's fluxes and average."""
    I, J, bounds = GRIDS[0]
    st, ss, q = W.random_medium(I, J, seed=12)
    sets = [O.Ordinates(*W.random_directions(M, seed=M, weights="random")) for M in (4, 9, 6)]
    b = solve_batch(rom, [(I, J, bounds, st, ss, q)], [3], sets=sets, fixed_iters=6)
    ctx = rom.RomContext(0)
    try:
        ctx.set_grid(I, J, bounds, st, ss, q)
        ctx.set_ordinates([(o.c, o.s, o.zeta, o.w) for o in sets])
        ctx.set_options(fixed_iters=6)
        ctx.solve()
        for k in range(3):
            assert rel(b["phi"][k], ctx.scalar_flux(k)) < 1e-6
        assert rel(b["avg"][0], ctx.scalar_flux(-1)) < 1e-6
        assert rel(ctx.grid_average(0), ctx.scalar_flux(-1)) == 0.0
    finally:
        ctx.close()
