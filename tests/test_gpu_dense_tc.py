"""GPU parity of the tensor-core dense scattering source (dense_precision = 1).

The dense operator's product D = A Psi runs on the tcgen05 tensor cores in
split BF16 ((A_hi + A_lo)(Psi_hi + Psi_lo), all four products, FP32 accumulation).  The
bar is the one of every other GPU parity test: relative l2 difference of each
sample's scalar flux <= 1e-5 against the FP64 oracle.  The cases cover uneven M
per sample (sample row offsets that are not multiples of the 128-row operand
tile, zero-padded operator columns), grids whose cell count is not a multiple
of the 128-cell tile, full 128 x 128 operators, samples that stop iterating at
different sweeps, and the FP32 CUDA-core path as a second reference.
"""
import numpy as np
import pytest

from oracle import oracle as O
import rom_workloads as W
from parity_util import rel

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def rom():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__
    __graft_entry__.build()
    from paper_2407_12527_gb300 import rom as R
    return R




def gpu_solve(R, I, J, bounds, st, ss, q, seed, nz, nt, kernel="hg", g=0.8, flags=0, **opts):
    ctx = R.RomContext(0)
    ctx.set_grid(I, J, bounds, st, ss, q)
    ctx.set_ordinates_seed(seed, nz, nt)
    ctx.set_kernel(kernel, g, flags)
    ctx.set_options(**opts)
    st_ = ctx.solve()
    phi = np.stack([ctx.scalar_flux(k) for k in range(ctx.n_samples)])
    it, _ = ctx.iterations()
    ctx.close()
    return {"phi": phi, "iters": it, "stats": st_}


@pytest.mark.parametrize("flags", [0, 1, 2])
def test_tc_hg_parity_uneven_m(rom, flags):
    """M = 20, 16, 48 per sample on a 53 x 41 grid (2120 cells: 16 full tiles and a
    ragged one); flags 1 = row-normalised operator, 2 = raw hemisphere kernel."""
    I, J = 53, 41
    bounds = (0.0, 1.0, 0.0, 0.8)
    st, ss, q = W.random_medium(I, J, seed=71, ratio_max=0.8)
    nz, nt = [1, 2, 2], [5, 2, 6]
    gpu = gpu_solve(rom, I, J, bounds, st, ss, q, 73, nz, nt, flags=flags, fixed_iters=5,
                    dense_precision=1)
    sets = [O.rom_ordinates_xy(73, k, nz[k], nt[k]) for k in range(3)]
    ref = O.solve_xy(I, J, bounds, st, ss, q, sets, kernel="hg", g=0.8, fixed_iters=5,
                     normalize_rows=bool(flags & 1), raw=bool(flags & 2))
    for k in range(3):
        assert rel(gpu["phi"][k], ref["phi"][k]) < TOL, k


def test_tc_hg_full_tiles(rom):
    """M = 128 per sample (full 128 x 128 operator), 96 x 96 disc problem."""
    p = W.hg_disc(n=96, n_samples=2)
    nz, nt = [4, 4], [8, 8]
    seed = W.ordinate_seed(3)
    gpu = gpu_solve(rom, p.I, p.J, p.bounds, p.sigma_t, p.sigma_s, p.q, seed, nz, nt,
                    fixed_iters=4, dense_precision=1)
    sets = [O.rom_ordinates_xy(seed, k, 4, 8) for k in range(2)]
    ref = O.solve_xy(p.I, p.J, p.bounds, p.sigma_t, p.sigma_s, p.q, sets, kernel="hg", g=0.8,
                     fixed_iters=4)
    for k in range(2):
        assert rel(gpu["phi"][k], ref["phi"][k]) < TOL, k


def test_tc_equals_fp32_product(rom):
    """Split BF16 on the tensor cores against the FP32 CUDA-core product, same inputs."""
    I, J = 64, 40
    st, ss, q = W.random_medium(I, J, seed=3, ratio_max=0.9)
    nz, nt = [2, 4, 3], [4, 8, 3]
    kw = dict(fixed_iters=6)
    a = gpu_solve(rom, I, J, (0, 1, 0, 1), st, ss, q, 17, nz, nt, dense_precision=0, **kw)
    b = gpu_solve(rom, I, J, (0, 1, 0, 1), st, ss, q, 17, nz, nt, dense_precision=1, **kw)
    for k in range(3):
        assert rel(b["phi"][k], a["phi"][k]) < TOL, k


def test_tc_converged_samples_leave_at_different_sweeps(rom):
    """Converged solve: samples with different M stop at different sweeps, so later
    launches skip the units of finished samples.  Row-normalised operator, so that
    source iteration contracts for every M (an unnormalised Henyey-Greenstein
    operator with few ordinates can have row sums above 1)."""
    I, J = 48, 48
    st, ss, q = W.random_medium(I, J, seed=9, ratio_max=0.9)
    nz, nt = [1, 2, 4, 1], [2, 3, 8, 8]
    gpu = gpu_solve(rom, I, J, (0, 1, 0, 1), st, ss, q, 29, nz, nt, flags=1, tol=1e-6,
                    max_iter=400, dense_precision=1)
    sets = [O.rom_ordinates_xy(29, k, nz[k], nt[k]) for k in range(4)]
    ref = O.solve_xy(I, J, (0, 1, 0, 1), st, ss, q, sets, kernel="hg", g=0.8, tol=1e-12,
                     max_iter=4000, normalize_rows=True)
    for k in range(4):
        assert rel(gpu["phi"][k], ref["phi"][k]) < 2e-5, k
    assert len(set(int(x) for x in gpu["iters"])) > 1


def test_tc_isotropic_dense_equals_moments(rom):
    p = W.example_2_1(I=40, J=36)
    kw = dict(fixed_iters=6)
    a = gpu_solve(rom, p.I, p.J, p.bounds, p.sigma_t, p.sigma_s, p.q, 5, [2, 1], [2, 3],
                  kernel="iso", g=0.0, **kw)
    b = gpu_solve(rom, p.I, p.J, p.bounds, p.sigma_t, p.sigma_s, p.q, 5, [2, 1], [2, 3],
                  kernel="iso", g=0.0, dense_source=1, dense_precision=1, **kw)
    for k in range(2):
        assert rel(b["phi"][k], a["phi"][k]) < TOL, k


def test_tc_rejects_more_than_128_ordinates(rom):
    ctx = rom.RomContext(0)
    ctx.set_grid(8, 8, (0, 1, 0, 1), 1.0, 0.5, 1.0)
    ctx.set_ordinates_seed(1, [4], [9])  # M = 144
    ctx.set_kernel("hg", 0.5)
    ctx.set_options(fixed_iters=1, dense_precision=1)
    with pytest.raises(rom.RomError) as e:
        ctx.solve()
    assert e.value.code == -7
    ctx.close()


def test_tc_hg_disc_full_size_sampled(rom):
    """The 512 x 512 Henyey-Greenstein workload in the benchmark's launch
    configuration (32 samples x 128 ordinates, tensor-core contraction, device-side
    loop) at 3 sweeps; samples 0 and 31 against the oracle."""
    p = W.hg_disc()
    seed = W.ordinate_seed(3)
    S = 32
    gpu = gpu_solve(rom, p.I, p.J, p.bounds, p.sigma_t, p.sigma_s, p.q, seed, [4] * S, [8] * S,
                    fixed_iters=3, dense_precision=1)
    for k in (0, 31):
        ref = O.solve_xy(p.I, p.J, p.bounds, p.sigma_t, p.sigma_s, p.q,
                         [O.rom_ordinates_xy(seed, k, 4, 8)], kernel="hg", g=0.8,
                         fixed_iters=3)
        assert rel(gpu["phi"][k], ref["phi"][0]) < TOL, k


def test_dense_mode_runs_four_rows_per_step(rom):
    """The 2-row sweep shape exists for the moment modes only: a dense-operator solve
    asked for 2 rows per step runs 4 and stays in parity."""
    I, J = 40, 30
    st, ss, q = W.random_medium(I, J, seed=19, ratio_max=0.8)
    gpu = gpu_solve(rom, I, J, (0, 1, 0, 1), st, ss, q, 23, [1, 2], [3, 2], fixed_iters=3,
                    dense_precision=1, rows_per_step=2)
    assert gpu["stats"]["rows_per_step"] == 4
    sets = [O.rom_ordinates_xy(23, k, nz, nt) for k, (nz, nt) in enumerate([(1, 3), (2, 2)])]
    ref = O.solve_xy(I, J, (0, 1, 0, 1), st, ss, q, sets, kernel="hg", g=0.8, fixed_iters=3)
    for k in range(2):
        assert rel(gpu["phi"][k], ref["phi"][k]) < TOL, k


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("scheme", ["dd", "step"])
@pytest.mark.parametrize("homog", [False, True])
@pytest.mark.parametrize("tile_g", [1, 2])
def test_dense_mode_one_row_sweep(rom, precision, scheme, homog, tile_g):
    """The one-row sweep in the dense operator mode (per-ordinate sources in, psi of
    every ordinate out as FP32 or split BF16): ragged 53 x 41 grid, uneven M, uniform
    and varying sigma_T, both schemes, against the oracle."""
    I, J = 53, 41
    bounds = (0.0, 1.0, 0.0, 0.8)
    st, ss, q = W.random_medium(I, J, seed=81, ratio_max=0.8)
    if homog:
        st = np.full((J, I), 2.0)
        ss = np.minimum(ss, 1.6)
    nz, nt = [1, 2, 2], [5, 2, 6]
    gpu = gpu_solve(rom, I, J, bounds, st, ss, q, 83, nz, nt, fixed_iters=4,
                    dense_precision=precision, rows_per_step=1, tile_g=tile_g,
                    scheme=rom.SCHEME[scheme])
    assert gpu["stats"]["rows_per_step"] == 1
    sets = [O.rom_ordinates_xy(83, k, nz[k], nt[k]) for k in range(3)]
    ref = O.solve_xy(I, J, bounds, st, ss, q, sets, kernel="hg", g=0.8, fixed_iters=4,
                     scheme=scheme)
    for k in range(3):
        assert rel(gpu["phi"][k], ref["phi"][k]) < TOL, k


def test_dense_mode_one_row_sweep_inflow_and_two_warps(rom):
    """Dense mode, one-row sweep: per-ordinate inflow on every face and a 300-wide
    grid whose rows span two warps (a shared-memory hand-off per step)."""
    I, J = 300, 23
    bounds = (-1.0, 2.0, 0.0, 0.5)
    st, ss, q = W.random_medium(I, J, seed=91, ratio_max=0.8)
    nz, nt = [1, 2], [2, 3]
    sets = [O.rom_ordinates_xy(93, k, nz[k], nt[k]) for k in range(2)]
    M = sum(o.M for o in sets)
    per = W.random_inflow(I, J, seed=94, per_ordinate_M=M)
    ctx = rom.RomContext(0)
    ctx.set_grid(I, J, bounds, st, ss, q)
    ctx.set_ordinates_seed(93, nz, nt)
    ctx.set_kernel("hg", 0.8)
    off = [0, J, 2 * J, 2 * J + I, 2 * J + 2 * I]
    for f in range(4):
        ctx.set_inflow_ordinates(f, np.ascontiguousarray(per[:, off[f]:off[f + 1]]))
    ctx.set_options(fixed_iters=3, dense_precision=1, rows_per_step=1)
    stats = ctx.solve()
    phi = [ctx.scalar_flux(k) for k in range(2)]
    ctx.close()
    assert stats["rows_per_step"] == 1
    ref = O.solve_xy(I, J, bounds, st, ss, q, sets, kernel="hg", g=0.8, fixed_iters=3,
                     inflow=per, inflow_per_ordinate=True)
    for k in range(2):
        assert rel(phi[k], ref["phi"][k]) < TOL, k
