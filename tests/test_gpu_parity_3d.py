"""GPU parity of the 3D (x-y-z) path against the FP64 oracle, through the C ABI.

Same bar as the X-Y tests: relative l2 difference of each sample's scalar flux
<= 1e-5 (FP32 sweeps against FP64).  The grids cover one tile with ragged
strips and row blocks, several x tiles, several y tiles and both, so that the
tile hand-off buffers and the inter-warp rings are all exercised.
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




def gpu_solve3(R, I, J, K, bounds, st, ss, q, sets=None, seed=None, nz=None, nt=None,
               inflow=None, inflow_ord=None, **opts):
    ctx = R.RomContext(0)
    ctx.set_grid3(I, J, K, bounds, st, ss, q)
    if sets is not None:
        ctx.set_ordinates([(o.c, o.s, o.zeta, o.w) for o in sets])
    else:
        ctx.set_ordinates_seed_xyz(seed, nz, nt)
    sizes = W.face_sizes3(I, J, K)
    off = np.concatenate([[0], np.cumsum(sizes)])
    if inflow is not None:
        for f in range(6):
            ctx.set_inflow_isotropic(f, inflow[off[f]:off[f + 1]])
    if inflow_ord is not None:
        for f in range(6):
            ctx.set_inflow_ordinates(f, np.ascontiguousarray(inflow_ord[:, off[f]:off[f + 1]]))
    ctx.set_options(**opts)
    st_ = ctx.solve()
    n = ctx.n_samples
    phi = np.stack([ctx.scalar_flux(k) for k in range(n)])
    avg = ctx.scalar_flux(-1)
    it, res = ctx.iterations()
    ctx.close()
    return {"phi": phi, "avg": avg, "iters": it, "resid": res, "stats": st_}


def sphere_sets(Ms, seed):
    return [O.Ordinates(*W.random_directions_sphere(M, seed=seed + k, weights="random"))
            for k, M in enumerate(Ms)]


# ----------------------------------------------------------- ordinates

def test_seeded_octant_sets_match_oracle(rom):
    nz, nt = [1, 2, 2, 3], [1, 3, 4, 2]
    seed = 987654321
    ctx = rom.RomContext(0)
    ctx.set_ordinates_seed_xyz(seed, nz, nt, first_sample=3)
    mt = 8 * int(np.dot(nz, nt))
    dirs, w = ctx.get_ordinates(mt)
    ctx.close()
    off = 0
    for k in range(len(nz)):
        o = O.rom_ordinates_xyz(seed, 3 + k, nz[k], nt[k])
        sl = slice(off, off + o.M)
        np.testing.assert_allclose(dirs[sl, 2], o.zeta, rtol=0, atol=4e-16)
        np.testing.assert_allclose(dirs[sl, 0], o.c, rtol=0, atol=2e-15)
        np.testing.assert_allclose(dirs[sl, 1], o.s, rtol=0, atol=2e-15)
        np.testing.assert_array_equal(w[sl], o.w)
        np.testing.assert_array_equal(np.sign(dirs[sl]), np.sign(np.stack([o.c, o.s, o.zeta], 1)))
        off += o.M


# ------------------------------------------------------- fixed-K parity

GRIDS3 = [
    (5, 4, 3, (0.0, 1.0, 0.0, 0.8, 0.0, 0.6)),          # one partial strip, one lane
    (13, 37, 7, (0.0, 1.3, -0.2, 0.9, 0.1, 0.5)),       # ragged strip and row block
    (16, 16, 16, (0.0, 1.0, 0.0, 1.0, 0.0, 1.0)),       # exact strips
    (131, 6, 5, (0.0, 2.0, 0.0, 0.3, 0.0, 0.4)),        # three x tiles, ragged
    (9, 133, 4, (0.0, 0.3, 0.0, 2.0, 0.0, 0.3)),        # two y tiles, ragged
    (136, 130, 3, (0.0, 1.0, 0.0, 1.0, 0.0, 0.2)),      # 3 x 2 tiles
    (1, 1, 9, (0.0, 0.1, 0.0, 0.1, 0.0, 1.0)),          # one column of cells
]


@pytest.mark.parametrize("tile_g", [1, 2])
@pytest.mark.parametrize("scheme", ["dd", "step"])
@pytest.mark.parametrize("grid", GRIDS3, ids=[f"{g[0]}x{g[1]}x{g[2]}" for g in GRIDS3])
def test_fixed_k_parity_3d(rom, scheme, grid, tile_g):
    """Explicit sets with odd per-octant counts, so G = 2 items include single ones."""
    I, J, K, bounds = grid
    st, ss, q = W.random_medium3(I, J, K, seed=I * 131 + J * 7 + K)
    sets = sphere_sets((9, 16, 3), seed=I + J + K)
    n_it = 3
    gpu = gpu_solve3(rom, I, J, K, bounds, st, ss, q, sets=sets, scheme=rom.SCHEME[scheme],
                     fixed_iters=n_it, tile_g=tile_g)
    ref = O.solve_xyz(I, J, K, bounds, st, ss, q, sets, scheme=scheme, fixed_iters=n_it)
    for k in range(len(sets)):
        assert rel(gpu["phi"][k], ref["phi"][k]) < TOL, k
    assert list(gpu["iters"]) == [n_it] * len(sets)
    np.testing.assert_allclose(gpu["avg"], ref["phi"].mean(axis=0), rtol=0,
                               atol=TOL * np.abs(ref["phi"]).max())


@pytest.mark.parametrize("scheme", ["dd", "step"])
def test_seeded_rom_converged_3d(rom, scheme):
    """Converged 3D ROM (octant sets from the seed) on a lognormal medium."""
    n = 20
    G = W.gaussian_random_field(n, 3.0, seed=77)
    st = np.exp(-0.125 + 0.5 * G) * 4.0
    ss = 0.8 * st
    q = np.zeros((n, n, n))
    q[8:12, 8:12, 8:12] = 1.0
    bounds = (0.0, 1.0, 0.0, 1.0, 0.0, 1.0)
    nz, nt, seed = [2, 1, 2], [3, 2, 2], 4242
    gpu = gpu_solve3(rom, n, n, n, bounds, st, ss, q, seed=seed, nz=nz, nt=nt,
                     scheme=rom.SCHEME[scheme], tol=1e-6, max_iter=300)
    sets = [O.rom_ordinates_xyz(seed, k, nz[k], nt[k]) for k in range(len(nz))]
    ref = O.solve_xyz(n, n, n, bounds, st, ss, q, sets, scheme=scheme, tol=1e-12, max_iter=2000)
    for k in range(len(nz)):
        assert rel(gpu["phi"][k], ref["phi"][k]) < 2e-5, k
        assert abs(int(gpu["iters"][k]) - int(ref["iters"][k])) <= 40


def test_equilibrium_inflow_3d(rom):
    I, J, K, st, ss, q = 11, 7, 9, 2.0, 1.2, 0.9
    val = q / (st - ss)
    inflow = np.full(sum(W.face_sizes3(I, J, K)), val)
    gpu = gpu_solve3(rom, I, J, K, (0, 1, 0, 1.3, 0, 0.7), np.full((K, J, I), st),
                     np.full((K, J, I), ss), np.full((K, J, I), q), seed=11, nz=[2, 1], nt=[3, 2],
                     inflow=inflow, fixed_iters=40)
    np.testing.assert_allclose(gpu["phi"], val, rtol=2e-5)


@pytest.mark.parametrize("grid", [GRIDS3[1], GRIDS3[5]], ids=["one_tile", "3x2_tiles"])
def test_isotropic_inflow_3d(rom, grid):
    I, J, K, bounds = grid
    st, ss, q = W.random_medium3(I, J, K, seed=5)
    inflow = np.random.default_rng(6).uniform(0.0, 1.5, size=sum(W.face_sizes3(I, J, K)))
    sets = sphere_sets((8, 5), seed=60)
    gpu = gpu_solve3(rom, I, J, K, bounds, st, ss, q, sets=sets, inflow=inflow, fixed_iters=2)
    ref = O.solve_xyz(I, J, K, bounds, st, ss, q, sets, fixed_iters=2, inflow=inflow)
    for k in range(len(sets)):
        assert rel(gpu["phi"][k], ref["phi"][k]) < TOL, k


def test_per_ordinate_inflow_reads_only_incoming_values_3d(rom):
    """Per-ordinate inflow whose incoming values equal an isotropic inflow gives the
    isotropic result, whatever the outgoing values hold."""
    I, J, K, bounds = GRIDS3[1]
    st, ss, q = W.random_medium3(I, J, K, seed=15)
    sizes = W.face_sizes3(I, J, K)
    iso = np.random.default_rng(16).uniform(0.0, 1.0, size=sum(sizes))
    sets = sphere_sets((10, 7), seed=70)
    dirs = np.concatenate([np.stack([o.c, o.s, o.zeta], 1) for o in sets])
    per = np.tile(iso, (dirs.shape[0], 1))
    off = np.concatenate([[0], np.cumsum(sizes)])
    garbage = np.random.default_rng(17).uniform(5.0, 9.0, size=per.shape)
    for f in range(6):
        comp, neg = f // 2, f % 2
        outgoing = (dirs[:, comp] < 0) if neg == 0 else (dirs[:, comp] >= 0)
        per[outgoing, off[f]:off[f + 1]] = garbage[outgoing, off[f]:off[f + 1]]
    gpu = gpu_solve3(rom, I, J, K, bounds, st, ss, q, sets=sets, inflow_ord=per, fixed_iters=2)
    ref = O.solve_xyz(I, J, K, bounds, st, ss, q, sets, fixed_iters=2, inflow=iso)
    for k in range(len(sets)):
        assert rel(gpu["phi"][k], ref["phi"][k]) < TOL, k


def test_many_items_per_cta_3d(rom):
    """More ordinates than resident CTAs: every CTA sweeps a list of items."""
    I, J, K, bounds = 12, 10, 6, (0.0, 1.0, 0.0, 1.0, 0.0, 0.5)
    st, ss, q = W.random_medium3(I, J, K, seed=21)
    nz, nt = [2] * 40, [3] * 40
    gpu = gpu_solve3(rom, I, J, K, bounds, st, ss, q, seed=99, nz=nz, nt=nt, fixed_iters=2)
    sets = [O.rom_ordinates_xyz(99, k, 2, 3) for k in range(40)]
    ref = O.solve_xyz(I, J, K, bounds, st, ss, q, sets, fixed_iters=2)
    for k in range(40):
        assert rel(gpu["phi"][k], ref["phi"][k]) < TOL, k


def test_graph_loop_equals_host_loop_3d(rom):
    I, J, K, bounds = GRIDS3[1]
    st, ss, q = W.random_medium3(I, J, K, seed=31)
    kw = dict(seed=5, nz=[2, 2], nt=[3, 2], tol=1e-5, max_iter=200)
    a = gpu_solve3(rom, I, J, K, bounds, st, ss, q, check_every=0, **kw)
    b = gpu_solve3(rom, I, J, K, bounds, st, ss, q, check_every=3, **kw)
    # atomic accumulation order may differ between runs: compare within FP32 rounding
    assert rel(a["phi"], b["phi"]) < 1e-6
    assert np.all(np.abs(a["iters"] - b["iters"]) <= 1)


def test_3d_rejects_unsupported_and_bad_faces(rom):
    ctx = rom.RomContext(0)
    n = 6
    ctx.set_grid3(n, n, n, (0, 1, 0, 1, 0, 1), 1.0, 0.5, 1.0)
    ctx.set_ordinates_seed_xyz(1, [1], [1])
    with pytest.raises(rom.RomError):
        ctx.set_inflow_isotropic(6, np.zeros(n * n))
    ctx.set_kernel("linear", 0.5)
    with pytest.raises(rom.RomError) as e:
        ctx.solve()
    assert e.value.code == -7
    ctx.close()
    ctx = rom.RomContext(0)
    ctx.set_grid(4, 4, (0, 1, 0, 1), 1.0, 0.5, 1.0)
    with pytest.raises(rom.RomError):
        ctx.set_inflow_isotropic(4, np.zeros(4))  # no z faces in X-Y
    ctx.close()


@pytest.mark.slow
def test_full_size_lognormal_cube_sampled(rom):
    """The 128^3 lognormal workload in the benchmark's launch configuration (64
    samples x 48 ordinates); two samples checked against the oracle at 3 sweeps."""
    p = W.lognormal_cube()
    o = p.ordinates
    gpu = gpu_solve3(rom, p.I, p.J, p.K, p.bounds, p.sigma_t, p.sigma_s, p.q, seed=4000,
                     nz=o["n_zeta"], nt=o["n_theta"], fixed_iters=3)
    for k in (0, 37):
        s = O.rom_ordinates_xyz(4000, k, o["n_zeta"][k], o["n_theta"][k])
        ref = O.solve_xyz(p.I, p.J, p.K, p.bounds, p.sigma_t, p.sigma_s, p.q, [s],
                          fixed_iters=3)
        assert rel(gpu["phi"][k], ref["phi"][0]) < TOL, k


@pytest.mark.parametrize("g", [1, 5])
def test_3d_context_reuse_new_coefficients_and_reseed(rom, g):
    """A 3D grid of the same shape keeps the work items and the graph but must see
    the new coefficients (the diagonal copies are refilled at every solve); a second
    seeded octant set with the same layout must see the new ordinates."""
    I, J, K, bounds = GRIDS3[g]
    ctx = rom.RomContext(0)
    ctx.set_options(fixed_iters=3)
    nz, nt = [2, 1], [1, 3]
    for k, seed in enumerate((41, 42)):
        st, ss, q = W.random_medium3(I, J, K, seed=seed)
        ctx.set_grid3(I, J, K, bounds, st, ss, q)
        first = 4 * k
        ctx.set_ordinates_seed_xyz(17, nz, nt, first_sample=first)
        ctx.solve()
        gpu = np.stack([ctx.scalar_flux(s) for s in range(2)])
        sets = [O.rom_ordinates_xyz(17, first + s, nz[s], nt[s]) for s in range(2)]
        ref = O.solve_xyz(I, J, K, bounds, st, ss, q, sets, fixed_iters=3)["phi"]
        for s in range(2):
            assert rel(gpu[s], ref[s]) < TOL, (k, s)
    ctx.close()
