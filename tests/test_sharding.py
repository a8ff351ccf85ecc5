"""Sample sharding over processes: the host logic of the multi-GPU path with the
gloo backend and two ranks.  On CPU each rank's samples are solved by the FP64
oracle; on the GPU (one device shared by the two ranks, whose kernels never wait
on one another) each rank solves its range through the library.  Either way the
all-reduced average must equal the average of one process over all samples."""
import os
import socket

import numpy as np
import pytest

from paper_2407_12527_gb300.sharding import sample_range

N_TOTAL = 7
SEED = 4321


def test_sample_range_partitions():
    for n in (0, 1, 5, 64, 257):
        for world in (1, 2, 3, 8):
            got = [sample_range(r, world, n) for r in range(world)]
            covered = [i for first, cnt in got for i in range(first, first + cnt)]
            assert covered == list(range(n))
            assert max(c for _, c in got) - min(c for _, c in got) <= 1
    with pytest.raises(ValueError):
        sample_range(2, 2, 10)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    import rom_workloads as W
    return W.example_2_1(I=24, J=20)


def _rank_main(rank, world, port, out_path):
    import torch.distributed as dist
    from oracle import oracle as O
    from paper_2407_12527_gb300.sharding import allreduce_average, sample_range as sr

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = _problem()
    first, cnt = sr(rank, world, N_TOTAL)
    sets = [O.rom_ordinates_xy(SEED, first + k, 2, 2) for k in range(cnt)]
    r = O.solve_xy(p.I, p.J, p.bounds, p.sigma_t, p.sigma_s, p.q, sets, tol=1e-12)
    avg = allreduce_average(r["phi"].sum(axis=0), cnt)
    if rank == 0:
        np.save(out_path, avg)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_average_equals_single_process(tmp_path):
    import torch.multiprocessing as mp
    from oracle import oracle as O

    out = str(tmp_path / "avg.npy")
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    got = np.load(out)
    p = _problem()
    sets = [O.rom_ordinates_xy(SEED, k, 2, 2) for k in range(N_TOTAL)]
    want = O.rom_average(O.solve_xy(p.I, p.J, p.bounds, p.sigma_t, p.sigma_s, p.q, sets,
                                    tol=1e-12)["phi"])
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-15)


# ---------------------------------------------- the library on each rank (GPU)
#
# Two gloo ranks share the one GPU: each solves its own contiguous range of
# samples through the C ABI (global sample indices for the seeded draws, uneven
# ordinate counts) and the host all-reduce adds the FP64 partial sums.  The
# ranks' kernels never wait on one another; the only exchange is on the host.

GPU_SEED = 97531
GPU_NZ = [1, 2, 2, 1, 3, 2, 1]
GPU_NT = [2, 2, 4, 3, 2, 1, 4]


def _gpu_problem():
    import rom_workloads as W
    return W.example_2_1(I=45, J=38)


def _gpu_rank_main(rank, world, port, out_path):
    import torch.distributed as dist
    from paper_2407_12527_gb300 import rom as R
    from paper_2407_12527_gb300.sharding import allreduce_average, sample_range as sr

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = _gpu_problem()
    first, cnt = sr(rank, world, len(GPU_NZ))
    ctx = R.RomContext(0)
    ctx.set_grid(p.I, p.J, p.bounds, p.sigma_t, p.sigma_s, p.q)
    ctx.set_ordinates_seed(GPU_SEED, GPU_NZ[first:first + cnt], GPU_NT[first:first + cnt],
                           first_sample=first)
    ctx.set_options(tol=1e-6, max_iter=200)
    ctx.solve()
    phi = np.stack([ctx.scalar_flux(k) for k in range(cnt)])
    psum, n = ctx.partial_sum()
    ctx.close()
    avg = allreduce_average(psum, n)
    np.save(out_path + ".rank%d.npy" % rank, phi)
    if rank == 0:
        np.save(out_path, avg)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.gpu
def test_two_rank_library_average_equals_one_context_and_oracle(tmp_path):
    import torch
    import torch.multiprocessing as mp
    from oracle import oracle as O
    from parity_util import rel

    assert torch.cuda.is_available()
    import __graft_entry__
    __graft_entry__.build()
    from paper_2407_12527_gb300 import rom as R

    out = str(tmp_path / "avg_gpu.npy")
    mp.start_processes(_gpu_rank_main, args=(2, _free_port(), out), nprocs=2,
                       start_method="spawn", join=True)
    got = np.load(out)
    per_rank = np.concatenate([np.load(out + ".rank%d.npy" % r) for r in range(2)])

    p = _gpu_problem()
    ctx = R.RomContext(0)
    ctx.set_grid(p.I, p.J, p.bounds, p.sigma_t, p.sigma_s, p.q)
    ctx.set_ordinates_seed(GPU_SEED, GPU_NZ, GPU_NT)
    ctx.set_options(tol=1e-6, max_iter=200)
    ctx.solve()
    one = np.stack([ctx.scalar_flux(k) for k in range(len(GPU_NZ))])
    one_avg = ctx.scalar_flux(-1)
    ctx.close()

    # the same samples, whichever process swept them (draws from global indices)
    for k in range(len(GPU_NZ)):
        assert rel(per_rank[k], one[k]) < 1e-5, k
    assert rel(got, one_avg) < 1e-5
    sets = [O.rom_ordinates_xy(GPU_SEED, k, GPU_NZ[k], GPU_NT[k]) for k in range(len(GPU_NZ))]
    ref = O.solve_xy(p.I, p.J, p.bounds, p.sigma_t, p.sigma_s, p.q, sets, tol=1e-12)
    assert rel(got, O.rom_average(ref["phi"])) < 1e-5
