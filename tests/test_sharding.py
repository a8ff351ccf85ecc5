"""Sample sharding over processes: the host logic of the multi-GPU path, run on
CPU with the gloo backend and two ranks.  Each rank's samples are solved by the
FP64 oracle (there is no GPU here); the all-reduced average must equal the
average of one process over all samples."""
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
