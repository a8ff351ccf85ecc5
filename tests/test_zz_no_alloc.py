"""The no-allocation sweep entry point against the context API.

rom_sweep_xy_noalloc serves callers that must not call cudaMalloc (code that
runs while a graph is captured elsewhere, plug-ins whose host owns all device
memory, latency-bound paths).  It keeps its scratch in a fixed array inside the
library instead of allocating.  This test calls it twice in a row through the
C ABI -- the first sweep of source iteration (source q) and the second one
(source sigma_S phi^1 + q) -- and checks both results against rom_solve with
fixed_iters = 1 and 2 on the same ordinates, within the relative l2 bar the
other GPU parity tests use.  The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import rom_workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-5


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_sweep_matches_solve_twice():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__
    __graft_entry__.build()
    from paper_2407_12527_gb300 import rom as R

    I, J = 61, 47
    bounds = (0.0, 1.3, -0.4, 0.7)
    st, ss, q = W.random_medium(I, J, seed=909)
    nz, nt, seed = [2, 1, 3], [2, 3, 2], 31337

    # reference: the context API, one and two source-iteration sweeps
    ctx = R.RomContext(0)
    ctx.set_grid(I, J, bounds, st, ss, q)
    ctx.set_ordinates_seed(seed, nz, nt)
    mt = 4 * int(np.dot(nz, nt))
    dirs, w = ctx.get_ordinates(mt)
    ref = []
    for k in (1, 2):
        ctx.set_options(fixed_iters=k)
        ctx.solve()
        ref.append(np.stack([ctx.scalar_flux(s) for s in range(len(nz))]))
    ctx.close()

    L = R.lib()
    dev = torch.device("cuda", 0)
    S = len(nz)
    m = np.array([4 * a * b for a, b in zip(nz, nt)], dtype=np.int32)
    dirs = np.ascontiguousarray(dirs)
    w = np.ascontiguousarray(w)
    st_d = torch.tensor(st, dtype=torch.float32, device=dev).contiguous()
    src = torch.tensor(np.broadcast_to(q, (S, J, I)), dtype=torch.float32, device=dev).contiguous()
    phi = torch.empty((S, J, I), dtype=torch.float32, device=dev)
    err = ctypes.create_string_buffer(256)
    stream = torch.cuda.current_stream(dev)
    dx, dy = (bounds[1] - bounds[0]) / I, (bounds[3] - bounds[2]) / J

    def call():
        rc = L.rom_sweep_xy_noalloc(
            ctypes.c_void_p(stream.cuda_stream), I, J, dx, dy, 0,
            ctypes.c_void_p(st_d.data_ptr()), S, m.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
            dirs.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.c_void_p(src.data_ptr()),
            ctypes.c_void_p(phi.data_ptr()), err, ctypes.sizeof(err))
        assert rc == 0, err.value.decode()
        torch.cuda.synchronize(dev)
        return phi.cpu().numpy().astype(np.float64)

    first = call()                                     # sweep 1: source q
    for s in range(S):
        assert rel(first[s], ref[0][s]) < TOL
    ss_d = torch.tensor(ss, dtype=torch.float32, device=dev)
    q_d = torch.tensor(q, dtype=torch.float32, device=dev)
    src.copy_(ss_d[None] * phi + q_d[None])            # sweep 2: sigma_S phi^1 + q
    second = call()
    for s in range(S):
        assert rel(second[s], ref[1][s]) < TOL

    # a problem larger than the fixed scratch array is refused with a message
    big_I, big_J = 2048, 2048
    rc = L.rom_sweep_xy_noalloc(
        ctypes.c_void_p(stream.cuda_stream), big_I, big_J, 1.0, 1.0, 0,
        ctypes.c_void_p(st_d.data_ptr()), S, m.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
        dirs.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.c_void_p(src.data_ptr()),
        ctypes.c_void_p(phi.data_ptr()), err, ctypes.sizeof(err))
    assert rc == -1 and b"scratch" in err.value
