"""The no-allocation sweep entry point against the context API.

rom_sweep_xy_noalloc serves callers that must not call cudaMalloc (plug-ins
whose host application owns all device memory, latency-bound paths where an
allocation and its synchronisation are not allowed).  It keeps its scratch in a
fixed array inside the library instead of allocating.  The first test calls it
twice in a row through the C ABI, for both schemes -- the first sweep of source
iteration (source q) and the second one (source sigma_S phi^1 + q) -- and checks
both results against rom_solve with fixed_iters = 1 and 2 on the same
ordinates, within the bar the other GPU parity tests use; the second runs it at
its table and width limits and checks that one ordinate or work item more is
refused.  The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import rom_workloads as W
from parity_util import rel

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def R():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__
    __graft_entry__.build()
    from paper_2407_12527_gb300 import rom
    return rom


def _reference(R, I, J, bounds, st, ss, q, seed, nz, nt, scheme, iters):
    """rom_solve with fixed_iters = k for k in iters, and the ordinates it used."""
    ctx = R.RomContext(0)
    ctx.set_grid(I, J, bounds, st, ss, q)
    ctx.set_ordinates_seed(seed, nz, nt)
    mt = 4 * int(np.dot(nz, nt))
    dirs, w = ctx.get_ordinates(mt)
    ref = []
    for k in iters:
        ctx.set_options(fixed_iters=k, scheme=scheme)
        ctx.solve()
        ref.append(np.stack([ctx.scalar_flux(s) for s in range(len(nz))]))
    ctx.close()
    return np.ascontiguousarray(dirs), np.ascontiguousarray(w), ref


class _Caller:
    """rom_sweep_xy_noalloc through the C ABI on torch's current stream."""

    def __init__(self, R, I, J, dx, dy, scheme, st, m, dirs, w, S):
        import torch
        self.L = R.lib()
        self.dev = torch.device("cuda", 0)
        self.args = (I, J, dx, dy, scheme)
        self.st = torch.tensor(st, dtype=torch.float32, device=self.dev).contiguous()
        self.m = np.ascontiguousarray(m, dtype=np.int32)
        self.dirs, self.w = dirs, w
        self.phi = torch.empty((S, J, I), dtype=torch.float32, device=self.dev)
        self.S = S
        self.err = ctypes.create_string_buffer(256)

    def __call__(self, src):
        import torch
        stream = torch.cuda.current_stream(self.dev)
        I, J, dx, dy, scheme = self.args
        rc = self.L.rom_sweep_xy_noalloc(
            ctypes.c_void_p(stream.cuda_stream), I, J, dx, dy, scheme,
            ctypes.c_void_p(self.st.data_ptr()), self.S,
            self.m.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
            self.dirs.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            self.w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.c_void_p(src.data_ptr()),
            ctypes.c_void_p(self.phi.data_ptr()), self.err, ctypes.sizeof(self.err))
        torch.cuda.synchronize(self.dev)
        return rc


@pytest.mark.parametrize("scheme", [0, 1], ids=["dd", "step"])
def test_noalloc_sweep_matches_solve_twice(R, scheme):
    import torch
    I, J = 61, 47
    bounds = (0.0, 1.3, -0.4, 0.7)
    st, ss, q = W.random_medium(I, J, seed=909)
    nz, nt, seed = [2, 1, 3], [2, 3, 2], 31337
    S = len(nz)
    dirs, w, ref = _reference(R, I, J, bounds, st, ss, q, seed, nz, nt, scheme, (1, 2))
    dx, dy = (bounds[1] - bounds[0]) / I, (bounds[3] - bounds[2]) / J
    m = [4 * a * b for a, b in zip(nz, nt)]
    call = _Caller(R, I, J, dx, dy, scheme, st, m, dirs, w, S)
    dev = call.dev
    src = torch.tensor(np.broadcast_to(q, (S, J, I)), dtype=torch.float32, device=dev).contiguous()

    assert call(src) == 0, call.err.value.decode()     # sweep 1: source q
    first = call.phi.cpu().numpy().astype(np.float64)
    for s in range(S):
        assert rel(first[s], ref[0][s]) < TOL
    ss_d = torch.tensor(ss, dtype=torch.float32, device=dev)
    q_d = torch.tensor(q, dtype=torch.float32, device=dev)
    src.copy_(ss_d[None] * call.phi + q_d[None])       # sweep 2: sigma_S phi^1 + q
    assert call(src) == 0, call.err.value.decode()
    second = call.phi.cpu().numpy().astype(np.float64)
    for s in range(S):
        assert rel(second[s], ref[1][s]) < TOL

    # a problem larger than the fixed scratch array is refused with a message
    big = _Caller(R, 2048, 2048, 1.0, 1.0, scheme, np.ones((1, 1)), m, dirs, w, S)
    big.st, big.phi = call.st, call.phi          # never touched: refused before any work
    assert big(src) == -1 and b"scratch" in big.err.value


def test_noalloc_at_its_limits(R):
    """8192 ordinates in 4096 work items (the two table limits, one sample of
    32 x 64 cells per quadrant) and I = 2048 columns (the width limit), each
    against rom_solve with one sweep; one ordinate or one work item more is
    refused with a message."""
    import torch
    dev = torch.device("cuda", 0)
    for (I, J, nz, nt) in ((24, 20, [32], [64]), (2048, 6, [1], [1])):
        bounds = (0.0, 1.0, 0.0, 0.5)
        st, ss, q = W.random_medium(I, J, seed=I + J)
        dirs, w, ref = _reference(R, I, J, bounds, st, ss, q, 4242, nz, nt, 0, (1,))
        m = [4 * nz[0] * nt[0]]
        call = _Caller(R, I, J, 1.0 / I, 0.5 / J, 0, st, m, dirs, w, 1)
        src = torch.tensor(np.broadcast_to(q, (1, J, I)), dtype=torch.float32,
                           device=dev).contiguous()
        assert call(src) == 0, call.err.value.decode()
        assert rel(call.phi.cpu().numpy()[0], ref[0][0]) < TOL, (I, J)

    # 8193 ordinates: over the ordinate table
    rng = np.random.default_rng(1)
    M = 8193
    th = rng.uniform(0, 2 * np.pi, M)
    z = rng.uniform(0.05, 0.95, M)
    d = np.ascontiguousarray(np.stack([np.sqrt(1 - z * z) * np.cos(th),
                                       np.sqrt(1 - z * z) * np.sin(th), z], 1))
    wt = np.full(M, 1.0 / M)
    call = _Caller(R, 8, 8, 0.1, 0.1, 0, np.ones((8, 8)), [M], d, wt, 1)
    src = torch.ones((1, 8, 8), dtype=torch.float32, device=dev)
    assert call(src) == -1 and b"ordinates exceed" in call.err.value
    # 820 samples of 6 ordinates, 3 in one quadrant: 5 work items each, 4100 in all
    one = np.array([[0.6, 0.6], [0.5, 0.7], [0.7, 0.5], [-0.6, 0.6], [-0.6, -0.6],
                    [0.6, -0.6]])
    zz = np.sqrt(1.0 - np.sum(one ** 2, 1))
    per = np.concatenate([one, zz[:, None]], 1)
    S = 820
    d = np.ascontiguousarray(np.tile(per, (S, 1)))
    wt = np.full(6 * S, 1.0 / 6)
    call = _Caller(R, 8, 8, 0.1, 0.1, 0, np.ones((8, 8)), [6] * S, d, wt, S)
    src = torch.ones((S, 8, 8), dtype=torch.float32, device=dev)
    assert call(src) == -1 and b"work items" in call.err.value
