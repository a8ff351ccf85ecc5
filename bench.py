#!/usr/bin/env python
"""Benchmark of the ROM hot path on GB300: cell-ordinate updates per second.

Workload (one "step" = one pass of the whole hot path over one batch):
  point source, 256 x 256 cells on [-1,1]^2, sigma_T = 1, sigma_S = 0.9
  (isotropic), q = exp(-r^2 / (2 * 0.02^2)), vacuum inflow; one batch = 64 ROM
  samples of M = 16 ordinates (2 x 2 cells per quadrant, Sec. 4.2) drawn on the
  device from a seed (every step draws fresh samples), source iteration of every
  sample to a relative change of 1e-6 (device-side loop), FP64 sample average.
  Synthetic inputs (rom_workloads.point_source); no dataset is involved.

value: total updates (sum over samples of cells * M * sweeps) / device time of
the steps, CUDA events on the library's stream, inputs resident in HBM, L2
flushed between steps (outside the timed events).  Multi-GPU: one process per
GPU, each solving its own disjoint samples (weak scaling, no collective on the
data path), time = max over ranks.

--impl reference times the FP64 CPU oracle on the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import rom_workloads as W  # noqa: E402

METRIC = "cell-ordinate updates/s (ROM source iteration, 1 GB300)"
UNIT = "updates/s"
FLOP_PER_UPDATE = 11  # diamond difference, homogeneous sigma_T: 5 FMA + 1 MUL
FLOP_PER_UPDATE_HET = 13  # heterogeneous sigma_T: + 1 add + 1 reciprocal per cell-ordinate
FLOP_PER_UPDATE_3D = 17   # 3D, heterogeneous: 3 FMA + add + reciprocal + MUL, 3 FMA outflows, 1 FMA phi
TOL = 1e-6
DENSE_SWEEP_BYTES_PER_UPDATE = 8  # dense-mode sweep: FP32 source read + BF16 hi/lo psi written


class Workload:
    """One benchmark workload: a problem of rom_workloads, its ordinate sets per
    step (seeded ROM partitions, or one deterministic DOM set) and kernel."""

    def __init__(self, name, problem, desc, nz=None, nt=None, quad=None, kernel="iso", g=0.0,
                 cfg_index=1):
        self.name, self.p, self.desc = name, problem, desc
        self.nz, self.nt, self.quad = nz, nt, quad
        self.kernel, self.g = kernel, g
        self.seed = W.ordinate_seed(cfg_index)
        self.dim = 3 if hasattr(problem, "K") else 2

    @property
    def cells(self):
        return self.p.I * self.p.J * (self.p.K if self.dim == 3 else 1)

    @property
    def samples(self):
        return 1 if self.quad else len(self.nz)

    def m_total(self):
        if self.quad:
            from paper_2407_12527_gb300 import quadrature_xy
            return quadrature_xy(*self.quad)[0].shape[0]
        per = 8 if self.dim == 3 else 4
        return int(sum(per * a * b for a, b in zip(self.nz, self.nt)))


def make_workload(name):
    partition = W.partition
    if name == "point_source":
        p = W.point_source()
        return Workload(name, p, "point_source_256 (256x256 on [-1,1]^2, sigma_T=1, sigma_S=0.9 "
                        "isotropic, Gaussian q std 0.02, vacuum): ROM 64 samples x 16 ordinates, "
                        "SI to 1e-6", nz=[2] * 64, nt=[2] * 64, cfg_index=1)
    if name == "point_source_dom":
        p = W.point_source()
        return Workload(name, p, "point_source_256, plain DOM with the 2D uniform set N = 8 "
                        "(256 ordinates), SI to 1e-6", quad=("uniform", 8, 0), cfg_index=1)
    if name == "dom_small":
        p = W.dom_small()
        return Workload(name, p, "dom_small_32x32 (sigma_T=1, sigma_S=0.5, central 8x8 source), "
                        "DOM product set 4 Gauss-Legendre polar x 8 azimuthal = 32, SI to 1e-6",
                        quad=("product_gl", 4, 8), cfg_index=0)
    if name == "checkerboard":
        p = W.checkerboard()
        parts = [partition(m) for m in p.ordinates["m_quadrant"]]
        return Workload(name, p, "checkerboard_448 (7x7 blocks of 64x64; absorber sigma_T=10, "
                        "background sigma_T=1, sigma_S=0.9; centre q=1): 256 ROM samples, M "
                        "uniform in {8,16,32,64}, one launch per sweep, SI to 1e-6",
                        nz=[a for a, _ in parts], nt=[b for _, b in parts], cfg_index=2)
    if name == "hg_disc":
        p = W.hg_disc()
        return Workload(name, p, "hg_disc_512 (512x512, sigma_T=1, sigma_S=0.95, Henyey-Greenstein "
                        "g=0.8, q=1 in a disc r<=0.05): ROM 32 samples x 128 ordinates, dense "
                        "operator contraction per sweep, SI to 1e-6", nz=[4] * 32, nt=[8] * 32,
                        kernel="hg", g=0.8, cfg_index=3)
    if name == "lognormal_cube":
        p = W.lognormal_cube()
        o = p.ordinates
        return Workload(name, p, "lognormal_cube_128 (128^3 on [0,1]^3, sigma_T lognormal mean 1, "
                        "log-std 0.5, correlation 8 cells; sigma_S=0.8 sigma_T isotropic; q=1 on "
                        "the central 8^3; vacuum): ROM 64 samples x 48 ordinates (8 octants x 2 x 3), "
                        "SI to 1e-6", nz=o["n_zeta"], nt=o["n_theta"], cfg_index=4)
    raise SystemExit(f"unknown workload {name}")


WL = None  # the workload of this run (set in main)
ARGS = None  # the command line of this run


def workload_config(extra=None):
    p = WL.p
    cfg = {
        "workload": WL.desc, "grid": [p.I, p.J] + ([p.K] if WL.dim == 3 else []),
        "samples_per_step": WL.samples,
        "ordinates_per_step": WL.m_total(), "si_tol": TOL, "scheme": "diamond difference",
        "kernel": WL.kernel + (f" g={WL.g}" if WL.g else ""),
        "dense_product": (("split BF16 x3, tcgen05 tensor cores, FP32 accumulate"
                           if ARGS.dense_precision == 1 else "FP32 CUDA cores")
                          if WL.kernel == "hg" else None),
        "l2": "flushed between steps (256 MiB write outside the timed events)",
    }
    if extra:
        cfg.update(extra)
    return cfg


# ------------------------------------------------------------------ clocks

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200",
                                          "-i", str(self.dev)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def traffic_record(name, source_file, samples_now, shape=None):
    """DRAM bytes of one full launch (every sample active) of a kernel, from the
    committed ncu capture profiles/<name>.traffic.json, scaled from the captured
    batch to samples_now samples; None when the kernel source differs from the
    one captured (sha256) or no record exists.  Records with a "shapes" table
    hold one capture per work-item shape (e.g. "G2H1": 2 ordinates per item, one
    row per step), each with the source file it was built from."""
    import hashlib
    tpath = os.path.join(ROOT, "profiles", name + ".traffic.json")
    if not os.path.exists(tpath):
        return None
    with open(tpath) as f:
        tr = json.load(f)
    if "shapes" in tr:
        rec = tr["shapes"].get(shape)
        if rec is None:
            return None
        source_file = rec["source_file"]
    else:
        rec = tr
    if source_file is None:
        return None
    spath = os.path.join(ROOT, "paper_2407_12527_gb300", "csrc", source_file)
    with open(spath, "rb") as f:
        digest = hashlib.sha256(f.read()).hexdigest()
    if rec.get("source_sha256") != digest:
        return None
    return rec["dram_bytes_per_launch"] * samples_now / tr["samples"]


def measured_hbm_gbs():
    """Measured copy bandwidth of this GPU pool (MEASURED_PEAKS.json), else the
    fallback figure of an earlier GB300 measurement."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"])
    except Exception:
        return 6800.0


# ------------------------------------------------------------------ dist

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def barrier_max(x: float, world: int, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier_sum(x: float, world: int, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------ CPU oracle

def oracle_sets(first: int, count: int):
    """The oracle's ordinate sets for samples first .. first+count-1 of the workload
    (its own generator and quadratures)."""
    from oracle import oracle as O
    if WL.quad:
        kind, n1, n2 = WL.quad
        maker = {"uniform": lambda: O.quad_uniform_xy(n1), "gauss": lambda: O.quad_gauss_xy(n1),
                 "product_gl": lambda: O.quad_product_gl_xy(n1, n2)}[kind]
        return [maker()]
    S = WL.samples
    gen = O.rom_ordinates_xyz if WL.dim == 3 else O.rom_ordinates_xy
    return [gen(WL.seed, first + k, WL.nz[(first + k) % S], WL.nt[(first + k) % S])
            for k in range(count)]


def oracle_rate(budget_s: float, max_samples: int, first: int = 0):
    """The FP64 oracle, as it stands, on consecutive samples of the workload until
    the time budget is used (the dense kernel: one source-iteration sweep per
    sample, its cost being M^2 per cell): returns (updates/s, samples, threads,
    updates, seconds)."""
    from oracle import oracle as O
    p = WL.p
    threads = O.max_threads()
    upd, n, m_max = 0, 0, 1
    t0 = time.perf_counter()
    while n < max_samples:
        o = oracle_sets(first + n, 1)[0]
        kw = {"fixed_iters": 1} if WL.kernel == "hg" else {"tol": TOL}
        if WL.dim == 3:
            r = O.solve_xyz(p.I, p.J, p.K, p.bounds, p.sigma_t, p.sigma_s, p.q, [o],
                            allow_not_converged=True, **kw)
        else:
            r = O.solve_xy(p.I, p.J, p.bounds, p.sigma_t, p.sigma_s, p.q, [o], kernel=WL.kernel,
                           g=WL.g, allow_not_converged=True, **kw)
        upd += WL.cells * o.M * int(r["iters"][0])
        m_max = max(m_max, o.M)
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return upd / dt, n, min(threads, m_max), upd, dt


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        oracle_rate(0.0, 1)
    # each step: consecutive samples of the workload for a share of a ~1 minute budget
    per_step = max(0.02, args.ref_total / max(args.steps, 1))
    t_tot, upd_tot, ns_tot = 0.0, 0, 0
    threads = 1
    for k in range(args.steps):
        rate, ns, threads, upd, dt = oracle_rate(per_step, WL.samples,
                                                 first=WL.samples * (k + 1))
        t_tot += dt
        upd_tot += upd
        ns_tot += ns
    value = upd_tot / t_tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": workload_config({"reference": "FP64 CPU oracle (oracle/rom_oracle.c, OpenMP)"}),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{ns_tot} ordinate sets of the workload over {args.steps} "
                                   f"steps (each step about {per_step:.2f} s of CPU work)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ ours

def run_ours(args):
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2407_12527_gb300 import RomContext

    p = WL.p
    S = WL.samples
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def setup(ctx):
        if WL.kernel != "iso":
            ctx.set_kernel(WL.kernel, WL.g)

    ctx = RomContext(local)
    ctx.set_stream(stream.cuda_stream)
    st_d, ss_d, q_d = (torch.tensor(a, dtype=torch.float32, device=dev).contiguous()
                       for a in (p.sigma_t, p.sigma_s, p.q))
    torch.cuda.synchronize(dev)
    if WL.dim == 3:
        ctx.set_grid3_device(p.I, p.J, p.K, p.bounds, st_d, ss_d, q_d)
    else:
        ctx.set_grid_device(p.I, p.J, p.bounds, st_d, ss_d, q_d)
    setup(ctx)
    ctx.set_options(tol=TOL, check_every=args.check_every, tile_g=args.tile_g,
                    rows_per_step=args.rows_per_step,
                    dense_precision=args.dense_precision)

    def first_sample(step):
        return (step * world + rank) * S

    def set_ordinates(c, step):
        if WL.quad:
            if step == 0 or getattr(c, "_quad_set", False) is False:
                c.set_quadrature(*WL.quad)
                c._quad_set = True
        elif WL.dim == 3:
            c.set_ordinates_seed_xyz(WL.seed, WL.nz, WL.nt, first_sample=first_sample(step))
        else:
            c.set_ordinates_seed(WL.seed, WL.nz, WL.nt, first_sample=first_sample(step))

    def one_step(step):
        set_ordinates(ctx, step)
        return ctx.solve(allow_not_converged=True)

    for k in range(args.warmup):
        one_step(10_000 + k)
    torch.cuda.synchronize(dev)

    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize(dev)
    ms, upd, launches, iters = [], 0, 0, []
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s = one_step(k)
        e1.record(stream)
        stream.synchronize()
        ms.append(e0.elapsed_time(e1))
        upd += s["updates"]
        launches += (0 if WL.quad else 1) + s["kernel_launches"]  # ordinate generation + solve
        iters.append(s["iterations_max"])
    torch.cuda.synchronize(dev)
    barrier(world)
    clk = clocks.stop()
    t_rank = sum(ms) / 1e3
    t_max = barrier_max(t_rank, world, dev)
    upd_all = barrier_sum(float(upd), world, dev)
    value = upd_all / t_max

    if args.only_timed:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                              "steps": args.steps, "warmup": args.warmup,
                              "ms_per_step": 1e3 * t_max / args.steps, "only_timed": True,
                              "workload": WL.name}))
        ctx.close()
        return 0

    # roofline: the same steps with CUDA events around every sweep (and, for the dense
    # operator, every contraction) launch
    ctx.set_options(tol=TOL, time_kernels=1, check_every=8, tile_g=args.tile_g,
                    rows_per_step=args.rows_per_step,
                    dense_precision=args.dense_precision)
    sweep_ms, sweep_upd, sweep_n, src_ms, src_n = 0.0, 0, 0, 0.0, 0
    src_flop, src_bytes = 0.0, 0.0
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        s = one_step(k)
        sweep_ms += s["sweep_ms"]
        sweep_upd += s["updates"]
        sweep_n += s["sweep_launches"]
        src_ms += s["source_ms"]
        src_n += s["source_launches"]
        if WL.kernel == "hg":  # 2 M^2 flops per cell and contraction, per active sample
            it, _ = ctx.iterations()
            M = 4 * WL.nz[0] * WL.nt[0]
            src_flop += 2.0 * M * M * p.I * p.J * float(np.sum(it))
            # algorithmic HBM bytes of a contraction: psi read + sources written, 4 B each
            src_bytes += 8.0 * M * p.I * p.J * float(np.sum(it))
    ctx.set_options(tol=TOL, check_every=args.check_every, tile_g=args.tile_g,
                    rows_per_step=args.rows_per_step,
                    dense_precision=args.dense_precision)
    peak_tflops = 152 * 128 * 2 * 2070e6 / 1e12
    homog = float(np.min(p.sigma_t)) == float(np.max(p.sigma_t))
    fpu = FLOP_PER_UPDATE_3D if WL.dim == 3 else (FLOP_PER_UPDATE if homog else FLOP_PER_UPDATE_HET)
    hbm_peak = measured_hbm_gbs()
    tc = WL.kernel == "hg" and args.dense_precision == 1
    if WL.kernel == "hg" and src_ms > 0 and tc:
        achieved = src_bytes / (src_ms / 1e3) / 1e9
        kernel_name, n_l, avg_us, fu = ("dense_tc_kernel (K4, tcgen05 split BF16)", src_n,
                                        1e3 * src_ms / max(src_n, 1), None)
    elif WL.kernel == "hg" and src_ms > 0:
        achieved = src_flop / (src_ms / 1e3) / 1e12
        kernel_name, n_l, avg_us, fu = ("dense_source_kernel (K4, FP32 SIMT GEMM)", src_n,
                                        1e3 * src_ms / max(src_n, 1), None)
    else:
        achieved = sweep_upd * fpu / (sweep_ms / 1e3) / 1e12
        kernel_name = ("sweep3d_kernel (K9)" if WL.dim == 3 else
                       "sweep2d_row_kernel (K1, one row per step)" if s["rows_per_step"] == 1
                       else "sweep2d_kernel (K1, %d rows per step)" % s["rows_per_step"])
        kernel_name, n_l, avg_us, fu = (kernel_name, sweep_n, 1e3 * sweep_ms / max(sweep_n, 1), fpu)
    # DRAM bytes of one full launch from the committed ncu captures, used only
    # while the kernel source is the one that was captured
    traffic = None
    if WL.name == "point_source":
        traffic = traffic_record("sweep2d_point_source_256", None, WL.samples,
                                 shape="G%dH%d" % (s["tile_g"], s["rows_per_step"]))
    elif WL.name == "lognormal_cube" and s["tile_g"] == 2:
        traffic = traffic_record("sweep3d_lognormal_cube_128", "sweep3d.cu", WL.samples)
    elif WL.name == "checkerboard" and s["tile_g"] == 4 and s["rows_per_step"] == 2:
        traffic = traffic_record("sweep2d_checkerboard_448", "sweep2d_impl.cuh", WL.samples)
    if tc and src_ms > 0:
        roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved / hbm_peak,
                    "traffic": traffic_record("dense_tc_hg_disc_512", "dense_tc.cu", WL.samples),
                    "traffic_note": "DRAM read+write bytes of one launch with every sample "
                                    "active (ncu, scaled by samples); achieved counts the "
                                    "algorithmic bytes, psi (BF16 hi + lo) read and FP32 sources "
                                    "written, 8 B per cell and ordinate",
                    "kernel": kernel_name, "launches": n_l, "avg_launch_us": avg_us,
                    "contraction_tflops": src_flop / (src_ms / 1e3) / 1e12,
                    "sweep_avg_launch_us": 1e3 * sweep_ms / max(sweep_n, 1),
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy bandwidth)"}
        if sweep_ms > src_ms:
            # the dense-mode sweep takes longer than the contraction: it is the dominant
            # kernel, bound by HBM (its per-ordinate source read, 4 B, and psi written as
            # BF16 hi + lo, 4 B, per cell-ordinate update)
            sw = sweep_upd * DENSE_SWEEP_BYTES_PER_UPDATE / (sweep_ms / 1e3) / 1e9
            secondary = dict(roofline)
            roofline = {"bound": "hbm", "achieved": sw, "peak": hbm_peak, "unit": "GB/s",
                        "frac": sw / hbm_peak,
                        "traffic": traffic_record("sweep2d_dense_hg_disc_512",
                                                  "sweep2d_impl.cuh", WL.samples),
                        "traffic_note": "DRAM read+write bytes of one launch with every sample "
                                        "active (ncu, scaled by samples); achieved counts the "
                                        "algorithmic bytes, 8 B per cell-ordinate update",
                        "kernel": "sweep2d_kernel (K1, dense mode: per-ordinate sources in, "
                                  "split-BF16 psi out)",
                        "launches": sweep_n, "avg_launch_us": 1e3 * sweep_ms / max(sweep_n, 1),
                        "bytes_per_update": DENSE_SWEEP_BYTES_PER_UPDATE,
                        "sweep_share_of_sweep_plus_contraction": sweep_ms / (sweep_ms + src_ms),
                        "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy bandwidth)",
                        "secondary": secondary}
    else:
        roofline = None
    if roofline is None:
        roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tflops,
                    "unit": "TFLOP/s", "frac": achieved / peak_tflops, "traffic": traffic,
                    "traffic_note": "DRAM read+write bytes of one sweep launch with every "
                                    "sample active (ncu, scaled by samples)",
                    "kernel": kernel_name, "launches": n_l, "avg_launch_us": avg_us,
                    "flop_per_update": fu,
                    "sweep_avg_launch_us": 1e3 * sweep_ms / max(sweep_n, 1),
                    "tile_g": s["tile_g"], "rows_per_step": s["rows_per_step"],
                    "peak_source": "FP32 CUDA cores: 152 SM x 128 lanes x 2 flop x 2070 MHz"}
        if "sweep" in kernel_name and sweep_ms > 0:
            # the same kernel against HBM: per cell and sample the source moments read
            # and the flux moments written (4 B each), sigma_T, sigma_S, q shared by the
            # samples, divided over the sample's ordinates
            mom = 3 if WL.kernel == "linear" else 1
            m_avg = WL.m_total() / WL.samples
            bpu = (8.0 * mom + 12.0 / WL.samples) / m_avg
            gbs = sweep_upd * bpu / (sweep_ms / 1e3) / 1e9
            roofline["secondary"] = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak,
                                     "unit": "GB/s", "frac": gbs / hbm_peak,
                                     "bytes_per_update": bpu,
                                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy bandwidth)"}

    # end to end through the C ABI with host buffers
    ctx2 = RomContext(local)
    setup(ctx2)
    ctx2.set_options(tol=TOL, tile_g=args.tile_g, rows_per_step=args.rows_per_step,
                     dense_precision=args.dense_precision)
    st_h, ss_h, q_h = (np.ascontiguousarray(a, dtype=np.float64) for a in
                       (p.sigma_t, p.sigma_s, p.q))
    e2e_upd, e2e_t = 0, 0.0
    for k in range(args.warmup + args.steps):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        if WL.dim == 3:
            ctx2.set_grid3(p.I, p.J, p.K, p.bounds, st_h, ss_h, q_h)
        else:
            ctx2.set_grid(p.I, p.J, p.bounds, st_h, ss_h, q_h)
        ctx2._quad_set = False
        set_ordinates(ctx2, k)
        s = ctx2.solve(allow_not_converged=True)
        phi_bar = ctx2.scalar_flux(-1)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            e2e_upd += s["updates"]
            e2e_t += dt
    assert np.isfinite(phi_bar).all()
    e2e_t = barrier_max(e2e_t, world, dev)
    e2e_upd = barrier_sum(float(e2e_upd), world, dev)
    e2e = {"value": e2e_upd / e2e_t, "unit": UNIT,
           "h2d_bytes_per_step": 3 * WL.cells * 8, "d2h_bytes_per_step": WL.cells * 8}
    ctx2.close()
    ctx.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, ns, threads, _, dt = oracle_rate(args.cpu_budget, S)
        what = "one source-iteration sweep of each" if WL.kernel == "hg" else "solved to 1e-6"
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"first {ns} of the {S} ordinate sets of one step, one after another, "
                         f"{what} ({dt:.1f} s)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": workload_config({"sweeps_per_step_max": max(iters),
                                       "parallelism": f"{world} replicas, disjoint samples"}),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk,
        }
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------ ROM vs DOM

def run_rom_vs_dom(args):
    """GPU time for ROM and for plain DOM to reach a relative l2 error of the scalar
    flux of args.target (1e-3) against a fine-ordinate FP64 reference.

    Reference: the FP64 oracle with the 2D Gaussian set N = args.ref_n (2 N (N + 1)
    ordinates; N = 200: 80400), source iteration to 1e-12, cross-checked against
    N = args.ref_check_n (its relative l2 difference is reported and must be far below
    the target).  DOM: the uniform set N = 2 ... 32 (4 N^2 ordinates), one solve each
    to the library tolerance (time = that solve).  ROM: M = 4 m ordinates per sample
    for m in args.rom_m (M = 16, 36, 64), samples solved in batches, the running
    average compared after each batch (time = cumulative GPU time of the batches);
    for each M the first t whose running average is within the target, repeated over
    args.rom_seeds seeds, median reported.  The bias floor of each M is the
    least-squares fit of err(t)^2 = B^2 + V / t over the seeds' curves (the Monte
    Carlo part falls as t^(-1/2), Sec. 4.1); ROM cannot reach a target below B.
    Problems: the 256 x 256 point source (isotropic), Example 2.1, or the
    Henyey-Greenstein disc (g = 0.8, sigma_S = 0.95) reduced to args.rvd_n cells per
    side (the FP64 dense reference costs M^2 per cell and sweep).  The disc runs with
    row-normalised kernel matrices on both sides (the normalisation the Remark of
    Sec. 3.1 offers for sigma_S / sigma_T near 1): unnormalised, a 16-ordinate set
    puts w P(u, u) = (1 + g) / (1 - g)^2 / 16 = 2.8 on the diagonal alone, the
    source iteration's spectral radius exceeds 1 and the solve diverges.  A ROM run
    stops at args.rom_max samples or after args.rom_max_ms of GPU time."""
    import torch
    from oracle import oracle as O
    import __graft_entry__
    __graft_entry__.build()
    from paper_2407_12527_gb300 import RomContext
    from paper_2407_12527_gb300.rom import KERNEL_FLAG_NORMALIZE

    if args.rvd_problem == "point_source":
        p = W.point_source()
    elif args.rvd_problem == "example_2_1":
        p = W.example_2_1()
    else:
        p = W.hg_disc(n=args.rvd_n)
    kw = {} if p.kernel == "iso" else {"kernel": p.kernel, "g": p.g}
    norm = p.kernel == "hg"
    if norm:
        kw["normalize_rows"] = True

    def reference(N):
        t = time.perf_counter()
        o = O.quad_gauss_xy(N) if args.ref_kind == "gauss" else O.quad_uniform_xy(N)
        r = O.solve_xy(p.I, p.J, p.bounds, p.sigma_t, p.sigma_s, p.q, [o], tol=1e-12,
                       **kw)["phi"][0]
        return r, o.M, time.perf_counter() - t

    ref, ref_m, ref_s = reference(args.ref_n)
    nref = float(np.linalg.norm(ref))

    def rel(phi):
        return float(np.linalg.norm(phi - ref) / nref)

    chk = None
    if args.ref_check_n > 0:
        r2, m2, s2 = reference(args.ref_check_n)
        chk = {"N": args.ref_check_n, "M": m2, "rel_l2_to_reference": rel(r2), "host_s": s2}

    ctx = RomContext(0)
    ctx.set_grid(p.I, p.J, p.bounds, p.sigma_t, p.sigma_s, p.q)
    if p.kernel != "iso":
        ctx.set_kernel(p.kernel, p.g, KERNEL_FLAG_NORMALIZE if norm else 0)
    ctx.set_options(tol=TOL, tile_g=-1, dense_precision=args.dense_precision)
    dom = []
    for N in args.dom_n:
        ctx.set_quadrature("uniform", N)
        if p.kernel == "hg":  # the tensor-core product takes at most 128 ordinates
            ctx.set_options(tol=TOL, tile_g=-1,
                            dense_precision=args.dense_precision if 4 * N * N <= 128 else 0)
        ctx.solve(allow_not_converged=True)   # warm-up (graph capture, tuning)
        s = ctx.solve(allow_not_converged=True)
        dom.append({"N": N, "M": 4 * N * N, "ms": s["gpu_ms"], "sweeps": s["iterations_max"],
                    "rel_l2": rel(ctx.scalar_flux(-1)),
                    "tensor_cores": bool(p.kernel == "hg" and args.dense_precision == 1
                                         and 4 * N * N <= 128)})
    target = args.target

    def first(points, tgt=target):
        hit = [q for q in points if q["rel_l2"] <= tgt]
        return hit[0] if hit else None

    ctx.set_options(tol=TOL, tile_g=-1, dense_precision=args.dense_precision)
    rom = []
    for m in args.rom_m:
        nz, nt = W.partition(m)
        batch = args.rom_batch
        runs = []
        for rep in range(args.rom_seeds):
            seed = W.ordinate_seed(1, 7 + rep)
            ctx.set_ordinates_seed(seed, [nz] * batch, [nt] * batch, first_sample=0)
            ctx.solve(allow_not_converged=True)  # warm-up
            tot_ms, acc, n, curve = 0.0, np.zeros((p.J, p.I)), 0, []
            while n < args.rom_max and tot_ms < args.rom_max_ms:
                ctx.set_ordinates_seed(seed, [nz] * batch, [nt] * batch, first_sample=n)
                s = ctx.solve(allow_not_converged=True)
                tot_ms += s["gpu_ms"]
                part, cnt = ctx.partial_sum()
                acc += part
                n += cnt
                curve.append({"samples": n, "ms": tot_ms, "rel_l2": rel(acc / n)})
                if curve[-1]["rel_l2"] <= target and n >= args.rom_min:
                    break
            runs.append({"seed": seed, "curve": curve, "at_target": first(curve)})
        # bias floor: err(t)^2 = B^2 + V / t, least squares over every point of every run
        ts = np.array([c["samples"] for r in runs for c in r["curve"]], dtype=np.float64)
        e2 = np.array([c["rel_l2"] ** 2 for r in runs for c in r["curve"]])
        A = np.stack([np.ones_like(ts), 1.0 / ts], 1)
        (b2, v), *_ = np.linalg.lstsq(A, e2, rcond=None)
        hits = [r["at_target"] for r in runs if r["at_target"]]
        med = None
        if len(hits) * 2 > len(runs):  # a median exists among the runs that reached it
            ms_all = sorted([h["ms"] for h in hits] + [float("inf")] * (len(runs) - len(hits)))
            sm_all = sorted([h["samples"] for h in hits] + [10 ** 9] * (len(runs) - len(hits)))
            med = {"ms": ms_all[len(runs) // 2], "samples": sm_all[len(runs) // 2]}
        rom.append({"M": 4 * m, "runs_reaching_target": len(hits), "runs": len(runs),
                    "median_at_target": med,
                    "bias_floor_rel_l2": float(np.sqrt(max(b2, 0.0))),
                    "mc_spread_rel_l2": float(np.sqrt(max(v, 0.0))),
                    "final": [r["curve"][-1] for r in runs]})
    ctx.close()

    dom_hit = first(dom)
    rom_reached = [r for r in rom if r["median_at_target"]]
    rom_best = min(rom_reached, key=lambda r: r["median_at_target"]["ms"]) if rom_reached else None
    line = {
        "metric": f"GPU time to relative l2 flux error {target:g}, ROM vs DOM ({p.name}, "
                  f"{p.I}x{p.J}, kernel {p.kernel}{' g=%g' % p.g if p.kernel != 'iso' else ''}"
                  f"{', rows normalised' if norm else ''})",
        "unit": "ms", "higher_is_better": False, "data": "synthetic",
        "reference": f"FP64 oracle, 2D {args.ref_kind} set N={args.ref_n} ({ref_m} ordinates), "
                     f"SI to 1e-12 ({ref_s:.0f} s on the host)",
        "reference_check": chk,
        "dom_ms_to_target": dom_hit["ms"] if dom_hit else None,
        "dom_M_at_target": dom_hit["M"] if dom_hit else None,
        "dom_best_rel_l2": min(d["rel_l2"] for d in dom) if dom else None,
        "rom_median_ms_to_target": rom_best["median_at_target"]["ms"] if rom_best else None,
        "rom_M_at_target": rom_best["M"] if rom_best else None,
        "rom_median_samples_at_target": rom_best["median_at_target"]["samples"] if rom_best else None,
        "dom": dom,
        "rom": rom,
        "settings": {"rom_batch": args.rom_batch, "rom_max": args.rom_max,
                     "rom_max_ms": args.rom_max_ms,
                     "rom_seeds": args.rom_seeds, "tol": TOL,
                     "dense_precision": args.dense_precision if p.kernel == "hg" else None},
    }
    out = json.dumps(line)
    print(out)
    if args.out:
        with open(args.out, "w") as f:
            f.write(json.dumps(line, indent=1) + "\n")
    return 0


# ------------------------------------------------- Example 2.1 experiment tables

# Values the paper prints for Example 2.1 (Sec. 4.2): error E and bias B of ROM with
# t = 10240 samples, Delta S = pi/64, pi/36, pi/16, pi/4, and the ray-effect measure
# e_inf of DOM with 36 and 144 ordinates and of ROM with 16 samples of 36 ordinates.
PAPER_E8 = {
    "E": {"0.0": [8.09e-3, 1.25e-2, 2.26e-2, 6.28e-2], "0.9": [8.18e-3, 1.26e-2, 2.28e-2, 6.36e-2]},
    "B": {"0.0": [1.12e-4, 2.62e-4, 6.44e-4, 6.22e-3], "0.9": [1.09e-4, 2.01e-4, 3.95e-4, 5.42e-3]},
    "order_E": {"0.0": 0.74, "0.9": 0.74}, "order_B": {"0.0": 1.44, "0.9": 1.41},
}
PAPER_E10 = {"dom_36": 0.0373, "dom_144": 0.0206, "rom_16x36": 0.012}


def run_paper_tables(args):
    """Example 2.1 at the paper's scale on the GPU: ROM error E (mean over samples of
    the l2 error of one sample) and bias B (l2 error of the sample average), eq.
    (l2norm2D), for t samples at Delta S = pi/(4 N^2), N = 4, 3, 2, 1, kernels g = 0
    and g = 0.9; e_inf for DOM (uniform N = 3, 6) and ROM (16 samples of N = 3).
    Reference: the FP64 oracle with the Gaussian set N = args.ref_n (2 N (N + 1)
    ordinates; the linear kernel through its three moments), SI to 1e-10."""
    from oracle import oracle as O
    import __graft_entry__
    __graft_entry__.build()
    from paper_2407_12527_gb300 import RomContext

    t = args.table_samples
    batch = args.table_batch
    out = {"metric": f"ROM error and bias on Example 2.1 (100x100, t = {t} samples) and the "
                     f"ray-effect measure, 1 GB300", "data": "synthetic",
           "reference": f"FP64 oracle, 2D Gaussian set N={args.ref_n}, SI to 1e-10",
           "paper": {"table_t10240": PAPER_E8, "e_inf": PAPER_E10}, "ours": {}}
    for g in (0.0, 0.9):
        p = W.example_2_1(g=g)
        ref_set = O.quad_gauss_xy(args.ref_n)
        t0 = time.perf_counter()
        if g == 0.0:
            ref = O.solve_xy(p.I, p.J, p.bounds, p.sigma_t, p.sigma_s, p.q, [ref_set],
                             tol=1e-10)["phi"][0]
        else:
            ref = O.solve_xy_linear_moments(p.I, p.J, p.bounds, p.sigma_t, p.sigma_s, p.q,
                                            [ref_set], g, tol=1e-10)["phi"][0]
        ref_s = time.perf_counter() - t0
        ctx = RomContext(0)
        ctx.set_grid(p.I, p.J, p.bounds, p.sigma_t, p.sigma_s, p.q)
        if g:
            ctx.set_kernel("linear", g)
        ctx.set_options(tol=TOL)
        rows = []
        for N in (4, 3, 2, 1):
            errs, acc, n, gpu_ms = [], np.zeros((p.J, p.I)), 0, 0.0
            while n < t:
                b = min(batch, t - n)
                ctx.set_ordinates_seed(W.ordinate_seed(10, int(10 * g)), [N] * b, [N] * b,
                                       first_sample=n)
                st = ctx.solve()
                gpu_ms += st["gpu_ms"]
                errs.extend(O.l2_xy(ctx.scalar_flux(k), ref) for k in range(b))
                part, cnt = ctx.partial_sum()
                acc += part
                n += cnt
            rows.append({"delta_S": f"pi/{4 * N * N}", "M": 4 * N * N,
                         "E": float(np.mean(errs)), "B": O.l2_xy(acc / n, ref),
                         "gpu_ms": gpu_ms})
        dS = np.log([np.pi / r["M"] for r in rows])  # Delta S = pi / (4 N^2) = pi / M
        order_E = float(np.polyfit(dS, np.log([r["E"] for r in rows]), 1)[0])
        order_B = float(np.polyfit(dS, np.log([r["B"] for r in rows]), 1)[0])
        res = {"rows": rows, "order_E": order_E, "order_B": order_B,
               "reference_host_s": ref_s}
        if g == 0.0:  # ray-effect measure (the paper does not say which kernel: g = 0 assumed)
            e = {}
            for name, n_uni in (("dom_36", 3), ("dom_144", 6)):
                ctx.set_quadrature("uniform", n_uni)
                ctx.solve()
                e[name] = O.e_inf(ctx.scalar_flux(-1), ref)
            ctx.set_ordinates_seed(W.ordinate_seed(10, 5), [3] * 16, [3] * 16)
            ctx.solve()
            e["rom_16x36"] = O.e_inf(ctx.scalar_flux(-1), ref)
            res["e_inf"] = e
        ctx.close()
        out["ours"][f"{g}"] = res
    print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--check-every", type=int, default=0,
                    help="0: device-side source-iteration loop (CUDA graph); k > 0: host loop "
                         "checking every k sweeps (profilers cannot look inside the graph loop)")
    ap.add_argument("--rows-per-step", type=int, default=0, choices=[0, 1, 2, 4],
                    help="X-Y sweep rows per wavefront step (0: 4, or measured with --tile-g -1); "
                         "fixing it (with --tile-g) reproduces the autotuned shape in profiler "
                         "captures")
    ap.add_argument("--tile-g", type=int, default=-1,
                    help="ordinates per sweep work item (1, 2, 4; 0: size heuristic; "
                         "-1: measured by the library's autotuner)")
    ap.add_argument("--dense-precision", type=int, default=1, choices=[0, 1],
                    help="dense scattering operator product: 0 FP32 CUDA cores, 1 split BF16 "
                         "on the tcgen05 tensor cores")
    ap.add_argument("--samples", type=int, default=0,
                    help="ROM samples per step (0: the workload's own count); smaller batches "
                         "serve the small-case profiler captures")
    ap.add_argument("--only-timed", action="store_true",
                    help="run the warm-up and timed steps only (no roofline, e2e or CPU legs)")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-total", type=float, default=60.0,
                    help="CPU seconds the reference (oracle) arm spends over all its steps")
    ap.add_argument("--workload", default="point_source",
                    choices=["point_source", "point_source_dom", "dom_small", "checkerboard",
                             "hg_disc", "lognormal_cube"])
    ap.add_argument("--rom-vs-dom", action="store_true",
                    help="measure GPU time to a relative l2 error target, ROM vs plain DOM")
    ap.add_argument("--target", type=float, default=1e-3)
    ap.add_argument("--ref-n", type=int, default=200)
    ap.add_argument("--ref-check-n", type=int, default=150,
                    help="second reference set whose distance to the first is reported (0: none)")
    ap.add_argument("--rom-seeds", type=int, default=5)
    ap.add_argument("--rom-min", type=int, default=0,
                    help="samples a ROM run always accumulates before stopping at the target")
    ap.add_argument("--rvd-n", type=int, default=128,
                    help="cells per side of the reduced Henyey-Greenstein disc problem")
    ap.add_argument("--out", default="", help="also write the JSON line (indented) to this file")
    ap.add_argument("--ref-kind", default="gauss", choices=["gauss", "uniform"])
    ap.add_argument("--rvd-problem", default="point_source",
                    choices=["point_source", "example_2_1", "hg_disc"])
    ap.add_argument("--dom-n", type=int, nargs="+", default=[2, 3, 4, 6, 8, 12, 16, 24, 32])
    ap.add_argument("--rom-m", type=int, nargs="+", default=[4, 9, 16],
                    help="ordinate cells per quadrant (M = 4 m)")
    ap.add_argument("--rom-batch", type=int, default=256)
    ap.add_argument("--rom-max-ms", type=float, default=30000.0,
                    help="GPU time after which one ROM run stops accumulating samples")
    ap.add_argument("--rom-max", type=int, default=4096)
    ap.add_argument("--paper-tables", action="store_true",
                    help="Example 2.1 ROM error / bias table and ray-effect measure (Sec. 4.2)")
    ap.add_argument("--table-samples", type=int, default=10240)
    ap.add_argument("--table-batch", type=int, default=1024)
    args = ap.parse_args()
    global WL, ARGS
    ARGS = args
    if args.rom_vs_dom:
        return run_rom_vs_dom(args)
    if args.paper_tables:
        return run_paper_tables(args)
    WL = make_workload(args.workload)
    if args.samples > 0 and not WL.quad:
        k = args.samples
        WL.nz = [WL.nz[i % len(WL.nz)] for i in range(k)]
        WL.nt = [WL.nt[i % len(WL.nt)] for i in range(k)]
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
