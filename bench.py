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
N_SAMPLES, NZ, NT, TOL = 64, 2, 2, 1e-6
SEED = W.ordinate_seed(1)


def workload_config(extra=None):
    p = W.point_source()
    cfg = {
        "workload": "point_source_256 (256x256 on [-1,1]^2, sigma_T=1, sigma_S=0.9 isotropic, "
                    "Gaussian q std 0.02, vacuum): ROM 64 samples x 16 ordinates, SI to 1e-6",
        "grid": [p.I, p.J], "samples_per_step": N_SAMPLES, "ordinates_per_sample": 4 * NZ * NT,
        "si_tol": TOL, "scheme": "diamond difference", "kernel": "isotropic",
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

def oracle_rate(budget_s: float, max_samples: int, first: int = 0):
    """The FP64 oracle, as it stands, on consecutive samples of the workload until
    the time budget is used: returns (updates/s, samples, threads, updates)."""
    from oracle import oracle as O
    p = W.point_source()
    threads = O.max_threads()
    upd = 0
    n = 0
    t0 = time.perf_counter()
    while n < max_samples:
        o = O.rom_ordinates_xy(SEED, first + n, NZ, NT)
        r = O.solve_xy(p.I, p.J, p.bounds, p.sigma_t, p.sigma_s, p.q, [o], tol=TOL)
        upd += p.I * p.J * o.M * int(r["iters"][0])
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return upd / dt, n, min(threads, 4 * NZ * NT), upd, dt


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
        rate, ns, threads, upd, dt = oracle_rate(per_step, 64, first=N_SAMPLES * (k + 1))
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
                         "sample": f"{ns_tot} ROM samples of the workload over {args.steps} "
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

    p = W.point_source()
    nz = [NZ] * N_SAMPLES
    nt = [NT] * N_SAMPLES
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    ctx = RomContext(local)
    ctx.set_stream(stream.cuda_stream)
    st_d, ss_d, q_d = (torch.tensor(a, dtype=torch.float32, device=dev).contiguous()
                       for a in (p.sigma_t, p.sigma_s, p.q))
    torch.cuda.synchronize(dev)
    ctx.set_grid_device(p.I, p.J, p.bounds, st_d, ss_d, q_d)
    ctx.set_options(tol=TOL, check_every=args.check_every, tile_g=args.tile_g)

    def first_sample(step):
        return (step * world + rank) * N_SAMPLES

    def one_step(step):
        ctx.set_ordinates_seed(SEED, nz, nt, first_sample=first_sample(step))
        return ctx.solve()

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
        launches += 1 + s["kernel_launches"]  # ordinate generation + the solve's kernels
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
                              "ms_per_step": 1e3 * t_max / args.steps, "only_timed": True}))
        ctx.close()
        return 0

    # roofline: the same steps with CUDA events around every sweep launch
    ctx.set_options(tol=TOL, time_kernels=1, check_every=8, tile_g=args.tile_g)
    sweep_ms, sweep_upd, sweep_n = 0.0, 0, 0
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        s = one_step(k)
        sweep_ms += s["sweep_ms"]
        sweep_upd += s["updates"]
        sweep_n += s["sweep_launches"]
    ctx.set_options(tol=TOL, tile_g=args.tile_g)
    peak_tflops = 152 * 128 * 2 * 2070e6 / 1e12
    achieved = sweep_upd * FLOP_PER_UPDATE / (sweep_ms / 1e3) / 1e12
    # DRAM bytes of one full sweep launch from the committed ncu capture, used
    # only while the sweep source is the one that was captured
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "sweep2d_point_source_256x64.traffic.json")
    spath = os.path.join(ROOT, "paper_2407_12527_gb300", "csrc", "sweep2d.cu")
    if os.path.exists(tpath) and args.tile_g in (0, 2):
        import hashlib
        with open(tpath) as f:
            tr = json.load(f)
        with open(spath, "rb") as f:
            digest = hashlib.sha256(f.read()).hexdigest()
        if tr.get("sweep2d_cu_sha256") == digest:
            traffic = tr.get("dram_bytes_per_launch")
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops, "traffic": traffic,
                "traffic_note": "DRAM read+write bytes of one full sweep launch (ncu)",
                "kernel": "sweep2d_kernel (K1)",
                "launches": sweep_n, "avg_launch_us": 1e3 * sweep_ms / max(sweep_n, 1),
                "flop_per_update": FLOP_PER_UPDATE,
                "peak_source": "FP32 CUDA cores: 152 SM x 128 lanes x 2 flop x 2070 MHz"}

    # end to end through the C ABI with host buffers
    ctx2 = RomContext(local)
    ctx2.set_options(tol=TOL, tile_g=args.tile_g)
    st_h, ss_h, q_h = (np.ascontiguousarray(a, dtype=np.float64) for a in
                       (p.sigma_t, p.sigma_s, p.q))
    e2e_upd, e2e_t = 0, 0.0
    for k in range(args.warmup + args.steps):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        ctx2.set_grid(p.I, p.J, p.bounds, st_h, ss_h, q_h)
        ctx2.set_ordinates_seed(SEED, nz, nt, first_sample=first_sample(k))
        s = ctx2.solve()
        phi_bar = ctx2.scalar_flux(-1)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            e2e_upd += s["updates"]
            e2e_t += dt
    assert np.isfinite(phi_bar).all()
    e2e_t = barrier_max(e2e_t, world, dev)
    e2e_upd = barrier_sum(float(e2e_upd), world, dev)
    e2e = {"value": e2e_upd / e2e_t, "unit": UNIT,
           "h2d_bytes_per_step": 3 * p.I * p.J * 8, "d2h_bytes_per_step": p.I * p.J * 8}
    ctx2.close()
    ctx.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, ns, threads, _, dt = oracle_rate(args.cpu_budget, N_SAMPLES)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"first {ns} of the 64 ROM samples of one step, solved one after "
                         f"another to 1e-6 ({dt:.1f} s)"}

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
    ap.add_argument("--tile-g", type=int, default=0,
                    help="ordinates per sweep work item (0: library default)")
    ap.add_argument("--only-timed", action="store_true",
                    help="run the warm-up and timed steps only (no roofline, e2e or CPU legs)")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-total", type=float, default=60.0,
                    help="CPU seconds the reference (oracle) arm spends over all its steps")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
