#!/usr/bin/env python
"""Benchmark of the CHFPE hot path on B300: one step = one 2D response R2(t2, t1) (Eq. 2Dresponse)
of the two-mode workload (2 coupled anharmonic modes, 32^4 grid, depth 4 = 15 members, LL + SL
coupling, dt = 0.005, 64 x 64 samples at dtau = 0.2, all 64 t1 branches advanced in one batched
launch per RK4 stage), FP32 state and arithmetic, FP64 reductions.

Prints one JSON line (rank 0).  Metric: CHFPE cell-updates/s (one cell-update = one RK4 step of
one (grid point, hierarchy member)), plus 2D spectra/s.  `--impl reference` times the FP64 CPU
oracle on a bounded sample of the same workload instead.

Timing: W warm-up steps, then K steps bracketed by a barrier and torch.cuda.synchronize(), CUDA
events on the library's stream; inputs (3 x 64 branch states, 12 GB) are far larger than L2.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2509_25840_b300 import inputs  # noqa: E402

ELEM_ACCESSES_PER_CELL_STEP = 11      # Horner-form RK4: 2 + 3 + 3 + 3 element accesses
# launch shapes of the RK4 stage kernel the library's autotuner chooses from (variant index ->
# points per thread, threads per block, minimum resident blocks per SM), as in chfpe.cu
STAGE_SHAPES = {0: (2, 128, 8), 1: (2, 256, 4), 2: (2, 128, 6), 3: (4, 128, 4), 4: (4, 128, 4), 5: (4, 128, 4),
                6: (4, 256, 2), 7: (4, 64, 8), 8: (4, 128, 4),
                9: (4, 128, 4), 10: (4, 128, 3), 11: (4, 128, 2)}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1,
                    help="timed R2 spectra (one is ~52 s on a B300)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--nt", type=int, default=64, help="t1/t2 samples (64 is the workload)")
    ap.add_argument("--eq-steps", type=int, default=200, help="FP64 equilibration steps")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--workload", default="two_mode_32",
                    choices=["two_mode_32", "one_mode_64", "three_mode_20", "sweep"],
                    help="two_mode_32 is the benchmark; the others are secondary measurements")
    ap.add_argument("--instances", type=int, default=64, help="sweep: instances in the batch")
    ap.add_argument("--error-instances", type=int, default=8,
                    help="sweep: instances re-run in FP64 for the per-instance error report")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


# ------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        self.path = None
        self.dev = device_index

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.dev)],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------------------------------
# distributed plumbing (independent replicas: one spectrum per rank, no data-path collective)
# ------------------------------------------------------------------------------------------

def dist_setup(n: int):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if os.environ.get("CHFPE_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        dist.init_process_group(backend)
        pg = dist
    return rank, world, local, pg


def barrier(pg, device=None):
    if pg is not None:
        if device is not None:
            pg.barrier(device_ids=[device])
        else:
            pg.barrier()


def max_over_ranks(pg, value: float, device=None) -> float:
    if pg is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device if device is not None else "cpu")
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------------------------------
# CPU oracle on a bounded sample
# ------------------------------------------------------------------------------------------

def oracle_sample(wl, nsteps: int = 1):
    """Time `nsteps` FP64 RK4 steps of one full-size state with the oracle; cell-updates/s."""
    import numpy as np
    import oracle
    pb = oracle.Problem(wl.model, wl.grid, wl.depth)
    W = oracle.boltzmann(pb)
    W = oracle.insert(pb, wl.A, W)
    t0 = time.perf_counter()
    oracle.rk4(pb, W, wl.dt, nsteps)
    dt = time.perf_counter() - t0
    cells = pb.M * pb.P
    return cells * nsteps / dt, dt, oracle.threads(), np.isfinite(W).all()


def run_reference(args, rank, world):
    wl = inputs.two_mode_32(nt=args.nt)
    if rank != 0:
        return
    times = []
    per_step = 8                       # RK4 steps of the oracle per bench step (~6 s on 16 cores)
    for i in range(args.warmup + args.steps):
        rate, dt, threads, _ = oracle_sample(wl, per_step)
        if i >= args.warmup:
            times.append(dt)
    T = sum(times)
    cells = wl.cells * per_step * args.steps
    value = cells / T
    sample = (f"{per_step} FP64 RK4 steps of one 32^4 x 15-member state per bench step "
              f"({wl.cells * per_step} cell-updates), oracle = plain C loops")
    line = {
        "impl": "reference", "metric": "CHFPE cell-updates/s", "value": value,
        "unit": "cell-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * T / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "cells": wl.cells, "sample": sample},
        "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": threads,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------

def run_ours(args, rank, world, local, pg):
    import numpy as np
    import torch
    from paper_2509_25840_b300 import chfpe

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    wl = inputs.two_mode_32(nt=args.nt)
    nt1 = nt2 = args.nt
    h = chfpe.Handle(wl.model, wl.grid, depth=wl.depth, dt=wl.dt, precision=32,
                     max_batch=nt1, stream=stream.cuda_stream)
    t0 = time.perf_counter()
    eq_steps, eq_res = h.equilibrate(args.eq_steps, 1e-10, max(1, args.eq_steps))
    eq_s = time.perf_counter() - t0
    R = np.empty((nt1, nt2))
    spectrum_cells = wl.cells * ((nt1 - 1) * wl.stride + nt1 * (nt2 - 1) * wl.stride)

    def step():
        h.response2(wl.A, wl.B, wl.C, nt1, nt2, wl.stride, out=R)

    for _ in range(args.warmup):
        step()
    R_warm = R.copy()

    # device-resident inputs: the equilibrium stays in HBM, R (32 KB) comes back each step
    clocks = Clocks(local)
    torch.cuda.synchronize(dev)
    barrier(pg, local if pg is not None and torch.distributed.get_backend() == "nccl" else None)
    h.stats_reset(time_stages=True)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    st = h.stats()
    T = ev0.elapsed_time(ev1) / 1e3
    T = max_over_ranks(pg, T, dev if pg is not None and torch.distributed.get_backend() == "nccl" else None)
    units = spectrum_cells * args.steps * world
    value = units / T
    repeat_ok = bool(np.array_equal(R, R_warm))

    peak, peak_kind = peaks()
    achieved = st["stage_bytes"] / (st["stage_ms"] / 1e3) / 1e9 if st["stage_ms"] > 0 else None
    # the launch shape the autotuner picked at create: (points per thread, threads, min blocks)
    variant, tune_us = h.stage_tuning()
    V, NT, MINB = STAGE_SHAPES[variant]
    kernel = ("stage_bulk_kernel<4,128>" if variant == 4 else "stage_cpasync_kernel<4,128>" if variant == 5 else
              "stage_vec_kernel<float,2,4,%d,%d,%d,15,%d,%d>" % (V, NT, MINB, int(variant == 8),
                                                               int(variant == 9)))
    # DRAM bytes per launch from the committed ncu capture of this kernel: measured bytes per
    # cell-stage times the cells of one branch-phase launch (nt1 states)
    traffic = None
    prof = os.path.join(ROOT, "profiles", "stage_kernel_traffic.json")
    if os.path.exists(prof):
        try:
            tj = json.load(open(prof))
            per_cell = tj.get("bytes_per_cell_stage_two_mode_32")
            if per_cell and tj.get("kernel") == kernel:
                traffic = per_cell * nt1 * wl.cells
        except Exception:
            traffic = None
    roofline = {
        "kernel": kernel,
        "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
        "frac": (achieved / peak) if achieved else None, "peak_kind": peak_kind,
        "traffic": traffic,
        "algorithmic_bytes_per_cell_stage": ELEM_ACCESSES_PER_CELL_STEP * 4 / 4,
        "traffic_per": "branch-phase launch (%d states), stage 2, from profiles/stage_kernel_traffic.json" % nt1,
        "stage_launches": st["stage_launches"],
        "avg_launch_ms": st["stage_ms"] / max(1, st["stage_launches"]),
    }

    # end to end through the public API from pinned host memory: every step uploads the
    # equilibrium (M*P doubles) and reads R back
    e2e = None
    if not args.no_e2e:
        Weq = torch.empty(h.state_shape, dtype=torch.float64, pin_memory=True).numpy()
        Weq[...] = h.get_equilibrium()
        torch.cuda.synchronize(dev)
        barrier(pg, local if pg is not None and torch.distributed.get_backend() == "nccl" else None)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            h.set_equilibrium(Weq)
            step()
        torch.cuda.synchronize(dev)
        Te = time.perf_counter() - t0
        Te = max_over_ranks(pg, Te, dev if pg is not None and torch.distributed.get_backend() == "nccl" else None)
        e2e = {"value": spectrum_cells * args.steps * world / Te, "unit": "cell-updates/s",
               "h2d_bytes_per_step": int(Weq.nbytes), "d2h_bytes_per_step": int(R.nbytes),
               "spectra_per_s": args.steps * world / Te}

    cpu = None
    if rank == 0 and not args.no_cpu:
        rate, dt, threads, _ = oracle_sample(wl, 16)
        cpu = {"value": rate, "unit": "cell-updates/s", "cores": threads, "kind": "oracle",
               "sample": f"16 FP64 RK4 steps of one 32^4 x 15-member state ({dt:.1f} s)"}

    if rank == 0:
        line = {
            "metric": "CHFPE cell-updates/s", "value": value, "unit": "cell-updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * T / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl.name + ": 2 coupled anharmonic modes, 32^4 grid, depth 4 "
                       "(15 members), LL+SL, dt=0.005, R2 on %dx%d (t1,t2) at dtau=0.2, all t1 "
                       "branches batched" % (nt1, nt2),
                       "cells_per_state": wl.cells, "cell_updates_per_spectrum": spectrum_cells,
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2 (branch arrays 3 x %.1f GB)" % (
                           nt1 * wl.cells * 4 / 1e9),
                       "equilibration": {"steps": eq_steps, "residual": eq_res, "seconds": eq_s},
                       "stage_shape": {"variant": variant, "points_per_thread": V, "threads": NT,
                                       "min_blocks_per_sm": MINB,
                                       "autotune_us_per_launch": [round(u, 1) for u in tune_us]}},
            "spectra_per_s": args.steps * world / T,
            "roofline": roofline,
            "clocks": clk,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "gpu_launches": st["kernel_launches"],
            "repeatable": repeat_ok,
        }
        print(json.dumps(line), flush=True)
    h.close()


# ------------------------------------------------------------------------------------------
# secondary workloads (one GPU): the one-mode R1, the three-mode 20^6 R2 on a reduced t-grid,
# and the batched parameter sweep with bf16 deep tiers
# ------------------------------------------------------------------------------------------

def run_extra(args, local):
    import numpy as np
    import torch
    from paper_2509_25840_b300 import chfpe

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    peak, peak_kind = peaks()
    t_eq = time.perf_counter()
    if args.workload == "one_mode_64":
        wl = inputs.one_mode_64()
        prec, dtype = 64, "f64"
        h = chfpe.Handle(wl.model, wl.grid, depth=wl.depth, dt=wl.dt, precision=prec,
                         stream=stream.cuda_stream)
        eq = h.equilibrate(args.eq_steps, 1e-12, max(1, args.eq_steps))
        units = wl.cells * (wl.nt1 - 1) * wl.stride
        step = lambda: h.response1(wl.A, wl.C, wl.nt1, wl.stride)
        desc = ("one_mode_64: 1 harmonic mode, 64x64 on [-6,6]^2, zeta=0.2, gamma=1, LL, depth 5, "
                "dt=0.005, R1 sampled every step over 2000 steps (CUDA-graph sampling intervals)")
        unit_name = "R1 responses"
    elif args.workload == "three_mode_20":
        nt = args.nt if args.nt != 64 else 8
        wl = inputs.three_mode_20(nt=nt)
        prec, dtype = 32, "f32"
        h = chfpe.Handle(wl.model, wl.grid, depth=wl.depth, dt=wl.dt, precision=prec,
                         max_batch=nt, stream=stream.cuda_stream)
        eq = h.equilibrate(min(args.eq_steps, 20), 1e-10, max(1, min(args.eq_steps, 20)))
        units = wl.cells * wl.r2_state_steps()
        step = lambda: h.response2(wl.A, wl.B, wl.C, nt, nt, wl.stride)
        full = inputs.three_mode_20()
        desc = ("three_mode_20: 3 water-like modes (omega 0.5/1.0/1.6), 20^6 grid, depth 2 (10 members),"
                " dt=0.002, TRT R2 on %dx%d at dtau=0.1 (the 128x128 spectrum needs %d state-steps)"
                % (nt, nt, full.r2_state_steps()))
        unit_name = "R2 spectra (reduced t-grid)"
    else:
        n = args.instances
        wls = [inputs.sweep_instance(s) for s in range(n)]
        prec, dtype = 32, "f32+bf16(tiers 3-4)"
        h = chfpe.Batch([w.model for w in wls], [w.grid for w in wls], depth=4, dt=0.005,
                        precision=32, stream=stream.cuda_stream, bf16_tier=3)
        res = h.equilibrate_all(min(args.eq_steps, 50), 1e-10, max(1, min(args.eq_steps, 50)))
        eq = (min(args.eq_steps, 50), float(np.max(res)))
        nt, stride = 201, 10
        cells = sum(w.cells for w in wls)
        units = cells * (nt - 1) * stride
        mu = wls[0].A
        step = lambda: h.response1_all(mu, mu, nt, stride)
        desc = ("sweep: %d seeded two-mode instances (grids 24..48 per axis, depth 4), batched: one "
                "launch per RK4 stage for all; R1 over 2000 steps (201 samples); tiers 3-4 in bf16"
                % n)
        unit_name = "R1 responses of the batch"
    eq_s = time.perf_counter() - t_eq
    for _ in range(args.warmup):
        step()
    clocks = Clocks(local)
    torch.cuda.synchronize(dev)
    h.stats_reset(time_stages=args.workload != "one_mode_64")
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    st = h.stats()
    T = ev0.elapsed_time(ev1) / 1e3
    achieved = st["stage_bytes"] / (st["stage_ms"] / 1e3) / 1e9 if st["stage_ms"] > 0 else None
    line = {
        "metric": "CHFPE cell-updates/s", "value": units * args.steps / T, "unit": "cell-updates/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
        "data": "synthetic", "config": {"workload": desc, "equilibration": {"steps": eq[0],
                                         "residual": eq[1], "seconds": eq_s}},
        "per_s": {unit_name: args.steps / T},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if achieved else None, "peak_kind": peak_kind,
                     "note": None if achieved else "launch-bound: stage bursts inside CUDA graphs are not timed"},
        "clocks": clk, "gpu_launches": st["kernel_launches"],
    }
    if args.workload == "three_mode_20":
        line["extrapolated_s_per_128x128_spectrum"] = (inputs.three_mode_20().r2_state_steps() *
                                                        wl.cells / (units * args.steps / T))
    if args.workload == "sweep" and args.error_instances > 0:
        # error of the FP32 + bf16-tier propagation against FP64, per instance: the first
        # instances, from the same stored equilibria, R1 over 200 steps (21 samples)
        ne = min(args.error_instances, len(wls))
        sub = wls[:ne]
        Ws = [h.instance(i).get_equilibrium() for i in range(ne)]
        R = {}
        for prec_e, tier in ((32, 3), (64, 0)):
            with chfpe.Batch([w.model for w in sub], [w.grid for w in sub], depth=4, dt=0.005,
                             precision=prec_e, stream=stream.cuda_stream, bf16_tier=tier) as be:
                for i in range(ne):
                    be.instance(i).set_equilibrium(Ws[i])
                R[prec_e] = be.response1_all(mu, mu, 21, 10)
        errs = [float(np.abs(R[32][i] - R[64][i]).max() / np.abs(R[64][i]).max()) for i in range(ne)]
        line["error_vs_fp64"] = {
            "instances": ne, "steps": 200, "metric": "max_t |R1_f32+bf16 - R1_f64| / max_t |R1_f64|",
            "median": float(np.median(errs)), "max": float(np.max(errs)),
            "per_instance": [float("%.3g" % e) for e in errs]}
    print(json.dumps(line), flush=True)
    h.close()


def main():
    args = parse()
    rank, world, local, pg = dist_setup(args.gpus)
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        elif args.workload != "two_mode_32":
            run_extra(args, local)
        else:
            run_ours(args, rank, world, local, pg)
    finally:
        if pg is not None:
            pg.destroy_process_group()


if __name__ == "__main__":
    main()
