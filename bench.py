#!/usr/bin/env python
"""Benchmark of the CHFPE hot path on B300 (Eqs. HEOM and 2Dresponse; the paper's time-evolution
cost centre, Sec. IV C).

Workload (two_mode_32): 2 coupled anharmonic modes, 32^4 grid, depth 4 (15 members), LL + SL
coupling, dt = 0.005; the 2D response R2(t2, t1) on 64 x 64 samples at dtau = 40 dt, all 64 t1
branches advanced together (one batched launch per RK4 stage); FP32 state and arithmetic, FP64
reductions.

One bench step = one sampling interval of that spectrum's branch phase, which is 99.9 % of its
device time: the 64 branch states (spawned along the t1 chain by the library's insertion and RK4
calls) advance 40 RK4 steps and are observed, through chfpe_sample_device.  W warm-up steps, then
K timed steps bracketed by a barrier and torch.cuda.synchronize(), CUDA events on the library's
stream; the branch arrays (3 x 4 GB) are far larger than L2.  Beside the steps the run times one
whole 64 x 64 spectrum (chfpe_response2) once, which gives spectra/s and, measured from the
host-side upload of the FP64 equilibrium to the copy of R2 into host memory, the end-to-end
figure; the error of the FP32 path against the FP64 build on the same grid; the plain form
(branches one at a time) from measured single-branch intervals; and the FP64 CPU oracle on a
bounded sample.

Prints one JSON line (rank 0).  Metric: CHFPE cell-updates/s (one cell-update = one RK4 step of
one (grid point, hierarchy member)).  `--impl reference` times the FP64 CPU oracle on a bounded
sample of the same workload instead.  `--profile-case` runs a small fixed case of the stage
kernel for ncu captures.
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
ELEM_ACCESSES_TEXTBOOK = 16           # the three-array k1..k4 form: 3 + 5 + 5 + 3
# floating-point operations of one cell-stage of the two-mode stage kernel, an FMA counted as 2:
# four 7-point derivatives (7 each), the Liouvillian sum (6), damping (3), on average 8/3 hierarchy
# links of 5 for depth 4, and the RK4 combine (2)
FLOPS_PER_CELL_STAGE_D2 = 52
# launch shapes of the RK4 stage kernel the library's autotuner chooses from (variant index ->
# points per thread, threads per block, minimum resident blocks per SM), as in stage_launch.cuh
STAGE_SHAPES = {0: (2, 128, 8), 1: (2, 256, 4), 2: (2, 128, 6), 3: (4, 128, 4), 4: (4, 128, 4), 5: (4, 128, 4),
                6: (4, 256, 2), 7: (4, 64, 8), 8: (4, 128, 4),
                9: (4, 128, 4), 10: (4, 128, 3), 11: (4, 128, 2), 12: (4, 128, 5), 13: (4, 128, 5),
                14: (2, 128, 8), 15: (4, 256, 2), 16: (4, 128, 4), 17: (4, 128, 4)}
# early-store mode of each shape: 0 none, 1 storage order, 2 the open-accumulator order
STAGE_ES = {12: 2, 13: 1, 14: 1, 15: 1, 16: 1, 17: 2}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20,
                    help="timed sampling intervals (one is ~0.8 s on a B300)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--nt", type=int, default=64, help="t1/t2 samples (64 is the workload)")
    ap.add_argument("--eq-steps", type=int, default=200, help="FP64 equilibration steps")
    ap.add_argument("--err-nt", type=int, default=8,
                    help="R2 samples per axis of the FP32-vs-FP64 error check (0: skip)")
    ap.add_argument("--no-spectrum", action="store_true",
                    help="skip the whole-spectrum run (spectra/s and the end-to-end figure)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--workload", default="two_mode_32",
                    choices=["two_mode_32", "one_mode_64", "three_mode_20", "sweep",
                             "two_mode_hermite", "three_mode_hermite"],
                    help="two_mode_32 is the benchmark; the others are secondary measurements")
    ap.add_argument("--instances", type=int, default=64, help="sweep: instances in the batch")
    ap.add_argument("--error-instances", type=int, default=8,
                    help="sweep: instances re-run in FP64 for the per-instance error report")
    ap.add_argument("--hermite-k", type=int, default=10,
                    help="two_mode_hermite, three_mode_hermite: Hermite functions per mode")
    ap.add_argument("--q-scheme", type=int, default=0, choices=[0, 1, 2],
                    help="two_mode_hermite: q-derivatives, 0 explicit stencil, 1 compact (PCR), 2 its skew part")
    ap.add_argument("--save-r2", default=None,
                    help="secondary workloads: write the last timed response (numpy .npy) here")
    ap.add_argument("--profile-case", action="store_true",
                    help="run `--steps` RK4 steps of `--batch` random states of the workload "
                         "through chfpe_rk4_device (a small, fixed case for ncu)")
    ap.add_argument("--batch", type=int, default=4, help="profile case: states")
    ap.add_argument("--variant", type=int, default=None, help="profile case: forced stage shape")
    ap.add_argument("--precision", type=int, default=32, choices=[32, 64], help="profile case")
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
# the benchmark workload, its step and the units one step processes
# ------------------------------------------------------------------------------------------

def workload_config(wl, nt: int) -> dict:
    return {"workload": "two_mode_32: 2 coupled anharmonic modes (omega 1/1, g4 0.01/0.05, "
                        "g_12^2 = 0.12), 32^4 grid, depth 4 (15 members), LL+SL (V_SL/V_LL 0.3), "
                        "dt=0.005; R2 on %dx%d (t1,t2) at dtau=40 dt, all t1 branches batched; "
                        "one step = one sampling interval (40 RK4 steps + observation) of the "
                        "%d branches" % (nt, nt, nt),
            "cells_per_state": wl.cells, "branches": nt, "rk4_steps_per_step": wl.stride,
            "cell_updates_per_step": wl.cells * nt * wl.stride}


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
    per_step = 8                       # RK4 steps of the oracle per bench step (~3 s on 16 cores)
    for i in range(args.warmup + args.steps):
        rate, dt, threads, _ = oracle_sample(wl, per_step)
        if i >= args.warmup:
            times.append(dt)
    T = sum(times)
    cells = wl.cells * per_step * args.steps
    value = cells / T
    sample = (f"{per_step} FP64 RK4 steps of one 32^4 x 15-member state per bench step "
              f"({wl.cells * per_step} cell-updates), oracle = plain C loops")
    cfg = workload_config(wl, args.nt)
    cfg["sample"] = sample
    line = {
        "impl": "reference", "metric": "CHFPE cell-updates/s", "value": value,
        "unit": "cell-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * T / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
        "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": threads,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------

def spawn_branches(h, wl, nt1, torch, dev):
    """The t1 branches of Eq. 2Dresponse through the library's device-buffer calls: chain =
    A^x W_eq, branch i = B^x chain(t1 = i dtau), the chain advancing `stride` RK4 steps
    between spawns.  Returns the FP32 branch array [nt1][member][grid]."""
    Weq = torch.tensor(h.get_equilibrium(), dtype=torch.float32, device=dev)
    chain = torch.empty_like(Weq)
    branches = torch.empty((nt1,) + tuple(Weq.shape), dtype=torch.float32, device=dev)
    h.insert_device(wl.A, Weq.data_ptr(), chain.data_ptr(), 1)
    for i in range(nt1):
        h.insert_device(wl.B, chain.data_ptr(), branches[i].data_ptr(), 1)
        if i + 1 < nt1:
            h.rk4_device(chain.data_ptr(), 1, wl.stride)
    del Weq, chain
    return branches


def stage_kernel_name(variant: int, M: int = 15) -> str:
    """The chosen shape's kernel as ncu names it (template arguments of the two-mode, depth-4
    instantiation)."""
    V, NT, MINB = STAGE_SHAPES[variant]
    b = lambda x: "true" if x else "false"
    if variant == 4:
        return "stage_bulk_kernel<4, 128>"
    if variant == 5:
        return "stage_cpasync_kernel<4, 128>"
    return "stage_vec_kernel<float, 2, 4, %d, %d, %d, %d, %s, %s, %d>" % (
        V, NT, MINB, M, b(variant == 8), b(variant == 9), STAGE_ES.get(variant, 0))


def run_ours(args, rank, world, local, pg):
    import numpy as np
    import torch
    from paper_2509_25840_b300 import chfpe

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    nccl = pg is not None and torch.distributed.get_backend() == "nccl"
    bdev = local if nccl else None
    stream = torch.cuda.Stream(device=dev)
    wl = inputs.two_mode_32(nt=args.nt)
    nt1 = nt2 = args.nt
    h = chfpe.Handle(wl.model, wl.grid, depth=wl.depth, dt=wl.dt, precision=32,
                     max_batch=nt1, stream=stream.cuda_stream)
    t0 = time.perf_counter()
    eq_steps, eq_res = h.equilibrate(args.eq_steps, 1e-10, max(1, args.eq_steps))
    eq_s = time.perf_counter() - t0
    Weq_host = h.get_equilibrium()

    # ---- the timed steps: sampling intervals of the batched branch phase ----------------------
    with torch.cuda.stream(stream):
        branches = spawn_branches(h, wl, nt1, torch, dev)
        Rd = torch.zeros((nt1, 2), dtype=torch.float64, device=dev)
    torch.cuda.synchronize(dev)
    step_units = wl.cells * nt1 * wl.stride

    def step():
        h.sample_device(wl.C, branches.data_ptr(), nt1, 2, wl.stride, Rd.data_ptr(), 2)

    for _ in range(args.warmup):
        step()
    clocks = Clocks(local)
    torch.cuda.synchronize(dev)
    barrier(pg, bdev)
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
    T = max_over_ranks(pg, T, dev if nccl else None)
    value = step_units * args.steps * world / T
    R_last = Rd.cpu().numpy()
    finite = bool(np.isfinite(R_last).all())

    peak, peak_kind = peaks()
    stage_s = st["stage_ms"] / 1e3
    achieved = st["stage_bytes"] / stage_s / 1e9 if stage_s > 0 else None
    achieved_64 = (st["cell_updates"] * 4 * ELEM_ACCESSES_TEXTBOOK / stage_s / 1e9
                   if stage_s > 0 else None)
    variant, tune_us = h.stage_tuning()
    V, NT, MINB = STAGE_SHAPES[variant]
    kernel = stage_kernel_name(variant)
    # DRAM bytes per launch from the committed ncu capture of this kernel: measured bytes per
    # cell-stage times the cells of one launch (nt1 branch states)
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
    launches = max(1, st["stage_launches"])
    roofline = {
        "kernel": kernel, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
        "frac": (achieved / peak) if achieved else None, "peak_kind": peak_kind,
        "traffic": traffic,
        "algorithmic_bytes_per_cell_update": ELEM_ACCESSES_PER_CELL_STEP * 4,
        "algorithmic_bytes_per_launch": st["stage_bytes"] / launches,
        "avg_launch_ms": st["stage_ms"] / launches,
        "stage_launches": st["stage_launches"],
        "achieved_at_64B_per_cell_update": achieved_64,
        "frac_at_64B_per_cell_update": (achieved_64 / peak) if achieved_64 else None,
        "accounting": "achieved = Horner-form RK4 bytes (11 element accesses per cell-update, "
                      "44 B FP32) over the stage launches' CUDA-event time; the _64B fields use "
                      "the three-array k1..k4 form's 16 accesses (64 B) for the same run",
        "traffic_per": "one stage launch (%d branch states), from the committed ncu capture "
                       "of this kernel (bytes per cell-stage x cells)" % nt1,
    }

    # ---- plain form: one branch at a time (single-branch intervals, extrapolated) -------------
    plain = None
    if rank == 0:
        R1d = torch.zeros(2, dtype=torch.float64, device=dev)
        one = branches[0]
        h.sample_device(wl.C, one.data_ptr(), 1, 2, wl.stride, R1d.data_ptr(), 2)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(4):
            h.sample_device(wl.C, one.data_ptr(), 1, 2, wl.stride, R1d.data_ptr(), 2)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        t_int = e0.elapsed_time(e1) / 1e3 / 4
        intervals = (nt1 - 1) + nt1 * (nt2 - 1)        # the chain plus every branch, one by one
        plain = {"spectra_per_s": 1.0 / (intervals * t_int),
                 "s_per_interval_one_branch": t_int,
                 "cell_updates_per_s": wl.cells * wl.stride / t_int,
                 "how": "extrapolated: (nt1-1) + nt1 (nt2-1) single-branch intervals at the "
                        "measured time of one (4 timed after 1 warm-up)"}
        del R1d
    del branches, Rd
    torch.cuda.synchronize(dev)

    # ---- one whole spectrum: spectra/s (device) and end to end from host memory ----------------
    spectrum = e2e = None
    spectrum_units = wl.cells * wl.r2_state_steps()
    if not args.no_spectrum:
        Wpin = torch.empty(h.state_shape, dtype=torch.float64, pin_memory=True).numpy()
        Wpin[...] = Weq_host
        Rpin = torch.empty((nt1, nt2), dtype=torch.float64, pin_memory=True).numpy()
        torch.cuda.synchronize(dev)
        barrier(pg, bdev)
        h.stats_reset(time_stages=False)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        w0 = time.perf_counter()
        h.set_equilibrium(Wpin)                   # host -> device: M P doubles
        e0.record(stream)
        h.response2(wl.A, wl.B, wl.C, nt1, nt2, wl.stride, out=Rpin)   # R2 device -> host
        e1.record(stream)
        torch.cuda.synchronize(dev)
        w1 = time.perf_counter()
        sst = h.stats()
        Ts = max_over_ranks(pg, e0.elapsed_time(e1) / 1e3, dev if nccl else None)
        Te = max_over_ranks(pg, w1 - w0, dev if nccl else None)
        spectrum = {"spectra_per_s": world / Ts, "s_per_spectrum": Ts,
                    "cell_updates_per_s": spectrum_units * world / Ts,
                    "cell_updates_per_spectrum": spectrum_units,
                    "kernel_launches": sst["kernel_launches"],
                    "finite": bool(np.isfinite(Rpin).all()),
                    "r2_max_abs": float(np.abs(Rpin).max())}
        e2e = {"value": spectrum_units * world / Te, "unit": "cell-updates/s",
               "h2d_bytes_per_step": int(Wpin.nbytes), "d2h_bytes_per_step": int(Rpin.nbytes),
               "steps": 1, "spectra_per_s": world / Te,
               "how": "one whole 64x64 spectrum through chfpe_set_equilibrium (FP64 equilibrium "
                      "from pinned host memory) + chfpe_response2 (R2 into pinned host memory), "
                      "host wall clock around both"}

    # ---- error of the FP32 path against the FP64 build on the same grid and equilibrium -------
    err = None
    if args.err_nt > 0 and rank == 0:
        n = args.err_nt
        R = {}
        for prec in (32, 64):
            with chfpe.Handle(wl.model, wl.grid, depth=wl.depth, dt=wl.dt, precision=prec,
                              max_batch=n, stream=stream.cuda_stream) as he:
                he.set_equilibrium(Weq_host)
                R[prec] = he.response2(wl.A, wl.B, wl.C, n, n, wl.stride)
        R64_grid = R[64]
        e = float(np.abs(R[32] - R[64]).max() / np.abs(R[64]).max())
        err = {"metric": "max |R2_f32 - R2_f64| / max |R2_f64|", "value": e,
               "tolerance": 1e-4, "samples": "%dx%d at dtau=40 dt (t1, t2 <= %.2f)" % (
                   n, n, (n - 1) * wl.stride * wl.dt),
               "fp64_pinned_by": "tests/test_gpu_parity.py: the FP64 build on this workload's "
                                 "model and grid against the FP64 CPU oracle"}

    # ---- the same spectrum in the paper's own representation: momenta in Hermite functions
    #      (Sec. III A, Appendix A) on the same q grid, FP32, one whole 64 x 64 R2 -------------------
    paper_rep = None
    if rank == 0 and not args.no_spectrum:
        K = 6                     # converged: see the K = 10 check below
        hgrid_of = lambda k: inputs.Grid(nq=wl.grid.nq, np=(k, k), qmin=wl.grid.qmin,
                                         qmax=wl.grid.qmax, pmin=(0.0, 0.0), pmax=(1.0, 1.0))
        hgrid = hgrid_of(K)
        with chfpe.Handle(wl.model, hgrid, depth=wl.depth, dt=wl.dt, precision=32, max_batch=nt1,
                          stream=stream.cuda_stream, p_basis=1) as hh:
            hh.equilibrate(args.eq_steps, 1e-10, max(1, args.eq_steps))
            Ceq = hh.get_equilibrium()
            hh.response2(wl.A, wl.B, wl.C, 2, 2, wl.stride)            # warm-up
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            Rh = hh.response2(wl.A, wl.B, wl.C, nt1, nt2, wl.stride)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            th = e0.elapsed_time(e1) / 1e3
            hcells = hh.members * hh.points
        paper_rep = {"representation": "momenta in %d x %d Hermite functions, the same 32 x 32 q grid, "
                                       "explicit q stencil (Sec. III A, Appendix A)" % (K, K),
                     "cells_per_state": hcells, "s_per_spectrum": th, "spectra_per_s": 1.0 / th,
                     "finite": bool(np.isfinite(Rh).all())}
        if args.err_nt > 0:
            n = args.err_nt
            with chfpe.Handle(wl.model, hgrid, depth=wl.depth, dt=wl.dt, precision=64, max_batch=n,
                              stream=stream.cuda_stream, p_basis=1) as hh:
                hh.set_equilibrium(Ceq)
                Rh64 = hh.response2(wl.A, wl.B, wl.C, n, n, wl.stride)
            with chfpe.Handle(wl.model, hgrid_of(10), depth=wl.depth, dt=wl.dt, precision=64,
                              max_batch=n, stream=stream.cuda_stream, p_basis=1) as hh:
                hh.equilibrate(args.eq_steps, 1e-10, max(1, args.eq_steps))
                Rh64_10 = hh.response2(wl.A, wl.B, wl.C, n, n, wl.stride)
            paper_rep["difference_vs_grid_f64"] = float(np.abs(Rh64 - R64_grid).max() /
                                                        np.abs(R64_grid).max())
            paper_rep["difference_K6_vs_K10_f64"] = float(np.abs(Rh64 - Rh64_10).max() /
                                                          np.abs(Rh64_10).max())
            paper_rep["difference_how"] = ("max |R2_a - R2_b| / max |R2_b| on %dx%d samples (FP64): "
                                           "Hermite vs the 32^4 grid (the grid's momentum "
                                           "discretisation error), 6 vs 10 Hermite functions "
                                           "(the truncation's)" % (n, n))

    # ---- the FP64 path against the measured FP64 ALU peak (and the FP32 stage kernel's FLOP rate
    #      against the FP32 peak, for its arithmetic intensity) -----------------------------------
    alu = None
    if rank == 0:
        p64 = chfpe.alu_peak(64, stream.cuda_stream)
        p32 = chfpe.alu_peak(32, stream.cuda_stream)
        with chfpe.Handle(wl.model, wl.grid, depth=wl.depth, dt=wl.dt, precision=64,
                          stream=stream.cuda_stream) as h64:
            with torch.cuda.stream(stream):
                x64 = torch.tensor(Weq_host, dtype=torch.float64, device=dev).unsqueeze(0)
            torch.cuda.synchronize(dev)
            h64.rk4_device(x64.data_ptr(), 1, 2)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h64.rk4_device(x64.data_ptr(), 1, 10)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            t64 = e0.elapsed_time(e1) / 1e3
            del x64
        fp64_rate = wl.cells * 10 / t64
        fp64_flops = fp64_rate * 4 * FLOPS_PER_CELL_STAGE_D2
        fp32_flops = value / world * 4 * FLOPS_PER_CELL_STAGE_D2
        alu = {"fp64_peak_tflops": p64 / 1e12, "fp32_peak_tflops": p32 / 1e12,
               "flops_per_cell_stage": FLOPS_PER_CELL_STAGE_D2,
               "fp64_stage": {"cell_updates_per_s": fp64_rate, "tflops": fp64_flops / 1e12,
                              "frac_of_fp64_peak": fp64_flops / p64,
                              "how": "10 FP64 RK4 steps of one 32^4 x 15 state (chfpe_rk4_device, "
                                     "CUDA events)"},
               "fp32_stage_tflops": fp32_flops / 1e12, "fp32_stage_frac_of_fp32_peak": fp32_flops / p32,
               "peak_how": "chfpe_alu_peak: eight independent FMA chains per thread, every SM"}

    cpu = None
    if rank == 0 and not args.no_cpu:
        rate, dt, threads, _ = oracle_sample(wl, 16)
        cpu = {"value": rate, "unit": "cell-updates/s", "cores": threads, "kind": "oracle",
               "sample": f"16 FP64 RK4 steps of one 32^4 x 15-member state ({dt:.1f} s)"}

    if rank == 0:
        cfg = workload_config(wl, nt1)
        cfg.update({
            "parallelism": "replicas" if world > 1 else "single",
            "l2": "inputs larger than L2 (branch arrays 3 x %.1f GB)" % (nt1 * wl.cells * 4 / 1e9),
            "equilibration": {"steps": eq_steps, "residual": eq_res, "seconds": eq_s},
            "stage_shape": {"variant": variant, "points_per_thread": V, "threads": NT,
                            "min_blocks_per_sm": MINB,
                            "autotune_us_per_launch": [round(u, 1) for u in tune_us]}})
        line = {
            "metric": "CHFPE cell-updates/s", "value": value, "unit": "cell-updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * T / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
            "roofline": roofline,
            "clocks": clk,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "gpu_launches": st["kernel_launches"],
            "spectrum": spectrum,
            "plain_form": plain,
            "error_vs_fp64": err,
            "alu": alu,
            "paper_representation": paper_rep,
            "finite": finite,
        }
        print(json.dumps(line), flush=True)
    h.close()


def run_profile_case(args):
    """A small, fixed case of the RK4 stage kernel for ncu: `--batch` seeded states of the
    workload advanced `--steps` RK4 steps through chfpe_rk4_device (4 stage launches a step);
    --variant fixes the launch shape so that no tuning launches precede the profiled ones."""
    import torch
    from paper_2509_25840_b300 import chfpe
    if args.variant is not None:
        os.environ["CHFPE_STAGE_VARIANT"] = str(args.variant)
    if args.workload in ("two_mode_hermite", "three_mode_hermite"):
        wl = inputs.two_mode_32() if args.workload == "two_mode_hermite" else inputs.three_mode_20()
        K, d = args.hermite_k, wl.grid.d
        grid = inputs.Grid(nq=wl.grid.nq, np=(K,) * d, qmin=wl.grid.qmin, qmax=wl.grid.qmax,
                           pmin=(0.0,) * d, pmax=(1.0,) * d)
        h = chfpe.Handle(wl.model, grid, depth=wl.depth, dt=wl.dt, precision=args.precision,
                         max_batch=args.batch, p_basis=1, q_scheme=args.q_scheme)
    else:
        wl = {"two_mode_32": inputs.two_mode_32, "one_mode_64": inputs.one_mode_64,
              "three_mode_20": inputs.three_mode_20}[args.workload]()
        h = chfpe.Handle(wl.model, wl.grid, depth=wl.depth, dt=wl.dt, precision=args.precision,
                         max_batch=args.batch)
    dtype = torch.float32 if args.precision == 32 else torch.float64
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.rand((args.batch,) + h.state_shape, dtype=dtype, device="cuda", generator=g) * 1e-3
    h.rk4_device(x.data_ptr(), args.batch, args.steps)
    torch.cuda.synchronize()
    print(f"ok {args.workload} batch={args.batch} steps={args.steps} "
          f"variant={h.stage_tuning()[0]} max={float(x.abs().max()):.6g}")
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
    elif args.workload == "two_mode_hermite":
        base = inputs.two_mode_32(nt=args.nt)
        K = args.hermite_k
        hgrid = inputs.Grid(nq=base.grid.nq, np=(K, K), qmin=base.grid.qmin, qmax=base.grid.qmax,
                            pmin=(0.0, 0.0), pmax=(1.0, 1.0))
        prec, dtype = 32, "f32"
        nt = args.nt
        h = chfpe.Handle(base.model, hgrid, depth=base.depth, dt=base.dt, precision=prec,
                         max_batch=nt, stream=stream.cuda_stream, p_basis=1, q_scheme=args.q_scheme)
        eq = h.equilibrate(args.eq_steps, 1e-10, max(1, args.eq_steps))
        hcells = h.members * h.points
        units = hcells * base.r2_state_steps()
        step = lambda: h.response2(base.A, base.B, base.C, nt, nt, base.stride)
        desc = ("two_mode_hermite: the two_mode_32 model and q grid (32 x 32) with the momenta in %d x %d "
                "Hermite functions (Sec. III A, Appendix A), %s q-derivatives, depth 4, dt=0.005; R2 on "
                "%dx%d at dtau=0.2, all t1 branches batched; %d cells per state against %d on the "
                "32^4 grid" % (K, K, {0: "explicit 6th-order", 1: "compact (Sec. III B, PCR)",
                               2: "skew-symmetric compact (Sec. III B, two PCR solves)"}[args.q_scheme],
                              nt, nt, hcells, base.cells))
        unit_name = "R2 spectra"
    elif args.workload == "three_mode_hermite":
        nt = args.nt if args.nt != 64 else 128
        base = inputs.three_mode_20(nt=nt)
        K = args.hermite_k

        def hgrid_of(k):
            return inputs.Grid(nq=base.grid.nq, np=(k,) * 3, qmin=base.grid.qmin, qmax=base.grid.qmax,
                               pmin=(0.0,) * 3, pmax=(1.0,) * 3)
        hgrid = hgrid_of(K)
        prec, dtype = 32, "f32"
        h = chfpe.Handle(base.model, hgrid, depth=base.depth, dt=base.dt, precision=prec,
                         max_batch=nt, stream=stream.cuda_stream, p_basis=1)
        eq = h.equilibrate(args.eq_steps, 1e-10, max(1, args.eq_steps))
        hcells = h.members * h.points
        units = hcells * base.r2_state_steps()
        step = lambda: h.response2(base.A, base.B, base.C, nt, nt, base.stride)
        desc = ("three_mode_hermite: the three_mode_20 model (3 water-like modes, omega 0.5/1.0/1.6) "
                "and q grid (20^3) with the momenta in %d^3 Hermite functions (Sec. III A, Appendix A), "
                "explicit 6th-order q-derivatives, depth 2 (10 members), dt=0.002; TRT R2 on %dx%d "
                "at dtau=0.1, all t1 branches batched; %d cells per state against %d on the 20^6 grid"
                % (K, nt, nt, hcells, base.cells))
        unit_name = "R2 spectra"
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
        result = step()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    if args.save_r2 and args.steps > 0:
        np.save(args.save_r2, np.asarray(result))
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
    if args.workload == "two_mode_hermite" and args.err_nt > 0:
        # the Hermite representation against the 32^4 grid representation of the same model and
        # q grid (both FP64 on the GPU, each from its own equilibrium), and its FP32 path against
        # its FP64 path
        n = args.err_nt
        Ceq = h.get_equilibrium()
        R = {}
        for prec_e in (32, 64):
            with chfpe.Handle(base.model, hgrid, depth=base.depth, dt=base.dt, precision=prec_e,
                              max_batch=n, stream=stream.cuda_stream, p_basis=1,
                              q_scheme=args.q_scheme) as he:
                he.set_equilibrium(Ceq)
                R[prec_e] = he.response2(base.A, base.B, base.C, n, n, base.stride)
        with chfpe.Handle(base.model, base.grid, depth=base.depth, dt=base.dt, precision=64,
                          max_batch=n, stream=stream.cuda_stream) as hg:
            hg.equilibrate(args.eq_steps, 1e-10, max(1, args.eq_steps))
            Rg = hg.response2(base.A, base.B, base.C, n, n, base.stride)
        line["error"] = {
            "samples": "%dx%d at dtau=0.2 (t1, t2 <= %.1f)" % (n, n, (n - 1) * 0.2),
            "f32_vs_f64": float(np.abs(R[32] - R[64]).max() / np.abs(R[64]).max()),
            "hermite_f64_vs_grid_32^4_f64": float(np.abs(R[64] - Rg).max() / np.abs(Rg).max()),
            "metric": "max |R2 - R2_ref| / max |R2_ref|"}
    if args.workload == "three_mode_hermite":
        line["s_per_spectrum"] = T / args.steps
        if args.err_nt > 0:
            # FP32 against FP64 from the same equilibrium, and K against K + 2 Hermite functions
            # (FP64, each from its own equilibrium): the truncation of the momentum basis
            n = args.err_nt
            Ceq = h.get_equilibrium()
            R = {}
            for prec_e in (32, 64):
                with chfpe.Handle(base.model, hgrid, depth=base.depth, dt=base.dt, precision=prec_e,
                                  max_batch=n, stream=stream.cuda_stream, p_basis=1) as he:
                    he.set_equilibrium(Ceq)
                    R[prec_e] = he.response2(base.A, base.B, base.C, n, n, base.stride)
            with chfpe.Handle(base.model, hgrid_of(K + 2), depth=base.depth, dt=base.dt, precision=64,
                              max_batch=n, stream=stream.cuda_stream, p_basis=1) as hk:
                hk.equilibrate(args.eq_steps, 1e-10, max(1, args.eq_steps))
                Rk = hk.response2(base.A, base.B, base.C, n, n, base.stride)
            line["error"] = {
                "samples": "%dx%d at dtau=0.1 (t1, t2 <= %.1f)" % (n, n, (n - 1) * 0.1),
                "f32_vs_f64": float(np.abs(R[32] - R[64]).max() / np.abs(R[64]).max()),
                "K_vs_K+2_f64": float(np.abs(R[64] - Rk).max() / np.abs(Rk).max()),
                "metric": "max |R2 - R2_ref| / max |R2_ref|"}
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
        if args.profile_case:
            run_profile_case(args)
        elif args.impl == "reference":
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
