"""Learned surrogate of the two-mode R2 spectrum (12 parameters -> 64 x 64) on top of the solver.

Data: seeded parameter vectors drawn uniformly from the parameter sweep's ranges
(``inputs.surrogate_params``), each solved by ``chfpe_response2`` (A = B = C = q_1 + q_2,
FP32 state, FP64 equilibration).  Targets: the spectrum divided by its largest magnitude, and
log10 of that magnitude.  Inputs: the parameters mapped linearly onto [-1, 1].

Training and inference run in libchfpe's surrogate kernels (``chfpe.Surrogate``); this module
only marshals arrays, schedules the learning rate, and routes parameter vectors outside the
training ranges to the solver (the fallback).

    python -m paper_2509_25840_b300.surrogate --n-train 1024 --n-test 256 --data surr_data.npz
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import chfpe, inputs

LO, HI = inputs.SURROGATE_LO, inputs.SURROGATE_HI


def standardise(x) -> np.ndarray:
    return (2.0 * (np.asarray(x, dtype=np.float64) - LO) / (HI - LO) - 1.0).astype(np.float32)


def in_range(x) -> np.ndarray:
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    return np.all((x >= LO) & (x <= HI), axis=1)


# ------------------------------------------------------------------------------------------
# the solver
# ------------------------------------------------------------------------------------------

def solve(x, n_axis: int = 16, depth: int = 2, dt: float = 0.005, stride: int = 40, nt: int = 64,
          eq_steps: int = 4000, precision: int = 32) -> np.ndarray:
    """R2[t1][t2] of one parameter vector by the solver.  A dt the stability bound rejects is
    halved (and the stride doubled) until accepted, so the sampling times stay the same."""
    model = inputs.surrogate_model(x)
    grid = inputs.default_grid(model, [n_axis] * 4)
    mu = inputs.Optical(lin=(1.0, 1.0))
    sub = 1
    while True:
        try:
            h = chfpe.Handle(model, grid, depth=depth, dt=dt / sub, precision=precision,
                             max_batch=nt)
            break
        except chfpe.ChfpeError as e:
            if e.status != chfpe.EUNSTABLE or sub >= 64:
                raise
            sub *= 2
    with h:
        h.equilibrate(eq_steps * sub, 1e-10, 500)
        return h.response2(mu, mu, mu, nt, nt, stride * sub)


def make_dataset(seeds, **solver_kw):
    """(X [n][12] raw parameters, R [n][nt][nt], seconds spent in the solver)."""
    seeds = list(seeds)
    X = np.stack([inputs.surrogate_params(s) for s in seeds])
    R = np.empty((len(seeds), solver_kw.get("nt", 64), solver_kw.get("nt", 64)))
    t0 = time.perf_counter()
    for i, x in enumerate(X):
        R[i] = solve(x, **solver_kw)
    return X, R, time.perf_counter() - t0


def make_dataset_batched(seeds, n_axis: int = 16, depth: int = 2, dt: float = 0.005,
                         stride: int = 40, nt: int = 64, eq_steps: int = 4000, group: int = 64,
                         precision: int = 32):
    """The same data as make_dataset, solved `group` parameter vectors at a time by one batch
    (chfpe_create_batch: every instance's equilibration and R2 branches advance in the same
    launches; an instance that needs a smaller step substeps on its own)."""
    seeds = list(seeds)
    X = np.stack([inputs.surrogate_params(s) for s in seeds])
    R = np.empty((len(seeds), nt, nt))
    mu = inputs.Optical(lin=(1.0, 1.0))
    t0 = time.perf_counter()
    for i0 in range(0, len(seeds), group):
        xs = X[i0:i0 + group]
        models = [inputs.surrogate_model(x) for x in xs]
        grids = [inputs.default_grid(m, [n_axis] * 4) for m in models]
        with chfpe.Batch(models, grids, depth=depth, dt=dt, precision=precision, max_batch=nt) as b:
            b.equilibrate_all(eq_steps, 1e-10, 500)
            R[i0:i0 + len(xs)] = b.response2_all(mu, mu, mu, nt, nt, stride)
    return X, R, time.perf_counter() - t0


def targets(R):
    """(normalised spectra as float32 [n][4096], log10 scale as float32 [n])."""
    R = np.asarray(R, dtype=np.float64).reshape(len(R), -1)
    scale = np.abs(R).max(axis=1)
    scale = np.where(scale > 0, scale, 1.0)
    return (R / scale[:, None]).astype(np.float32), np.log10(scale).astype(np.float32)


# ------------------------------------------------------------------------------------------
# training and inference on the device
# ------------------------------------------------------------------------------------------

def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("the surrogate runs on a CUDA device")
    return torch


def train(sur: "chfpe.Surrogate", X, R, epochs: int, batch: int = 256, lr: float = 2e-3,
          lr_final: float = 2e-5, weight_decay: float = 1e-4, w_scale: float = 0.1,
          seed: int = 0):
    """Cosine learning-rate schedule, one library call per epoch; returns the epoch losses."""
    torch = _torch()
    T, TS = targets(R)
    dX = torch.from_numpy(standardise(X)).cuda()
    dT = torch.from_numpy(T).cuda()
    dTS = torch.from_numpy(TS).cuda()
    torch.cuda.synchronize()
    losses = []
    for ep in range(epochs):
        a = 0.5 * (1.0 + math.cos(math.pi * ep / max(1, epochs)))
        l = sur.train(dX.data_ptr(), dT.data_ptr(), dTS.data_ptr(), len(X), min(batch, len(X)),
                      1, lr_final + (lr - lr_final) * a, weight_decay, w_scale, seed + ep)
        losses.append(float(l[0]))
    return np.array(losses)


def infer(sur: "chfpe.Surrogate", X) -> np.ndarray:
    """R2 predictions [n][64][64] for raw parameter vectors (no range check)."""
    torch = _torch()
    n = len(X)
    dX = torch.from_numpy(standardise(X)).cuda()
    Y = torch.empty((n, chfpe.SURROGATE_NOUT), dtype=torch.float32, device="cuda")
    S = torch.empty(n, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    sur.infer(dX.data_ptr(), n, Y.data_ptr(), S.data_ptr())
    torch.cuda.synchronize()
    R = Y.double().cpu().numpy() * (10.0 ** S.double().cpu().numpy())[:, None]
    return R.reshape(n, 64, 64)


class Predictor:
    """Surrogate inside the training ranges, the solver outside them."""

    def __init__(self, sur: "chfpe.Surrogate", **solver_kw):
        self.sur, self.solver_kw = sur, solver_kw

    def predict(self, X):
        X = np.atleast_2d(np.asarray(X, dtype=np.float64))
        ok = in_range(X)
        R = np.empty((len(X), 64, 64))
        if ok.any():
            R[ok] = infer(self.sur, X[ok])
        for i in np.flatnonzero(~ok):
            R[i] = solve(X[i], **self.solver_kw)
        return R, ~ok


def rel_errors(pred, R) -> np.ndarray:
    """Per-spectrum relative Frobenius error ||pred - R|| / ||R||."""
    d = np.asarray(pred).reshape(len(R), -1) - np.asarray(R).reshape(len(R), -1)
    return np.linalg.norm(d, axis=1) / np.maximum(np.linalg.norm(np.asarray(R).reshape(len(R), -1), axis=1), 1e-300)


def make_surrogate(max_batch: int = 256, seed: int = 1) -> "chfpe.Surrogate":
    """A surrogate whose calls run on a torch stream of their own (so CUDA events can bracket
    them); ``sur.torch_stream`` is that stream."""
    torch = _torch()
    st = torch.cuda.Stream()
    sur = chfpe.Surrogate(max_batch=max_batch, seed=seed, stream=st.cuda_stream)
    sur.torch_stream = st
    return sur


def inference_rate(sur: "chfpe.Surrogate", n: int = 4096, reps: int = 5) -> float:
    """Spectra per second of chfpe_surrogate_infer on resident inputs: CUDA events on the
    surrogate's stream when it is a torch stream (``make_surrogate``), else wall clock around
    device synchronisations."""
    import time as _time
    torch = _torch()
    dX = torch.rand((n, 12), device="cuda") * 2 - 1
    Y = torch.empty((n, chfpe.SURROGATE_NOUT), device="cuda")
    S = torch.empty(n, device="cuda")
    torch.cuda.synchronize()          # inputs complete before the library's stream reads them
    sur.infer(dX.data_ptr(), n, Y.data_ptr(), S.data_ptr())
    torch.cuda.synchronize()
    st = getattr(sur, "torch_stream", None)
    if st is None:
        t0 = _time.perf_counter()
        for _ in range(reps):
            sur.infer(dX.data_ptr(), n, Y.data_ptr(), S.data_ptr())
        torch.cuda.synchronize()
        return n * reps / (_time.perf_counter() - t0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        sur.infer(dX.data_ptr(), n, Y.data_ptr(), S.data_ptr())
    e1.record(st)
    torch.cuda.synchronize()
    return n * reps / (e0.elapsed_time(e1) * 1e-3)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--n-train", type=int, default=1024)
    ap.add_argument("--n-test", type=int, default=256)
    ap.add_argument("--n-axis", type=int, default=10)
    ap.add_argument("--depth", type=int, default=2)
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--wd", type=float, default=1e-2, help="AdamW decoupled weight decay")
    ap.add_argument("--w-scale", type=float, default=0.1, help="weight of the log-scale loss")
    ap.add_argument("--data", default=None, help="npz cache of the solver data (read if present)")
    ap.add_argument("--extra-data", default=None,
                    help="further npz files (comma-separated) appended to the training set only")
    ap.add_argument("--generate-only", action="store_true",
                    help="solve and save the n-train + n-test spectra to --data, no training")
    ap.add_argument("--seed0", type=int, default=100000)
    ap.add_argument("--batched", type=int, default=0,
                    help="solve the data this many parameter vectors at a time in one batch "
                         "(0: one handle per vector)")
    args = ap.parse_args(argv)
    chfpe.load()
    kw = dict(n_axis=args.n_axis, depth=args.depth)
    n_all = args.n_train + args.n_test
    if args.data and os.path.exists(args.data):
        d = np.load(args.data)
        X, R = d["X"], d["R"].astype(np.float64)
        t_solve, n_solved = float(d["t_solve"]), int(d["n_solved"])
    elif args.batched > 0:
        X, R, t_solve = make_dataset_batched(range(args.seed0, args.seed0 + n_all), group=args.batched, **kw)
        n_solved = n_all
        if args.data:
            np.savez(args.data, X=X, R=R.astype(np.float32), t_solve=t_solve, n_solved=n_solved)
    else:
        X, R, t_solve = make_dataset(range(args.seed0, args.seed0 + n_all), **kw)
        n_solved = n_all
        if args.data:
            np.savez(args.data, X=X, R=R.astype(np.float32), t_solve=t_solve, n_solved=n_solved)
    if args.generate_only:
        print(json.dumps({"generated": int(n_solved), "seconds": t_solve, "data": args.data}))
        return None
    Xtr, Rtr = X[:args.n_train], R[:args.n_train]
    Xte, Rte = X[args.n_train:n_all], R[args.n_train:n_all]
    for extra in filter(None, (args.extra_data or "").split(",")):
        d = np.load(extra)
        Xtr = np.concatenate([Xtr, d["X"]])
        Rtr = np.concatenate([Rtr, d["R"].astype(np.float64)])
        t_solve += float(d["t_solve"])
        n_solved += int(d["n_solved"])
    torch = _torch()
    with make_surrogate(max_batch=max(args.batch, 256), seed=1) as sur:
        t0 = time.perf_counter()
        losses = train(sur, Xtr, Rtr, args.epochs, batch=args.batch, lr=args.lr,
                       weight_decay=args.wd, w_scale=args.w_scale)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        pred = infer(sur, Xte)
        err = rel_errors(pred, Rte)
        Tte, TSte = targets(Rte)
        Tp, TSp = targets(pred)
        err_shape = rel_errors(Tp, Tte)                       # normalised spectra
        err_log10_scale = np.abs(TSp - TSte)
        err_tr = rel_errors(infer(sur, Xtr[:len(Xte)]), Rtr[:len(Xte)])
        Ttr, TStr = targets(Rtr)
        mean_pred = Ttr.mean(axis=0)[None, :] * 10.0 ** TStr.mean()
        err_mean = rel_errors(np.repeat(mean_pred, len(Rte), axis=0), Rte)
        rate = inference_rate(sur)
        fallback_x = HI * 1.2
        t0 = time.perf_counter()
        Rfb, used = Predictor(sur, **kw).predict(fallback_x[None, :])
        t_fb = time.perf_counter() - t0
    report = {
        "n_train": int(len(Xtr)), "n_test": int(len(Xte)), "grid": [args.n_axis] * 4,
        "depth": args.depth, "epochs": args.epochs, "batch": args.batch,
        "solver_spectra_per_s": n_solved / t_solve,
        "train_s": t_train, "train_samples_per_s": args.epochs * (len(Xtr) // min(args.batch, len(Xtr))) * min(args.batch, len(Xtr)) / t_train,
        "loss_first": float(losses[0]), "loss_last": float(losses[-1]),
        "heldout_rel_err_median": float(np.median(err)), "heldout_rel_err_mean": float(err.mean()),
        "heldout_rel_err_p90": float(np.quantile(err, 0.9)),
        "train_rel_err_median": float(np.median(err_tr)),
        "heldout_shape_err_median": float(np.median(err_shape)),
        "heldout_log10_scale_err_median": float(np.median(err_log10_scale)),
        "lr": args.lr, "wd": args.wd, "w_scale": args.w_scale,
        "mean_predictor_rel_err_median": float(np.median(err_mean)),
        "surrogate_spectra_per_s": rate,
        "speedup_vs_solver": rate / (n_solved / t_solve),
        "fallback_used_solver": bool(used[0]), "fallback_s": t_fb,
    }
    print(json.dumps(report))
    return report


if __name__ == "__main__":
    main()
