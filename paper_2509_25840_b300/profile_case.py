"""Small, bounded case of the RK4 stage kernel for profilers (ncu): B states of a named workload
advanced `steps` RK4 steps through chfpe_rk4_device (4 stage launches per step).  --variant k
fixes the stage launch shape (no autotuning launches before the profiled ones).

    python -m paper_2509_25840_b300.profile_case --workload two_mode_32 --batch 4 --steps 2 --variant 3
"""
import argparse
import os

import torch

from . import chfpe, inputs

WORKLOADS = {"two_mode_32": inputs.two_mode_32, "one_mode_64": inputs.one_mode_64,
             "three_mode_20": inputs.three_mode_20}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="two_mode_32", choices=sorted(WORKLOADS))
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--precision", type=int, default=32, choices=[32, 64])
    ap.add_argument("--variant", type=int, default=None, choices=range(12))
    a = ap.parse_args()
    if a.variant is not None:
        os.environ["CHFPE_STAGE_VARIANT"] = str(a.variant)
    wl = WORKLOADS[a.workload]()
    h = chfpe.Handle(wl.model, wl.grid, depth=wl.depth, dt=wl.dt, precision=a.precision,
                     max_batch=a.batch)
    dtype = torch.float32 if a.precision == 32 else torch.float64
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.rand((a.batch,) + h.state_shape, dtype=dtype, device="cuda", generator=g) * 1e-3
    h.rk4_device(x.data_ptr(), a.batch, a.steps)
    torch.cuda.synchronize()
    print(f"ok {a.workload} batch={a.batch} steps={a.steps} variant={h.stage_tuning()[0]} "
          f"max={float(x.abs().max()):.6g}")
    h.close()


if __name__ == "__main__":
    main()
