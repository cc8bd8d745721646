"""Run one workload through libfga and print the Gaussian count and stage times.

  python -m paper_1304_3542_gb300.run_case [--workload layered_single|lens_2d|lens_3d|...] [--T 0.1]
                                           [--tau 1e-3] [--repeat 1] [--nshots 4]
                                           [--precision fp64|mixed] [--receivers] [--grad]
                                           [--z-method dynamic|divided] [--dz-eta 0.1]
                                           [--interp approx|interp] [--keep-n N]
                                           [--N 48 --eps 0.00694 --box 48 --stride 2 --k0 37.7]

A small driver for trying the library on the seeded workloads (and the command
the kernel profiles are taken with).
"""

from __future__ import annotations

import argparse
import json

import numpy as np


def main():
    import torch

    from . import fga as F
    from . import workloads as WL

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="layered_single",
                    choices=["layered_single", "layered_batch", "lens_2d", "lens_3d", "periodic_1d"])
    ap.add_argument("--T", type=float, default=None)
    ap.add_argument("--tau", type=float, default=None)
    ap.add_argument("--nshots", type=int, default=4)
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--receivers", action="store_true",
                    help="record traces at 368 surface receivers every 4 ms (layered model)")
    ap.add_argument("--grad", action="store_true",
                    help="with --receivers: also the adjoint dJ/dc for J = 1/2 |traces|^2")
    ap.add_argument("--z-method", choices=["dynamic", "divided"], default="dynamic")
    ap.add_argument("--dz-eta", type=float, default=0.1)
    ap.add_argument("--interp", choices=["approx", "interp"], default="approx")
    ap.add_argument("--keep-n", type=int, default=0)
    ap.add_argument("--N", type=int, default=None, help="lens workloads: grid points per axis")
    ap.add_argument("--eps", type=float, default=None, help="lens workloads: eps")
    ap.add_argument("--box", type=int, default=None, help="lens workloads: FBI box edge n_b")
    ap.add_argument("--stride", type=int, default=None, help="lens workloads: q-stride s")
    ap.add_argument("--k0", type=float, default=None, help="lens workloads: packet wavenumber")
    args = ap.parse_args()
    kw = {}
    for name, key in (("N", "N"), ("eps", "eps"), ("box", "box"), ("stride", "s"), ("k0", "k0")):
        if getattr(args, name) is not None:
            if not args.workload.startswith("lens"):
                ap.error("--%s applies to the lens workloads only" % name)
            kw[key] = getattr(args, name)
    if args.T is not None:
        kw["T"] = args.T
    if args.tau is not None:
        kw["tau"] = args.tau
    if args.workload == "layered_batch":
        kw["nshots"] = args.nshots
    prob = WL.by_name(args.workload, **kw)
    if args.keep_n > 0:
        prob = prob.with_(keep_n=args.keep_n)
    precision = F.FGA_MIXED_TF32X3 if args.precision == "mixed" else F.FGA_FP64
    divided = args.z_method == "divided"
    plan = F.plan_from_problem(prob, stream=torch.cuda.current_stream().cuda_stream,
                               precision=precision,
                               z_method=F.FGA_Z_DIVIDED if divided else F.FGA_Z_DYNAMIC,
                               dz_eta=args.dz_eta if divided else 0.0,
                               interp=F.FGA_BSPLINE_INTERP if args.interp == "interp"
                               else F.FGA_BSPLINE_APPROX)
    if args.receivers:
        xr = np.stack([0.025 * np.arange(368), np.zeros(368)], axis=1)
        plan.set_receivers(xr, int(round(0.004 / prob.dt)))
    u0, u1 = F.stacked_initial_data(prob)
    a, b = torch.from_numpy(u0).cuda(), torch.from_numpy(u1).cuda()
    out = torch.zeros((len(prob.shots),) + prob.n, dtype=torch.float64, device="cuda")
    for _ in range(args.repeat):
        counts = plan.decompose(a, b)
        plan.propagate()
        plan.reconstruct(out)
        plan.sync()
    extra = {}
    if args.receivers and args.grad:
        tr = plan.traces()
        g = plan.grad(np.ascontiguousarray(tr))
        extra = {"grad_max": float(np.abs(g).max())}
    times, launches = plan.stage_times()
    # (Gaussian, grid point) pairs inside the windows of the + branch (the reconstruction's
    # algorithmic work: one complex multiply-add each)
    pairs = sum(WL.window_evals(prob, plan.state(s)["Q"], prob.shots[s].eps)
                for s in range(len(prob.shots)))
    print(json.dumps({"workload": args.workload, "counts": counts.tolist(),
                      "ray_steps": plan.ray_steps(), "window_pairs": pairs,
                      "stage_ms": {k: float(v) for k, v in times.items()},
                      "launches": launches, "field_norm": float(out.norm()), **extra}))
    plan.close()


if __name__ == "__main__":
    main()
