"""Command line: plan and run square or cube solves on synthetic right-hand sides.

    python -m paper_1710_11259_gb300 --n 4096 --precision fp32_refine --reps 3 [--seed 2] [--power 2]
    python -m paper_1710_11259_gb300 --dim 3 --n 256 --seed 6 --reps 0 [--tol 0.5]
    python -m paper_1710_11259_gb300 --cylinder 128 --n 256 --reps 1     (modes 2..128, 4 rhs each)

Creates one plan, runs one warm-up solve and `reps` more solves on cuda:0 and
prints the plan facts and the mean time per timed solve (CUDA events).  Used as
the program under ncu when profiling a kernel on a chosen size.  Square right-hand
sides are F = g/((1+j)^p (1+k)^p), cube ones g/((1+i)^p (1+j)^p (1+k)^p); the
cylinder option solves the Fourier modes k = 2..KMAX (Sec. 4.1, Case 1) in FP64 with
four right-hand sides per mode of the square form.
"""
from __future__ import annotations

import argparse
import json


def main() -> None:
    ap = argparse.ArgumentParser(prog="python -m paper_1710_11259_gb300")
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--dim", type=int, default=2, choices=[2, 3])
    ap.add_argument("--precision", default="fp32_refine", choices=["fp64", "fp32_refine"])
    ap.add_argument("--tol", type=float, default=None)
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--cylinder", type=int, default=0, metavar="KMAX",
                    help="cylinder Fourier modes 2..KMAX (FP64) instead of a square or cube")
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--power", type=int, default=2)
    ap.add_argument("--instrument", action="store_true", help="time the ADI pass kernels (square plans)")
    a = ap.parse_args()

    import torch

    from . import api, build_ext, inputs

    build_ext.build()
    tol = a.tol if a.tol is not None else (1e-13 if a.precision == "fp64" else 1e-10)
    if a.cylinder:
        import numpy as np

        modes, nrhs = a.cylinder - 1, 4
        F = torch.from_numpy(np.stack([inputs.square_rhs(a.n, a.seed + m, power=a.power).reshape(1, a.n, a.n)
                                       .repeat(nrhs, 0) for m in range(modes)])).cuda()
        plan = api.plan_create_cylinder(a.n, 2, a.cylinder, 1e-13 if a.tol is None else a.tol, nrhs)
        Y = api.poisson_cylinder_solve(plan, F)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(a.reps):
            api.poisson_cylinder_solve(plan, F, Y)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / max(a.reps, 1)
        info = api.plan_info(plan)
        api.plan_destroy(plan)
        dofs = modes * nrhs * a.n * a.n
        print(json.dumps({"n": a.n, "cylinder_modes": [2, a.cylinder], "nrhs": nrhs,
                          "ms_per_solve": ms if a.reps > 0 else None,
                          "dofs_per_s": dofs / (ms * 1e-3) if a.reps > 0 and ms > 0 else None, **info}))
        return
    if a.dim == 2:
        F = torch.from_numpy(inputs.square_rhs(a.n, a.seed, power=a.power)).cuda()
        solve = api.poisson_square_solve
    else:
        F = torch.from_numpy(inputs.cube_rhs(a.n, a.seed, power=a.power)).cuda()
        solve = api.poisson_cube_solve
    plan = api.plan_create(a.n, a.dim, tol, a.precision)
    if a.instrument:
        api.plan_set_instrument(plan, True)
    X = solve(plan, F)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.reps):
        solve(plan, F, X)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(a.reps, 1)
    info = api.plan_info(plan)
    if a.instrument:
        info["pass_kernels"] = api.plan_kernel_times(plan)
    api.plan_destroy(plan)
    print(json.dumps({"n": a.n, "dim": a.dim, "precision": a.precision, "tol": tol,
                      "ms_per_solve": ms if a.reps > 0 else None,
                      "dofs_per_s": a.n ** a.dim / (ms * 1e-3) if a.reps > 0 and ms > 0 else None, **info}))


if __name__ == "__main__":
    main()
