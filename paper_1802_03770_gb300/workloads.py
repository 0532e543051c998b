"""The 3D time-stepping and batched workloads, timed on the GPU.

    python -m paper_1802_03770_gb300.workloads timestep [--steps 100]
    python -m paper_1802_03770_gb300.workloads batched [--count 64]

timestep: 256^3 interior grid (512^3 padded FFT), alpha = 1.5, backward
Euler dt = 1e-3, u0 = 16 seeded Gaussians (widths U(0.05, 0.15)), f = 0,
every step an FP32-CG + FP64-refinement solve of (I + dt M) u = u_prev to
1e-8 (preconditioner I + dt C h^d L), warm-started.
batched: 64 problems with sides uniform in {96, 128, ..., 768} and alpha ~
U(0.3, 1.8), seeded Gaussian-mixture right-hand sides, to 1e-8, solved in
lockstep (fl_solve_elliptic_batched) and, for comparison, one after another.
Each prints one JSON line.
"""

import argparse
import json
import time

from . import _lib as L
from . import inputs
from .api import Plan, solve_batched


def timestep(n=256, steps=100, alpha=1.5, dt=1e-3, seed=3):
    import torch
    p = Plan(3, (n, n, n), 1.0 / (n + 1), alpha)
    u = torch.tensor(inputs.gaussian_mixture(n, 3, 16, seed, 0.05, 0.15), dtype=torch.float64,
                     device="cuda").view(-1)
    nxt = torch.empty_like(u)
    its, ok = [], True
    p.time_step(u, dt, 1.0, out=nxt, tol=1e-8)          # warm-up (not timed)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        _, info = p.time_step(u, dt, 1.0, out=nxt, tol=1e-8)
        ok = ok and info["converged"] == 1
        its.append(info["iterations"])
        u, nxt = nxt, u
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    return {"workload": f"backward Euler, 3D {n}^3, alpha {alpha}, dt {dt}", "steps": steps,
            "seconds": t, "ms_per_step": 1e3 * t / steps, "mean_iterations": sum(its) / len(its),
            "all_converged": ok}


def batched(count=64, seed=7):
    import torch
    sides = inputs.batch_sides(count, seed)
    alphas = inputs.alpha_draws(count, seed + 1)
    plans, fs = [], []
    for i, (n, a) in enumerate(zip(sides, alphas)):
        plans.append(Plan(2, (n, n), 1.0 / (n + 1), a))
        fs.append(torch.tensor(inputs.gaussian_mixture(n, 2, 16, 100 + i), dtype=torch.float64,
                               device="cuda").view(-1))
    mode = L.FL_MODE_MIXED | L.FL_PRECOND_AUTO
    solve_batched(plans, fs, tol=1e-8, mode=mode)         # warm-up (graph capture)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, infos = solve_batched(plans, fs, tol=1e-8, mode=mode)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    t0 = time.perf_counter()
    for p, f in zip(plans, fs):
        p.solve(f, tol=1e-8, mode=mode)
    torch.cuda.synchronize()
    ts = time.perf_counter() - t0
    return {"workload": f"{count} 2D problems, sides 96..768, alpha U(0.3,1.8)",
            "batched_seconds": tb, "batched_solves_per_s": count / tb,
            "sequential_seconds": ts, "sequential_solves_per_s": count / ts,
            "all_converged": all(i["converged"] == 1 for i in infos),
            "total_dof": int(sum(n * n for n in sides))}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("which", choices=["timestep", "batched"])
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--count", type=int, default=64)
    args = ap.parse_args()
    res = timestep(steps=args.steps) if args.which == "timestep" else batched(args.count)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
