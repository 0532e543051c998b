"""The 3D time-stepping and batched workloads, timed on the GPU.

    python -m paper_1802_03770_gb300.workloads timestep [--steps 100]
    python -m paper_1802_03770_gb300.workloads batched [--count 64]
    python -m paper_1802_03770_gb300.workloads lshape
    python -m paper_1802_03770_gb300.workloads octagon
    python -m paper_1802_03770_gb300.workloads tiles
    python -m paper_1802_03770_gb300.workloads richardson

timestep: 256^3 interior grid (512^3 padded FFT), alpha = 1.5, backward
Euler dt = 1e-3, u0 = 16 seeded Gaussians (widths U(0.05, 0.15)), f = 0,
every step an FP32-CG + FP64-refinement solve of (I + dt M) u = u_prev to
1e-8 (preconditioner I + dt C h^d L), warm-started.
batched: 64 problems with sides uniform in {96, 128, ..., 768} and alpha ~
U(0.3, 1.8), seeded Gaussian-mixture right-hand sides, to 1e-8, solved in
one call (fl_solve_elliptic_batched: one launch per pass over all problems,
and with FL_BATCH_PERSISTENT one persistent launch per refinement step) and,
for comparison, one after another.
lshape: the occluded-domain example (Sec. 4.4) at n = 128 .. 1024, alpha =
1.75, FP64 CG with and without the FD preconditioner (and with its
balanced shift), to 1e-6 and 1e-9; octagon: the same on the paper's
octagonal domain.
--precond picks the preconditioner of timestep and batched: fd (the
paper's; batched default: auto, none for alpha < 1), shifted (FD with the
balanced shift) or stencil (the stencil part of M).  --autotune tunes the
column tiles of the batch before timing: every plan's own tuned tiles
(fl_plan_autotune) or the widest, whichever runs the batched solve faster.
persistent: one 1024^2 and one 256^2 problem (alpha = 1.5) through the
batched call, with the persistent launch and with the lockstep launches,
without and with the FD preconditioner: time per CG iteration.
tiles: one FP32 apply + FD preconditioner solve (the work of a CG
iteration) on square 2D grids of side 96 .. 1024 and cubes of side 64 .. 256,
alpha = 1, timed with the widest column tiles (row shape 0) and after
fl_plan_autotune (column tiles and the FP32 row-pass shape).
richardson: the paper's grid error estimates (eq. rich) on the GPU:
f = M g_1 and u = M^-1 1 on 255^2 / 511^2 / 1023^2 (Sec. 4.2) and
63^3 / 127^3 / 255^3 (Sec. 4.3), and Crank-Nicolson to T = 0.25 with
dt = 1/(n+1) from the cosine product (nu = 3, 11, 2) on 255^2 .. 1023^2 and
31^3 .. 127^3 (Sec. 4.5); alpha = 1.25, 1.5, 1.75, FP64 applies, solves to
1e-11 (mixed), time steps to 1e-11.
Each prints one JSON line.
"""

import argparse
import json
import time

from . import _lib as L
from . import inputs
from .api import Plan, solve_batched


PRECONDS = {"fd": L.FL_PRECOND_FD, "auto": L.FL_PRECOND_AUTO, "shifted": L.FL_PRECOND_SHIFTED,
            "stencil": L.FL_PRECOND_STENCIL, "none": L.FL_PRECOND_NONE}


def timestep(n=256, steps=100, alpha=1.5, dt=1e-3, seed=3, precond="fd"):
    import torch
    mode = L.FL_MODE_MIXED | PRECONDS[precond]
    p = Plan(3, (n, n, n), 1.0 / (n + 1), alpha)
    u = torch.tensor(inputs.gaussian_mixture(n, 3, 16, seed, 0.05, 0.15), dtype=torch.float64,
                     device="cuda").view(-1)
    nxt = torch.empty_like(u)
    its, ok = [], True
    p.time_step(u, dt, 1.0, out=nxt, tol=1e-8, mode=mode)   # warm-up (not timed)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        _, info = p.time_step(u, dt, 1.0, out=nxt, tol=1e-8, mode=mode)
        ok = ok and info["converged"] == 1
        its.append(info["iterations"])
        u, nxt = nxt, u
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    return {"workload": f"backward Euler, 3D {n}^3, alpha {alpha}, dt {dt}", "precond": precond,
            "steps": steps,
            "seconds": t, "ms_per_step": 1e3 * t / steps, "mean_iterations": sum(its) / len(its),
            "all_converged": ok}


def tune_batch(plans, fs, mode, reps=2):
    """Launch shapes for a batch: every plan's own tuned column tiles and
    row-pass shape (fl_plan_autotune: the fastest for that plan alone)
    against the widest tiles on every plan with either row-pass shape on
    every plan (the lockstep launches take the 256 x 8 row shape only when
    every plan has it), each timed on the batched solve itself (lockstep
    launches, after a warm-up call); keeps the fastest.  A plan tuned alone
    favours narrow tiles (more CTAs to fill the GPU), which a batch of many
    problems does not need.  Returns the choice and the times (s)."""
    import torch
    tuned = [p.autotune() for p in plans]
    shapes = [p.row_shape() for p in plans]

    def timed():
        solve_batched(plans, fs, tol=1e-8, mode=mode)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            solve_batched(plans, fs, tol=1e-8, mode=mode)
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps

    def use(choice):
        for p, tx, rs in zip(plans, tuned, shapes):
            if choice == "per_plan":
                p.set_tiles(tx)
                p.set_row_shape(rs)
            else:
                p.set_tiles([0] * 6)
                p.set_row_shape(1 if choice == "widest_rows256x8" else 0)

    times = {"per_plan": timed()}
    candidates = ["widest", "widest_rows256x8"]
    if any(p.describe()["fft_len"][-1] < 256 for p in plans):
        candidates = ["widest"]        # the 256 x 8 rows need rows of >= 256 points
    for choice in candidates:
        use(choice)
        times[choice] = timed()
    best = min(times, key=times.get)
    use(best)
    return best, times


def batched(count=64, seed=7, precond="auto", autotune=False):
    import torch
    sides = inputs.batch_sides(count, seed)
    alphas = inputs.alpha_draws(count, seed + 1)
    plans, fs = [], []
    for i, (n, a) in enumerate(zip(sides, alphas)):
        plans.append(Plan(2, (n, n), 1.0 / (n + 1), a))
        fs.append(torch.tensor(inputs.gaussian_mixture(n, 2, 16, 100 + i), dtype=torch.float64,
                               device="cuda").view(-1))
    t_tune = 0.0
    mode = L.FL_MODE_MIXED | PRECONDS[precond]
    tile_choice, tile_times = "widest", {}
    if autotune:
        t0 = time.perf_counter()
        tile_choice, tile_times = tune_batch(plans, fs, mode)
        t_tune = time.perf_counter() - t0

    def timed(m):
        solve_batched(plans, fs, tol=1e-8, mode=m)        # warm-up (graph capture)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, inf = solve_batched(plans, fs, tol=1e-8, mode=m)
        torch.cuda.synchronize()
        return time.perf_counter() - t0, inf

    tb, infos = timed(mode | L.FL_BATCH_PERSISTENT)       # one persistent launch per step
    tl, infos_l = timed(mode)                             # one launch per pass
    for p, f in zip(plans, fs):                          # warm-up (per-plan graph capture)
        p.solve(f, tol=1e-8, mode=mode)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for p, f in zip(plans, fs):
        p.solve(f, tol=1e-8, mode=mode)
    torch.cuda.synchronize()
    ts = time.perf_counter() - t0
    return {"workload": f"{count} 2D problems, sides 96..768, alpha U(0.3,1.8)", "precond": precond,
            "autotuned_tiles": autotune, "autotune_seconds": t_tune,
            "tile_choice": tile_choice,
            "tile_trial_seconds": tile_times,
            "batched_seconds": tb, "batched_solves_per_s": count / tb,
            "batched_how": "inner CG of every problem in one persistent cooperative launch "
                           "per refinement step (CUDA graph)",
            "lockstep_seconds": tl, "lockstep_solves_per_s": count / tl,
            "sequential_seconds": ts, "sequential_solves_per_s": count / ts,
            "mean_iterations": sum(i["iterations"] for i in infos) / count,
            "lockstep_mean_iterations": sum(i["iterations"] for i in infos_l) / count,
            "all_converged": all(i["converged"] == 1 for i in infos + infos_l),
            "total_dof": int(sum(n * n for n in sides))}


def l_shape_mask(n):
    """The paper's L-shaped domain (Sec. 4.4): the (n-1)^2 interior points of
    the unit square (h = 1/n) without the (n/2)^2 points of one corner."""
    import numpy as np
    m = n - 1
    mask = np.ones((m, m), dtype=bool)
    mask[m - n // 2:, m - n // 2:] = False
    return mask


def octagon_mask(n):
    """The paper's octagonal domain (Sec. 4.4): the (n-1)^2 interior points
    of the unit square (h = 1/n) without the four corner triangles
    |x - c|_1 <= 1/4 (c a corner of the square).  The printed sizes
    (Table tab:octagon2: N = 14145 ... 915969) fix the cut: symmetric legs of
    1/4, the cut line excluded from Omega."""
    import numpy as np
    i = np.arange(1, n)
    a = np.minimum(i, n - i)                # grid distance to the nearer edge
    return (a[:, None] + a[None, :]) > n // 4


def lshape(sizes=(128, 256, 512, 1024), alpha=1.75, shape="lshape"):
    """FP64 CG on the L-shaped (or octagonal) domain, f = 1 on Omega, to 1e-6
    and 1e-9, as in the paper's Tables tab:L2 / tab:octagon2: with the FD
    operator on Omega (the paper's preconditioner; its set-up -- the
    capacitance factor of the hole's boundary -- timed as t_pc), with the
    restricted box solve, with the balanced shift, and plain CG."""
    import numpy as np
    import torch
    rows = []
    for n in sizes:
        mask = l_shape_mask(n) if shape == "lshape" else octagon_mask(n)
        p = Plan(2, mask.shape, 1.0 / n, alpha, mask=mask)
        f = torch.tensor(np.where(mask, 1.0, 0.0), dtype=torch.float64, device="cuda").view(-1)
        row = {"n": n, "N": int(mask.sum())}
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        p.precond(f)                       # builds the capacitance factor for (0, 1)
        torch.cuda.synchronize()
        row["t_pc"] = time.perf_counter() - t0
        for tol in (1e-6, 1e-9):
            for name, pm in (("prec", L.FL_PRECOND_FD), ("box", L.FL_PRECOND_BOX),
                             ("shifted", L.FL_PRECOND_SHIFTED), ("plain", L.FL_PRECOND_NONE)):
                p.solve(f, tol=tol, mode=L.FL_MODE_F64 | pm, maxit=1000, raise_on_fail=False)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                _, info = p.solve(f, tol=tol, mode=L.FL_MODE_F64 | pm, maxit=1000,
                                  raise_on_fail=False)
                torch.cuda.synchronize()
                row[f"{name}_{tol:g}"] = {"iterations": info["iterations"],
                                          "seconds": time.perf_counter() - t0,
                                          "converged": info["converged"]}
        rows.append(row)
    name = "L-shaped" if shape == "lshape" else "octagonal"
    return {"workload": f"{name} domain, alpha {alpha}, FP64 CG, f = 1", "rows": rows}


def tiles(shapes=((2, 96), (2, 128), (2, 192), (2, 256), (2, 384), (2, 512), (2, 768),
                  (2, 1024), (3, 64), (3, 128), (3, 256)), reps=20):
    import torch

    def per_iteration_us(p, N):
        u = torch.zeros(N, dtype=torch.float32, device="cuda")
        for _ in range(2):
            p.precond(p.apply(u))
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            p.precond(p.apply(u))
        e1.record()
        torch.cuda.synchronize()
        return 1e3 * e0.elapsed_time(e1) / reps

    rows = []
    for d, n in shapes:
        p = Plan(d, (n,) * d, 1.0 / (n + 1), 1.0)
        t_default = per_iteration_us(p, n ** d)
        t0 = time.perf_counter()
        tx = p.autotune()
        t_tune = time.perf_counter() - t0
        rows.append({"d": d, "n": n, "us_widest": round(t_default, 1),
                     "us_tuned": round(per_iteration_us(p, n ** d), 1), "tiles": tx,
                     "row_shape": p.row_shape(), "tune_seconds": round(t_tune, 3)})
        p.close()
    return {"workload": "FP32 apply + FD preconditioner solve, alpha 1", "rows": rows}


def _rates(c, m, f):
    """R_p = (log ||f_f - f_m||_p - log ||f_m - f_c||_p) / log(1/2), p = 2, inf,
    of three fields already restricted to the common coarse grid (eq. rich)."""
    import numpy as np
    out = {}
    for p, name in ((2, "R2"), (np.inf, "Rinf")):
        a = np.linalg.norm((f - m).ravel(), p)
        b = np.linalg.norm((m - c).ravel(), p)
        out[name] = float((np.log(a) - np.log(b)) / np.log(0.5))
    return out


def _on_coarse(v, n, k, d):
    """Values of a grid of n = 2^k (n_c + 1) - 1 points per axis at the points
    of the coarse grid (every 2^k-th point)."""
    s = 2 ** k
    return v.reshape((n,) * d)[(slice(s - 1, None, s),) * d]


def richardson(alphas=(1.25, 1.5, 1.75), parts=("2d", "3d", "td2", "td3")):
    import torch
    grids = {"2d": (2, (255, 511, 1023)), "3d": (3, (63, 127, 255)),
             "td2": (2, (255, 511, 1023)), "td3": (3, (31, 63, 127))}
    rows = []
    for part in parts:
        d, ns = grids[part]
        for alpha in alphas:
            fs, us = [], []
            for k, n in enumerate(ns):
                p = Plan(d, (n,) * d, 1.0 / (n + 1), alpha)
                if part in ("2d", "3d"):
                    g1 = torch.tensor(inputs.cosine_product(n, d, (1, 1, 1)), dtype=torch.float64,
                                      device="cuda").view(-1)
                    fs.append(_on_coarse(p.apply(g1).cpu().numpy(), n, k, d))
                    one = torch.ones(n ** d, dtype=torch.float64, device="cuda")
                    u, info = p.solve(one, tol=1e-11, mode=L.FL_MODE_MIXED | L.FL_PRECOND_FD)
                    assert info["converged"] == 1, info
                else:
                    dt = 1.0 / (n + 1)
                    u = torch.tensor(inputs.cosine_product(n, d), dtype=torch.float64,
                                     device="cuda").view(-1)
                    nxt = torch.empty_like(u)
                    for _ in range(round(0.25 / dt)):
                        _, info = p.time_step(u, dt, 0.5, out=nxt, tol=1e-11,
                                              mode=L.FL_MODE_MIXED | L.FL_PRECOND_FD)
                        assert info["converged"] == 1, info
                        u, nxt = nxt, u
                us.append(_on_coarse(u.cpu().numpy(), n, k, d))
                p.close()
            row = {"part": part, "d": d, "grids": list(ns), "alpha": alpha, "u": _rates(*us)}
            if fs:
                row["f"] = _rates(*fs)
            rows.append(row)
    return {"workload": "grid error estimates (eq. rich)", "rows": rows}


def persistent(sides=(1024, 256), alpha=1.5, reps=3):
    """Time per CG iteration of one problem solved through
    fl_solve_elliptic_batched with the persistent launch and with the
    lockstep launches, without and with the FD preconditioner (four and six
    passes per iteration)."""
    import torch
    rows = []
    for n in sides:
        plans = [Plan(2, (n, n), 1.0 / (n + 1), alpha)]
        fs = [torch.tensor(inputs.gaussian_mixture(n, 2, 32, 41), dtype=torch.float64,
                           device="cuda").view(-1)]
        for pname in ("none", "fd"):
            row = {"n": n, "precond": pname}
            for launch, extra in (("persistent", L.FL_BATCH_PERSISTENT), ("lockstep", 0)):
                mode = L.FL_MODE_MIXED | PRECONDS[pname] | extra
                solve_batched(plans, fs, tol=1e-8, mode=mode)    # warm-up (graph capture)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for _ in range(reps):
                    _, inf = solve_batched(plans, fs, tol=1e-8, mode=mode)
                torch.cuda.synchronize()
                dt = (time.perf_counter() - t0) / reps
                its = inf[0]["iterations"]
                row[launch] = {"ms_per_solve": 1e3 * dt, "iterations": its,
                               "us_per_iteration": 1e6 * dt / max(1, its)}
            rows.append(row)
    return {"workload": f"one 2D problem per batched call, alpha {alpha}, to 1e-8", "rows": rows}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("which", choices=["timestep", "batched", "lshape", "octagon", "tiles",
                                      "richardson", "persistent"])
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--count", type=int, default=64)
    ap.add_argument("--precond", choices=sorted(PRECONDS), default=None)
    ap.add_argument("--autotune", action="store_true",
                    help="batched: tune every plan's column tiles before timing")
    args = ap.parse_args()
    if args.which == "timestep":
        res = timestep(steps=args.steps, precond=args.precond or "fd")
    elif args.which == "batched":
        res = batched(args.count, precond=args.precond or "auto", autotune=args.autotune)
    elif args.which == "tiles":
        res = tiles()
    elif args.which == "persistent":
        res = persistent()
    elif args.which == "richardson":
        res = richardson()
    elif args.which == "octagon":
        res = lshape(shape="octagon")
    else:
        res = lshape()
    print(json.dumps(res))


if __name__ == "__main__":
    main()
