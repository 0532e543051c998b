"""Training and evaluation of the learned preconditioner (GPU, through the C ABI).

Training pairs come from the solver itself: for a seeded Gaussian-mixture
right-hand side f and order alpha, the converged solution u* and the plain
FP64 CG iterates x_k stopped at tolerances 1e-1 ... 1e-4 give residual /
error pairs r = f - M x_k, e = u* - x_k.  With the base preconditioner z0
(the FD-Laplacian solve for alpha >= 1, the diagonal scaling 1 / M_ii
below) and root-mean-square scales s_r, s_z the network input is
[r / s_r, z0 / s_z, alpha] and its target (e - z0) / s_z, so that
z = z0 + s_z N(...) approximates e = M^{-1} r.

Usage (GPU):  python -m paper_1802_03770_gb300.learned --n 512 --pairs 20000 \
                  --out weights.bin
"""

import argparse
import json
import os
import time

import numpy as np

from . import _lib as L
from . import inputs
from .api import Net, Plan

STAGES = (1e-1, 1e-2, 1e-3, 1e-4)


def make_pairs(plan, alpha, f, kernel0, stages=STAGES):
    """Features [len(stages), 3, n, n] and targets [len(stages), n, n] (float32):
    the converged solution u* and the CG iterates x stopped at each stage's
    tolerance, turned into pairs by fl_net_training_pair (residual, base
    preconditioner, scales, features and target in the library's kernels).
    alpha and kernel0 are the plan's (kept for the callers' signature)."""
    import torch
    n0, n1 = plan.n[0], plan.n[1]
    u_star, info = plan.solve(f, tol=1e-11, mode=L.FL_MODE_F64 | L.FL_PRECOND_AUTO, maxit=4000)
    feats, targets = [], []
    for tau in stages:
        x, _ = plan.solve(f, tol=tau, mode=L.FL_MODE_F64 | L.FL_PRECOND_AUTO, maxit=4000,
                          raise_on_fail=False)
        feat, target = plan.training_pair(f, u_star, x)
        feats.append(feat.view(3, n0, n1))
        targets.append(target.view(n0, n1))
    return torch.stack(feats), torch.stack(targets)


class PlanPool:
    """Plans for a fixed set of seeded orders alpha ~ U(lo, hi) on an n x n grid."""

    def __init__(self, n, count, seed, lo=0.3, hi=1.8):
        self.n = n
        self.alphas = inputs.alpha_draws(count, seed, lo, hi)
        self.plans = [Plan(2, (n, n), 1.0 / (n + 1), a) for a in self.alphas]
        self.k0 = [p.describe()["kernel0"] for p in self.plans]

    def pick(self, i):
        j = i % len(self.plans)
        return self.plans[j], float(self.alphas[j]), self.k0[j]


def train(n=512, pairs=20000, batch=4, lr=1e-3, seed=0, pool=16, log_every=50, net=None,
          max_seconds=None):
    """Train a network on solver-generated pairs; returns (net, history)."""
    import torch
    plans = PlanPool(n, pool, seed + 1)
    if net is None:
        net = Net(n, n, seed=seed)
    hist = []
    steps = max(1, pairs // len(STAGES))
    t0 = time.time()
    for step in range(steps):
        plan, alpha, k0 = plans.pick(step)
        f = torch.tensor(inputs.gaussian_mixture(n, 2, 16, seed * 100000 + step), dtype=torch.float64,
                         device="cuda").view(-1)
        xs, ts = make_pairs(plan, alpha, f, k0)
        for b0 in range(0, xs.shape[0], batch):
            loss = net.train_step(xs[b0:b0 + batch].contiguous(), ts[b0:b0 + batch].contiguous(), lr)
        if step % log_every == 0:
            hist.append((step, loss, time.time() - t0))
            if not np.isfinite(loss):
                break
        if max_seconds and time.time() - t0 > max_seconds:
            break
    return net, hist


def evaluate(net, n=512, seeds=range(10000, 10256), tol=1e-8, pool=16, alpha_seed=777):
    """Held-out comparison: iterations and wall time of FL_MODE_MIXED (plain
    FD-preconditioned CG inside refinement) vs FL_MODE_LEARNED."""
    import torch
    alphas = inputs.alpha_draws(len(seeds), alpha_seed)
    res = []
    cache = {}
    for k, sd in enumerate(seeds):
        a = float(alphas[k])
        key = round(a, 2)
        if key not in cache:
            if len(cache) >= pool:
                cache.pop(next(iter(cache)))
            p = Plan(2, (n, n), 1.0 / (n + 1), a)
            p.attach_net(net)
            cache[key] = p
        p = cache[key]
        f = torch.tensor(inputs.gaussian_mixture(n, 2, 16, sd), dtype=torch.float64, device="cuda").view(-1)
        row = {"seed": sd, "alpha": a}
        for name, mode in (("plain", L.FL_MODE_MIXED | L.FL_PRECOND_AUTO),
                           ("learned", L.FL_MODE_LEARNED | L.FL_PRECOND_AUTO)):
            torch.cuda.synchronize()
            t = time.perf_counter()
            _, info = p.solve(f, tol=tol, mode=mode, maxit=4000)
            torch.cuda.synchronize()
            row[name] = {"iterations": info["iterations"], "seconds": time.perf_counter() - t,
                         "rel_residual": info["rel_residual"], "converged": info["converged"]}
        res.append(row)
    return res


GATE_LO, GATE_HI, GATE_BANDS = 0.3, 1.8, 15


def choose_gate(rows, lo=GATE_LO, hi=GATE_HI, bands=GATE_BANDS):
    """Alpha gate from validation solves (`rows` of evaluate, network always
    on): a band is enabled when the mean learned iteration count of its
    solves is below the mean plain count.  Returns (flags, per-band stats)."""
    stats = []
    for b in range(bands):
        a0 = lo + (hi - lo) * b / bands
        a1 = lo + (hi - lo) * (b + 1) / bands
        sel = [r for r in rows if a0 <= r["alpha"] < a1]
        pl = float(np.mean([r["plain"]["iterations"] for r in sel])) if sel else float("nan")
        le = float(np.mean([r["learned"]["iterations"] for r in sel])) if sel else float("nan")
        stats.append((a0, a1, len(sel), pl, le))
    flags = [1 if (s[2] > 0 and s[4] < s[3]) else 0 for s in stats]
    return flags, stats


def write_gate(path, flags, stats, note, lo=GATE_LO, hi=GATE_HI):
    with open(path, "w") as fh:
        fh.write(f"# alpha gate: {note}\n")
        fh.write("# band: alpha range, validation solves, mean plain / learned iterations\n")
        for (a0, a1, cnt, pl, le), f in zip(stats, flags):
            fh.write(f"# [{a0:.2f}, {a1:.2f}): {cnt} solves, {pl:.1f} / {le:.1f} -> {'on' if f else 'off'}\n")
        fh.write(f"{lo} {hi} {len(flags)}\n")
        fh.write(" ".join(str(f) for f in flags) + "\n")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--pairs", type=int, default=20000)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--max-seconds", type=float, default=None)
    ap.add_argument("--pool", type=int, default=16,
                    help="training plans: seeded orders alpha ~ U(0.3, 1.8), cycled over the steps")
    ap.add_argument("--eval", type=int, default=32, help="held-out seeds to evaluate")
    ap.add_argument("--out", default=None)
    ap.add_argument("--report", default=None)
    ap.add_argument("--load", default=None,
                    help="evaluate these weights instead of training (e.g. weights/unet512.bin)")
    ap.add_argument("--tensor-cores", action="store_true",
                    help="run the network's 3x3 convolutions on the tcgen05 path")
    ap.add_argument("--gate-out", default=None,
                    help="choose the alpha gate on validation seeds 20000... (own alpha draws) "
                         "and write it here; the held-out evaluation then runs gated")
    ap.add_argument("--gate-seeds", type=int, default=256)
    args = ap.parse_args()
    if args.load:
        import torch
        torch.cuda.init()
        net = Net(args.n, args.n)
        net.load(args.load)
        hist = []
    else:
        net, hist = train(args.n, args.pairs, args.batch, args.lr, args.seed, pool=args.pool,
                          max_seconds=args.max_seconds)
        print(json.dumps({"history": hist}), flush=True)
        if args.out:
            net.save(args.out)
    if args.tensor_cores:
        net.tensor_cores(True)
    gate = None
    if args.gate_out:
        val = evaluate(net, args.n, range(20000, 20000 + args.gate_seeds), alpha_seed=555)
        flags, stats = choose_gate(val)
        write_gate(args.gate_out, flags, stats,
                   f"{args.gate_seeds} validation solves (seeds 20000.., alpha draws seed 555), "
                   f"512^2, tol 1e-8")
        net.set_alpha_gate(GATE_LO, GATE_HI, flags)
        gate = {"flags": flags, "stats": stats}
    ev = evaluate(net, args.n, range(10000, 10000 + args.eval))
    summary = {
        "history": hist,
        "plain_iterations": float(np.mean([r["plain"]["iterations"] for r in ev])),
        "learned_iterations": float(np.mean([r["learned"]["iterations"] for r in ev])),
        "plain_seconds": float(np.mean([r["plain"]["seconds"] for r in ev])),
        "learned_seconds": float(np.mean([r["learned"]["seconds"] for r in ev])),
        "all_converged": all(r["plain"]["converged"] and r["learned"]["converged"] for r in ev),
        "gate": gate,
        "rows": ev,
    }
    text = json.dumps(summary)
    if args.report:
        with open(args.report, "w") as fh:
            fh.write(text)
    print(json.dumps({k: v for k, v in summary.items() if k != "rows"}))


if __name__ == "__main__":
    main()
