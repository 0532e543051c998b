"""Benchmark: elliptic solves of the fractional Laplacian on a 1024 x 1024
interior grid (2048^2 padded FFT), alpha in {0.5, 1.0, 1.5}, right-hand
sides = 32 seeded Gaussians, to 1e-8 relative residual.

One step = one solve per alpha (three solves) with the FP32-inner / FP64-
refinement CG (preconditioner: FD Laplacian for alpha >= 1, none below, as
the paper advises).  Reported beside it: the same solves by plain FP64 CG on
the same GPU, the end-to-end time through the host-array C-ABI call (same
right-hand sides, same L2 flush), the roofline of the dominant kernel, the
learned-preconditioner arm (512^2, alpha ~ U(0.3, 1.8), held-out seeds:
plain FP64 CG, mixed, mixed + learned), the 3D 256^3 backward-Euler run with
the FP32 apply's roofline there, the 64-problem batch of uneven grids (one
persistent launch per refinement step against one launch per pass), and the
FP64 CPU oracle timed on the host (one full solve per alpha).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank solves its own seeds (weak scaling, no collective
on the data path); rank 0 prints one JSON line.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_SIDE = 1024
ALPHAS = (0.5, 1.0, 1.5)
BUMPS = 32
TOL = 1e-8
METRIC = "solves/s at 1e-8 rel. residual, mixed+learned vs plain FP64 PCG; apply HBM GB/s"
UNIT = "solves/s"
WORKLOAD = ("elliptic solve 2D 1024x1024 interior grid (2048^2 padded FFT), alpha in "
            "{0.5,1.0,1.5}, RHS 32 seeded Gaussians, FP32 inner CG + FP64 refinement to 1e-8")
L2_FLUSH_BYTES = 512 << 20


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def rhs_seed(rank, step, j):
    """Seed of the right-hand side of solve j of step `step` on `rank`:
    every rank solves its own problems (replicas, weak scaling)."""
    return 1000 * rank + 10 * step + j


def max_over_ranks(values, world, device):
    """Element-wise maximum over the ranks of per-rank times: the job takes
    as long as its slowest rank.  One all-reduce, no data-path collective."""
    if world == 1:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(v) for v in t]


def job_rate(world, units_per_step, seconds_per_step):
    """Whole-job throughput: the units all ranks processed per second."""
    return world * units_per_step / seconds_per_step


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = [r.split(",") for r in (self.out or "").strip().splitlines() if r.count(",") >= 7]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in rows if r[0].strip().replace(".", "").isdigit()]
        smax = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4)
                          if r[4 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


def make_rhs(seed):
    from paper_1802_03770_gb300 import inputs
    return inputs.gaussian_mixture(N_SIDE, 2, BUMPS, seed)


# DRAM bytes (read + write) per launch of the dominant kernel from one ncu
# capture (`ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum` on
# `python bench.py --profile-case`, the first and the last preconditioner
# pass of a CG iteration averaged).  ncu flushes the caches before each
# captured launch, so this is the cold-cache traffic; in the timed loop the
# arrays stay in L2.  An entry holds only for the kernel source it was taken
# from: it is keyed by the SHA-256 of the CUDA sources (kernel_source_sha)
# and reported as null for any other source.
NCU_DRAM_BYTES = {
    # k_dst_rows<float, 128, 16>, 1024^2, mean of four launches: 16920576 /
    # 16920576 (first pass) and 8558080 / 8558336 (last pass) bytes read, 0
    # written (the launch list of the capture is summarised under profiles/)
    "dst_rows<f32>": ("af3ded8c2bf1acd9", 12739392),
}


# the sources that make up the single-plan pass kernels and their launch
# shapes (the roofline kernel's code and configuration)
PASS_KERNEL_SOURCES = ("chain.cuh", "fft_core.cuh", "internal.h", "kernels.cuh", "ops.cu")


def kernel_source_sha():
    """SHA-256 (first 16 hex digits) of the pass kernels' CUDA sources."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_1802_03770_gb300", "csrc")
    h = hashlib.sha256()
    for name in PASS_KERNEL_SOURCES:
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(name.encode() + b"\0" + fh.read())
    return h.hexdigest()[:16]


def measured_traffic(name):
    entry = NCU_DRAM_BYTES.get(name)
    if entry and entry[0] == kernel_source_sha():
        return entry[1]
    return None


def algorithmic_bytes(name, n, L, elem):
    """Compulsory HBM bytes of one launch of a pass kernel on an n x n grid
    (each pass reads and writes its working array once; the symbol is read
    once in its compact (L/2+1)^2 form)."""
    H = L // 2 + 1
    N = n * n
    spec = n * H * 2 * elem          # half spectrum, complex
    real = N * elem
    table = {
        "rows_fwd": 3 * real + spec,             # z, p in; p out; spectrum out
        "cols_conv": 2 * spec + (L // 2 + 1) * H * elem,
        "rows_inv": spec + 2 * real,             # spectrum, p in; q out
        # one CG iteration launches it twice: x, r, p, q in and x, r, t out
        # (with the CG update), then t, r in and z out: 10 N values per pair
        "dst_rows": 5 * real,
        "tri_cols": 2 * real,                    # t in, z out
        "dst_cols": 2 * real,
    }
    base = name.split("<")[0]
    return table.get(base)


def apply_bytes(n, L, elem):
    """Streamed bytes of one 2D apply (three passes, each reading and writing
    its working array once, the compact symbol read once)."""
    H = L // 2 + 1
    real = n * n * elem
    spec = n * H * 2 * elem
    return real + spec + (2 * spec + H * H * elem) + spec + real


def time_apply(plan, dev, reps=50):
    """Operator apply y = M u on the workload grid: ours (FP32 and FP64) and,
    beside it as a reference only, a cuFFT (torch.fft) zero-padded
    convolution of the same shape with a stand-in symbol.  Inputs are
    L2-resident, as inside the CG loop."""
    import torch
    L = 2 * N_SIDE
    out = {}
    for dt, tag in ((torch.float32, "f32"), (torch.float64, "f64")):
        u = torch.randn(N_SIDE * N_SIDE, dtype=dt, device=dev)
        y = torch.empty_like(u)
        for _ in range(5):
            plan.apply(u, y)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            plan.apply(u, y)
        e1.record()
        torch.cuda.synchronize()
        t_ours = e0.elapsed_time(e1) / reps * 1e3
        sym = torch.rand(L, L // 2 + 1, dtype=dt, device=dev)
        pad = torch.zeros(L, L, dtype=dt, device=dev)

        def cufft_apply():
            pad[:N_SIDE, :N_SIDE] = u.view(N_SIDE, N_SIDE)
            s = torch.fft.rfft2(pad)
            s *= sym
            return torch.fft.irfft2(s, s=(L, L))[:N_SIDE, :N_SIDE].contiguous()

        for _ in range(5):
            cufft_apply()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            cufft_apply()
        e1.record()
        torch.cuda.synchronize()
        t_ref = e0.elapsed_time(e1) / reps * 1e3
        ab = apply_bytes(N_SIDE, L, 4 if tag == "f32" else 8)
        out[tag] = {"us": round(t_ours, 2), "streamed_bytes": ab,
                    "gbs": round(ab / (t_ours * 1e-6) / 1e9, 1),
                    "cufft_reference_us": round(t_ref, 2)}
    return out


def run_ours(args, rank, world, local):
    import torch
    from paper_1802_03770_gb300 import _lib
    from paper_1802_03770_gb300.api import Plan, launch_count

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    h = 1.0 / (N_SIDE + 1)
    t0 = time.perf_counter()
    plans = [Plan(2, (N_SIDE, N_SIDE), h, a) for a in ALPHAS]
    torch.cuda.synchronize()
    t_con = (time.perf_counter() - t0) / len(plans)
    tiles = [p.autotune() for p in plans]     # column tiles (plan set-up, untimed)
    mode_mixed = _lib.FL_MODE_MIXED | _lib.FL_PRECOND_AUTO
    mode_f64 = _lib.FL_MODE_F64 | _lib.FL_PRECOND_AUTO
    steps, warm = args.steps, args.warmup
    nsteps = steps + warm
    # inputs resident in HBM before timing: one RHS per (step, alpha)
    rhs = [[torch.tensor(make_rhs(rhs_seed(rank, s, j)), dtype=torch.float64, device=dev)
            for j in range(len(ALPHAS))] for s in range(nsteps)]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def dist_barrier():
        if world > 1:
            torch.distributed.barrier()

    def timed(mode, nsteps_timed, nwarm, collect=None):
        infos = []
        for s in range(nwarm):
            for j, p in enumerate(plans):
                p.solve(rhs[s][j].view(-1), tol=TOL, mode=mode)
        dist_barrier()
        torch.cuda.synchronize()
        total_ms = 0.0
        l0 = launch_count()
        for s in range(nwarm, nwarm + nsteps_timed):
            flush.fill_(float(s))            # evict L2 between timed steps (untimed)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for j, p in enumerate(plans):
                # from u = 0 (no initial guess: the first residual is f itself)
                _, info = p.solve(rhs[s % nsteps][j].view(-1), tol=TOL, mode=mode)
                infos.append(info)
            e1.record()
            torch.cuda.synchronize()
            total_ms += e0.elapsed_time(e1)
        dist_barrier()
        torch.cuda.synchronize()
        launches = launch_count() - l0
        return total_ms / nsteps_timed, infos, launches

    with ClockSampler(local) as clk:
        ms_mixed, infos_mixed, launches = timed(mode_mixed, steps, warm)
    clocks = clk.summary()
    for info in infos_mixed:
        assert info["converged"] == 1 and info["rel_residual"] <= TOL, info
    # plain FP64 CG on the same GPU, same inputs (fewer steps: it is slower)
    k64 = max(1, min(steps, 2))
    ms_f64, infos_f64, _ = timed(mode_f64, k64, 1)
    for info in infos_f64:
        assert info["converged"] == 1, info
    # error of the mixed solutions against tight FP64 GPU PCG solutions (the
    # FP64 path is checked against the oracle by the parity tests), on the
    # first timed step's right-hand sides; untimed
    mixed_errors = []
    for j, p in enumerate(plans):
        fj = rhs[warm % nsteps][j].view(-1)
        um = torch.zeros_like(fj)
        p.solve(fj, um, tol=TOL, mode=mode_mixed)
        ur = torch.zeros_like(fj)
        p.solve(fj, ur, tol=1e-12, mode=mode_f64, maxit=4000)
        mixed_errors.append(float(torch.linalg.norm(um - ur) / torch.linalg.norm(ur)))

    # the same step as one batched call: the three problems advance in
    # lockstep, one launch per pass over all of them (CG iterations replayed
    # as a CUDA graph), same right-hand sides, same L2 flush
    from paper_1802_03770_gb300.api import solve_batched

    def timed_batched(nsteps_timed, nwarm):
        for s in range(nwarm):
            solve_batched(plans, [rhs[s][j].view(-1) for j in range(len(ALPHAS))], tol=TOL,
                          mode=mode_mixed)
        dist_barrier()
        torch.cuda.synchronize()
        total_ms, infos = 0.0, []
        for s in range(nwarm, nwarm + nsteps_timed):
            flush.fill_(float(s))
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            _, inf = solve_batched(plans, [rhs[s % nsteps][j].view(-1) for j in range(len(ALPHAS))],
                                   tol=TOL, mode=mode_mixed)
            e1.record()
            torch.cuda.synchronize()
            total_ms += e0.elapsed_time(e1)
            infos += inf
        return total_ms / nsteps_timed, infos

    ms_batched, infos_batched = timed_batched(steps, min(warm, 2))
    for info in infos_batched:
        assert info["converged"] == 1 and info["rel_residual"] <= TOL, info

    # the same mixed solves with the balanced-shift FD preconditioner (not
    # the paper's preconditioner; reported beside the headline, not in it)
    mode_shift = _lib.FL_MODE_MIXED | _lib.FL_PRECOND_SHIFTED
    ms_shift, infos_shift, _ = timed(mode_shift, steps, 1)
    for info in infos_shift:
        assert info["converged"] == 1 and info["rel_residual"] <= TOL, info

    ms_mixed, ms_f64, ms_shift, ms_batched = max_over_ranks([ms_mixed, ms_f64, ms_shift, ms_batched],
                                                            world, dev)
    solves_per_step = len(ALPHAS)
    value = job_rate(world, solves_per_step, ms_mixed / 1e3)
    value_f64 = job_rate(world, solves_per_step, ms_f64 / 1e3)
    value_shift = job_rate(world, solves_per_step, ms_shift / 1e3)

    # end to end: host arrays in, host arrays out, through the C ABI, on the
    # right-hand sides of the timed steps (pinned host copies), L2 flushed
    # between steps as for `value`
    f_host = [[rhs[s][j].cpu().pin_memory() for j in range(len(ALPHAS))]
              for s in range(nsteps)]
    for j, p in enumerate(plans):
        p.solve_host(f_host[0][j].numpy(), tol=TOL, mode=mode_mixed)
    torch.cuda.synchronize()
    dist_barrier()
    e2e_s = 0.0
    for s in range(warm, warm + steps):
        flush.fill_(float(s))                # untimed, as for `value`
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for j, p in enumerate(plans):
            _, info = p.solve_host(f_host[s][j].numpy(), tol=TOL, mode=mode_mixed)
            assert info["converged"] == 1
        e2e_s += time.perf_counter() - t0
    e2e_s /= steps
    dist_barrier()
    e2e_s = max_over_ranks([e2e_s], world, dev)[0]
    e2e = {"value": job_rate(world, solves_per_step, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": solves_per_step * N_SIDE * N_SIDE * 8,
           "d2h_bytes_per_step": solves_per_step * N_SIDE * N_SIDE * 8,
           "ms_per_step": e2e_s * 1e3}

    apply = time_apply(plans[-1], dev)

    # per-kernel device time over profiled steps (CUDA events around each launch)
    for p in plans:
        p.profile(True)
    for s in range(warm, warm + max(1, min(steps, 2))):
        for j, p in enumerate(plans):
            p.solve(rhs[s][j].view(-1), tol=TOL, mode=mode_mixed)
    stats = {}
    for p in plans:
        for name, (cnt, tot) in p.profile_read().items():
            c0, t0_ = stats.get(name, (0, 0.0))
            stats[name] = (c0 + cnt, t0_ + tot)
        p.profile(False)
    total = sum(t for _, t in stats.values())
    top = sorted(stats.items(), key=lambda kv: -kv[1][1])
    roofline = None
    peak, peak_kind = peaks()
    for name, (cnt, tot) in top:
        elem = 4 if "f32" in name else 8
        ab = algorithmic_bytes(name, N_SIDE, 2 * N_SIDE, elem)
        if ab is None:
            continue
        avg_s = tot / cnt / 1e3
        achieved = ab / avg_s / 1e9
        roofline = {"bound": "hbm", "kernel": name, "achieved": round(achieved, 1),
                    "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                    "frac": round(achieved / peak, 4), "traffic": measured_traffic(name),
                    "bytes_per_launch": ab, "avg_launch_us": round(avg_s * 1e6, 2),
                    "share": round(tot / total, 4) if total else None}
        break
    kernel_shares = {k: {"launches": c, "ms": round(t, 3), "share": round(t / total, 4)}
                     for k, (c, t) in top[:10]}
    learned = learned_arm(dev) if not args.no_learned else None
    td3 = timestep_3d(dev, peak, peak_kind) if not args.no_3d else None
    b64 = batched_64() if not args.no_batch64 else None
    its_mixed = [i["iterations"] for i in infos_mixed[: len(ALPHAS)]]
    its_f64 = [i["iterations"] for i in infos_f64[: len(ALPHAS)]]
    return {
        "value": value, "ms_per_step": ms_mixed, "clocks": clocks, "e2e": e2e,
        "gpu_launches": int(launches), "roofline": roofline, "t_con_s": t_con,
        "fp64_pcg": {"value": value_f64, "unit": UNIT, "ms_per_step": ms_f64,
                     "iterations": its_f64},
        "speedup_vs_fp64_pcg": value / value_f64,
        "batched": {"value": job_rate(world, len(ALPHAS), ms_batched / 1e3), "unit": UNIT,
                    "ms_per_step": ms_batched,
                    "how": "the step's three solves in one fl_solve_elliptic_batched call (one "
                           "launch per pass over all problems, CG iterations as a CUDA graph)",
                    "iterations": [i["iterations"] for i in infos_batched[: len(ALPHAS)]]},
        "balanced_shift": {
            "value": value_shift, "unit": UNIT, "ms_per_step": ms_shift,
            "preconditioner": "(x I + C h^d L)^-1, x balancing the extreme sine modes (not in the paper)",
            "x": [p.precond_params(mode_shift)[0] for p in plans],
            "iterations": [i["iterations"] for i in infos_shift[: len(ALPHAS)]],
            "refinements": [i["outer_iterations"] for i in infos_shift[: len(ALPHAS)]]},
        "mixed_error_vs_fp64": {"alphas": list(ALPHAS), "rel_error": mixed_errors,
                                "reference": "FP64 PCG on the GPU to 1e-12 relative residual"},
        "iterations_mixed": its_mixed,
        "refinements": [i["outer_iterations"] for i in infos_mixed[: len(ALPHAS)]],
        "kernels": kernel_shares, "apply": apply, "tiles": tiles,
        "learned": learned, "timestep_3d": td3, "batched_64": b64,
    }


def batched_64():
    """The 64-problem batch: sides uniform in {96, 128, ..., 768}, alpha ~
    U(0.3, 1.8), seeded Gaussian-mixture right-hand sides, FP32 inner CG +
    FP64 refinement to 1e-8, the inner CG of every refinement step in one
    persistent launch (graph-captured) with column tiles tuned for the batch
    (each plan's own tuned tiles or the widest, whichever ran the batch
    faster);
    beside it the same batch with one launch per pass (lockstep) and the 64
    solves one after another (host wall clock, each after a warm-up call)."""
    from paper_1802_03770_gb300 import workloads
    r = workloads.batched(count=64, seed=7, precond="auto", autotune=True)
    return {"workload": r["workload"], "value": r["batched_solves_per_s"], "unit": UNIT,
            "how": r["batched_how"] + ", column tiles tuned for the batch",
            "tile_choice": r["tile_choice"], "tile_trial_seconds": r["tile_trial_seconds"],
            "lockstep": r["lockstep_solves_per_s"], "sequential": r["sequential_solves_per_s"],
            "mean_iterations": r["mean_iterations"],
            "lockstep_mean_iterations": r["lockstep_mean_iterations"],
            "autotune_seconds": r["autotune_seconds"], "total_dof": r["total_dof"],
            "all_converged": r["all_converged"]}


LEARNED_N = 512
LEARNED_SEEDS = 32
WEIGHTS = os.path.join(ROOT, "paper_1802_03770_gb300", "weights", "unet512.bin")
# the weights' alpha gate (learned.py --gate-out, chosen on validation seeds
# 20000.. with their own alpha draws, disjoint from the held-out seeds here)
WEIGHTS_GATE = os.path.join(ROOT, "paper_1802_03770_gb300", "weights", "unet512_gate.txt")


def learned_arm(dev, seeds=LEARNED_SEEDS):
    """The learned-preconditioner configuration: 512 x 512, alpha ~
    U(0.3, 1.8) (one draw per held-out seed 10000, 10001, ...), right-hand
    sides of 16 seeded Gaussians, to 1e-8: plain FP64 CG, the mixed path and
    the mixed path with the trained network, each plan's launch shapes tuned
    at set-up (fl_plan_autotune) and each (plan, mode) warmed up on another
    right-hand side first.  Solves/s over the timed solves and mean
    iterations per mode.  `learned` runs FL_MODE_LEARNED with the weights'
    alpha gate (the network only in the alpha bands where it lowered the
    validation iteration count, plain preconditioned CG elsewhere);
    `learned_network_always` runs it without the gate."""
    import torch
    from paper_1802_03770_gb300 import _lib, inputs
    from paper_1802_03770_gb300.api import Net, Plan
    n = LEARNED_N
    if not os.path.exists(WEIGHTS):
        return {"unavailable": "no trained weights"}
    net = Net(n, n)
    net.load(WEIGHTS)
    net.tensor_cores(True)
    gated = os.path.exists(WEIGHTS_GATE)
    alphas = inputs.alpha_draws(seeds, 777)
    modes = {"fp64": _lib.FL_MODE_F64 | _lib.FL_PRECOND_AUTO,
             "mixed": _lib.FL_MODE_MIXED | _lib.FL_PRECOND_AUTO,
             "learned": _lib.FL_MODE_LEARNED | _lib.FL_PRECOND_AUTO}
    if gated:
        modes["learned_network_always"] = _lib.FL_MODE_LEARNED | _lib.FL_PRECOND_AUTO
    ms = {k: 0.0 for k in modes}
    its = {k: [] for k in modes}
    ok = True
    for k in range(seeds):
        a = float(alphas[k])
        p = Plan(2, (n, n), 1.0 / (n + 1), a)
        p.autotune()                # column tiles and row-pass shape (set-up, untimed)
        p.attach_net(net)
        f = torch.tensor(inputs.gaussian_mixture(n, 2, 16, 10000 + k), dtype=torch.float64,
                         device=dev).view(-1)
        fw = torch.tensor(inputs.gaussian_mixture(n, 2, 16, 30000 + k), dtype=torch.float64,
                          device=dev).view(-1)
        for name, mode in modes.items():
            if name == "learned" and gated:
                net.load_gate(WEIGHTS_GATE)
            elif name == "learned_network_always":
                net.set_alpha_gate()
            p.solve(fw, tol=TOL, mode=mode, maxit=4000)          # warm-up (untimed)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            _, info = p.solve(f, tol=TOL, mode=mode, maxit=4000)
            e1.record()
            torch.cuda.synchronize()
            ms[name] += e0.elapsed_time(e1)
            its[name].append(info["iterations"])
            ok = ok and info["converged"] == 1 and info["rel_residual"] <= TOL
        p.close()
    net.check()
    out = {"workload": f"elliptic solve 2D {n}x{n}, alpha ~ U(0.3,1.8), RHS 16 seeded Gaussians, "
                       f"{seeds} held-out seeds 10000..{10000 + seeds - 1}, to 1e-8",
           "network": "3-level U-Net 16/32/64, BF16 weights, tcgen05 3x3 convolutions",
           "gate": ("alpha bands where the network lowered the validation iteration count "
                    "(weights/unet512_gate.txt); plain preconditioned CG elsewhere") if gated else None,
           "all_converged": ok}
    for name in modes:
        out[name] = {"value": seeds / (ms[name] / 1e3), "unit": UNIT,
                     "ms_per_solve": ms[name] / seeds,
                     "mean_iterations": float(np.mean(its[name]))}
    out["learned_vs_fp64"] = out["learned"]["value"] / out["fp64"]["value"]
    out["learned_vs_mixed"] = out["learned"]["value"] / out["mixed"]["value"]
    return out


def timestep_3d(dev, peak, peak_kind, n=256, steps=100, alpha=1.5, dt=1e-3):
    """The 3D diffusion configuration: 256^3 interior grid (512^3 padded
    FFT), alpha = 1.5, backward Euler, dt = 1e-3, 100 steps, u0 = 16 seeded
    Gaussians (widths U(0.05, 0.15)), f = 0, each step to 1e-8 in FP32 +
    FP64 refinement; and the FP32 apply on this grid, whose arrays stream
    from HBM (1.82 GB of algorithmic traffic per apply, five passes)."""
    import torch
    from paper_1802_03770_gb300 import _lib, inputs
    from paper_1802_03770_gb300.api import Plan
    p = Plan(3, (n, n, n), 1.0 / (n + 1), alpha)
    u = torch.tensor(inputs.gaussian_mixture(n, 3, 16, 3, 0.05, 0.15), dtype=torch.float64,
                     device=dev).view(-1)
    nxt = torch.empty_like(u)
    mode = _lib.FL_MODE_MIXED | _lib.FL_PRECOND_FD
    p.time_step(u, dt, 1.0, out=nxt, tol=TOL, mode=mode)       # warm-up (untimed)
    torch.cuda.synchronize()
    its, ok = [], True
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        _, info = p.time_step(u, dt, 1.0, out=nxt, tol=TOL, mode=mode)
        ok = ok and info["converged"] == 1
        its.append(info["iterations"])
        u, nxt = nxt, u
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    # FP32 apply on the same plan: inputs far larger than L2
    x = torch.randn(n ** 3, dtype=torch.float32, device=dev)
    y = torch.empty_like(x)
    for _ in range(3):
        p.apply(x, y)
    torch.cuda.synchronize()
    reps = 20
    e0.record()
    for _ in range(reps):
        p.apply(x, y)
    e1.record()
    torch.cuda.synchronize()
    us = e0.elapsed_time(e1) / reps * 1e3
    ab = apply_bytes_3d(n, 2 * n, 4)
    achieved = ab / (us * 1e-6) / 1e9
    p.close()
    return {"workload": f"backward Euler 3D {n}^3 (512^3 padded FFT), alpha {alpha}, dt {dt}, "
                        f"{steps} steps, u0 16 seeded Gaussians, f = 0, each step to 1e-8",
            "ms_per_step": ms / steps, "mean_iterations": float(np.mean(its)),
            "all_converged": ok,
            "apply_f32": {"us": round(us, 1), "bytes_per_apply": ab,
                          "roofline": {"bound": "hbm", "achieved": round(achieved, 1),
                                       "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                                       "frac": round(achieved / peak, 4)}}}


def apply_bytes_3d(n, L, elem):
    """Streamed bytes of one 3D apply (five passes): u -> S (rows), S -> S'
    (middle axis forward, spectrum grows to L along it), S' -> S' (outer
    axis convolution, compact symbol read once), S' -> S (middle axis
    inverse), S -> y (rows)."""
    H = L // 2 + 1
    real = n ** 3 * elem
    spec = n * n * H * 2 * elem
    spec_l = n * L * H * 2 * elem
    sym = H ** 3 * elem
    return (real + spec) + (spec + spec_l) + (2 * spec_l + sym) + (spec_l + spec) + (spec + real)


def oracle_solve(alpha, seed):
    """One full FP64 oracle solve of the workload (operator construction
    untimed): (seconds, iterations)."""
    from oracle import precond as opc
    from oracle import solvers as osv
    from oracle.operator import Plan as OPlan
    f = make_rhs(seed)
    op = OPlan(2, N_SIDE, 1.0 / (N_SIDE + 1), alpha)
    op.kernel_hat()                       # operator construction, untimed
    prec = (lambda r, op=op: opc.solve_box(op, r)) if alpha >= 1.0 else None
    t0 = time.perf_counter()
    _, its, ok, _ = osv.pcg(op.apply, f, prec, None, TOL, 4000)
    dt = time.perf_counter() - t0
    assert ok
    return dt, its


def oracle_warm():
    """One oracle CG iteration (primes scipy's FFT plans; untimed)."""
    from oracle import solvers as osv
    from oracle.operator import Plan as OPlan
    op = OPlan(2, N_SIDE, 1.0 / (N_SIDE + 1), 1.0)
    osv.pcg(op.apply, make_rhs(0), None, None, 1e-30, 1)


def profile_case():
    """The workload's alpha = 1.5 solve, twice (the second is the captured one)."""
    import torch
    from paper_1802_03770_gb300 import _lib
    from paper_1802_03770_gb300.api import Plan
    p = Plan(2, (N_SIDE, N_SIDE), 1.0 / (N_SIDE + 1), 1.5)
    f = torch.tensor(make_rhs(0), dtype=torch.float64, device="cuda:0").view(-1)
    for _ in range(2):
        u, info = p.solve(f, tol=TOL, mode=_lib.FL_MODE_MIXED | _lib.FL_PRECOND_AUTO)
    torch.cuda.synchronize()
    print(json.dumps(info))


def profile_case_unet(n=512, reps=20):
    """U-Net forwards of the learned preconditioner at 512^2 (seeded weights
    and features): five on the tensor cores (the ncu captures take their
    tcgen05 3x3 convolutions), then `reps` timed forwards (CUDA events) on
    the tensor cores and on the CUDA cores."""
    import torch
    from paper_1802_03770_gb300.api import Net
    net = Net(n, n, seed=1)
    g = torch.Generator().manual_seed(5)
    x = torch.randn(3 * n * n, generator=g).to("cuda:0")
    out = {}
    for tc in (True, False):
        net.tensor_cores(tc)
        for _ in range(5):
            y = net.forward(x)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            y = net.forward(x)
        e1.record()
        torch.cuda.synchronize()
        out["tcgen05" if tc else "cuda_cores"] = {"ms_per_forward": e0.elapsed_time(e1) / reps,
                                                  "y_norm": float(y.norm())}
    print(json.dumps({"unet512_forward": out}))


def profile_case_3d(n=256):
    """Five FP32 applies on the 3D time-step grid (n^3 interior, (2n)^3 padded
    FFT), from a seeded field; the passes of the first are the captured ones."""
    import torch
    from paper_1802_03770_gb300 import inputs
    from paper_1802_03770_gb300.api import Plan
    p = Plan(3, (n, n, n), 1.0 / (n + 1), 1.5)
    x = torch.tensor(inputs.gaussian_mixture(n, 3, 16, 3, 0.05, 0.15), dtype=torch.float32,
                     device="cuda:0").view(-1)
    y = torch.empty_like(x)
    for _ in range(5):
        p.apply(x, y)
    torch.cuda.synchronize()
    print(json.dumps({"n": n, "y_norm": float(y.norm())}))
    p.close()


def cores_used():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-preconditioner arm")
    ap.add_argument("--no-3d", action="store_true", help="skip the 3D 256^3 time-step entry")
    ap.add_argument("--no-batch64", action="store_true", help="skip the 64-problem batch entry")
    ap.add_argument("--profile-case", action="store_true",
                    help="run two mixed solves at alpha = 1.5 and exit (for ncu captures)")
    ap.add_argument("--profile-case-3d", action="store_true",
                    help="run five FP32 applies on the 256^3 grid and exit (for ncu captures)")
    ap.add_argument("--profile-case-unet", action="store_true",
                    help="time 512^2 U-Net forwards (tensor cores, CUDA cores) and exit")
    args = ap.parse_args()
    if args.profile_case:
        profile_case()
        return
    if args.profile_case_3d:
        profile_case_3d()
        return
    if args.profile_case_unet:
        profile_case_unet()
        return
    rank, world, local = dist_env()
    config = {"workload": WORKLOAD, "n": N_SIDE, "fft_len": 2 * N_SIDE, "alphas": list(ALPHAS),
              "tol": TOL, "l2": "flushed between timed steps (512 MB write)",
              "parallelism": f"replicas x{world} (independent seeds per rank)"}
    if args.impl == "reference":
        # the FP64 oracle on the host cores: every timed step is one full
        # solve (alpha cycling through the workload's three, right-hand sides
        # of the GPU arm's timed steps); warm-up steps run one oracle CG
        # iteration each (they prime scipy's FFT plans)
        if rank != 0:
            return
        import scipy.fft
        cores = cores_used()
        for _ in range(args.warmup):
            with scipy.fft.set_workers(cores):
                oracle_warm()
        total_s, its = 0.0, []
        for k in range(args.steps):
            j = k % len(ALPHAS)
            with scipy.fft.set_workers(cores):
                dt, it = oracle_solve(ALPHAS[j], rhs_seed(0, args.warmup + k // len(ALPHAS), j))
            total_s += dt
            its.append(it)
        value = args.steps / total_s
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": total_s / args.steps * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": config,
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                                 "sample": f"{args.steps} full FP64 oracle solves of the 1024^2 "
                                           "workload to 1e-8 (one per step, alpha cycling through "
                                           "0.5, 1, 1.5; the GPU arm's timed right-hand sides), "
                                           "measured; FFTs on all host cores (scipy.fft workers), "
                                           "vector updates on one; warm-up steps run one oracle "
                                           "CG iteration each",
                                 "iterations": its},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    res = run_ours(args, rank, world, local)
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            import scipy.fft
            cores = cores_used()
            secs, its = [], []
            for j, a in enumerate(ALPHAS):
                with scipy.fft.set_workers(cores):
                    dt, it = oracle_solve(a, rhs_seed(0, args.warmup, j))
                secs.append(dt)
                its.append(it)
            cpu = {"value": len(ALPHAS) / sum(secs), "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": "one full FP64 oracle solve per alpha of the 1024^2 workload to 1e-8 "
                             "(the right-hand sides of the first timed step), measured; FFTs on all "
                             "host cores (scipy.fft workers), vector updates on one",
                   "seconds": secs, "iterations": its}
        line = {"metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64", "data": "synthetic", "config": config,
                "clocks": res["clocks"], "e2e": res["e2e"], "gpu_launches": res["gpu_launches"],
                "roofline": res["roofline"], "cpu_baseline": cpu,
                "fp64_pcg": res["fp64_pcg"], "speedup_vs_fp64_pcg": res["speedup_vs_fp64_pcg"],
                "batched": res["batched"], "balanced_shift": res["balanced_shift"],
                "iterations_mixed": res["iterations_mixed"], "refinements": res["refinements"],
                "mixed_error_vs_fp64": res["mixed_error_vs_fp64"],
                "t_con_s": res["t_con_s"], "apply": res["apply"], "kernels": res["kernels"],
                "tiles": res["tiles"], "learned": res["learned"],
                "timestep_3d": res["timestep_3d"], "batched_64": res["batched_64"]}
        print(json.dumps(line))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
