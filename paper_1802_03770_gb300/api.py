"""Thin Python API over the C ABI, for torch CUDA tensors.

Each method marshals tensor pointers, sizes and the current torch CUDA
stream into the matching ``fl_*`` call; all arithmetic happens in
``libfraclap.so``.
"""

import ctypes

import numpy as np

from . import _lib as L


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _check_tensor(t, dtype, numel, what):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{what} must have dtype {dtype}")
    if t.numel() != numel or not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous with {numel} elements")


def launch_count():
    """Kernels launched by libfraclap.so in this process so far."""
    return int(L.load().fl_launch_count())


def read_gate(path):
    """(lo, hi, enabled flags) of a gate file: comment lines start with '#',
    then a line "lo hi bands" and a line of `bands` 0/1 flags."""
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.lstrip().startswith("#")]
    lo, hi, bands = float(rows[0][0]), float(rows[0][1]), int(rows[0][2])
    flags = [int(v) for v in rows[1]]
    if len(flags) != bands:
        raise ValueError(f"{path}: {len(flags)} flags for {bands} bands")
    return lo, hi, flags


class Net:
    """The U-Net of the learned preconditioner (fl_net_*); H, W multiples of 64."""

    def __init__(self, H, W, seed=0, stream=None):
        import torch
        self._lib = L.load()
        if stream is None:
            stream = torch.cuda.current_stream()
        h = ctypes.c_void_p()
        L.check(self._lib.fl_net_create(int(H), int(W), int(seed), ctypes.c_void_p(stream.cuda_stream),
                                        ctypes.byref(h)), "fl_net_create")
        self._h, self.H, self.W = h, int(H), int(W)
        self.nparams = int(self._lib.fl_net_num_params(h))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.fl_net_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def tensor_cores(self, enable=True):
        L.check(self._lib.fl_net_set_tensor_cores(self._h, int(enable)), "fl_net_set_tensor_cores")

    def check(self):
        L.check(self._lib.fl_net_check(self._h), "fl_net_check")

    def set_alpha_gate(self, lo=0.0, hi=0.0, enabled=()):
        """FL_MODE_LEARNED uses the network only for alpha in [lo, hi) in an
        enabled band (len(enabled) equal bands); no bands = no gate."""
        flags = np.ascontiguousarray([1 if e else 0 for e in enabled], dtype=np.uint8)
        L.check(self._lib.fl_net_set_alpha_gate(self._h, float(lo), float(hi), int(flags.size),
                                                flags.ctypes.data_as(ctypes.c_void_p) if flags.size else None),
                "fl_net_set_alpha_gate")

    def load_gate(self, path):
        """Set the alpha gate from a gate file written by learned.write_gate."""
        lo, hi, flags = read_gate(path)
        self.set_alpha_gate(lo, hi, flags)

    def get_params(self, grads=False):
        p = np.empty(self.nparams, np.float32)
        g = np.empty(self.nparams, np.float32) if grads else None
        L.check(self._lib.fl_net_get_params(self._h, p.ctypes.data_as(ctypes.c_void_p),
                                            g.ctypes.data_as(ctypes.c_void_p) if grads else None),
                "fl_net_get_params")
        return (p, g) if grads else p

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        if p.size != self.nparams:
            raise ValueError("wrong parameter count")
        L.check(self._lib.fl_net_set_params(self._h, p.ctypes.data_as(ctypes.c_void_p)),
                "fl_net_set_params")

    # channels and level (resolution H >> level) of tensor index 0..11
    TENSORS = ((3, 0), (16, 0), (16, 0), (32, 1), (32, 1), (64, 2), (64, 2), (32, 1), (32, 1),
               (16, 0), (16, 0), (1, 0))

    def get_tensor(self, index, grad=False):
        """Activation (or its loss gradient) `index` of the last call, as a
        float32 array [channels, H >> level, W >> level]."""
        c, lev = self.TENSORS[index]
        shape = (c, self.H >> lev, self.W >> lev)
        out = np.empty(shape, np.float32)
        L.check(self._lib.fl_net_get_tensor(self._h, int(bool(grad)), int(index),
                                            out.ctypes.data_as(ctypes.c_void_p), out.size),
                "fl_net_get_tensor")
        return out

    def forward(self, x):
        import torch
        _check_tensor(x, torch.float32, 3 * self.H * self.W, "x")
        y = torch.empty(self.H * self.W, dtype=torch.float32, device=x.device)
        L.check(self._lib.fl_net_forward(self._h, _ptr(x), _ptr(y)), "fl_net_forward")
        return y

    def loss_grad(self, xs, ts):
        import torch
        b = xs.shape[0]
        _check_tensor(xs, torch.float32, b * 3 * self.H * self.W, "xs")
        _check_tensor(ts, torch.float32, b * self.H * self.W, "ts")
        loss = ctypes.c_double()
        L.check(self._lib.fl_net_loss_grad(self._h, _ptr(xs), _ptr(ts), int(b), ctypes.byref(loss)),
                "fl_net_loss_grad")
        return loss.value

    def train_step(self, xs, ts, lr=1e-3):
        import torch
        b = xs.shape[0]
        _check_tensor(xs, torch.float32, b * 3 * self.H * self.W, "xs")
        _check_tensor(ts, torch.float32, b * self.H * self.W, "ts")
        loss = ctypes.c_double()
        L.check(self._lib.fl_net_train_step(self._h, _ptr(xs), _ptr(ts), int(b), float(lr),
                                            ctypes.byref(loss)), "fl_net_train_step")
        return loss.value

    def save(self, path):
        L.check(self._lib.fl_net_save(self._h, str(path).encode()), "fl_net_save")

    def load(self, path):
        L.check(self._lib.fl_net_load(self._h, str(path).encode()), "fl_net_load")


def solve_batched(plans, fs, tol=1e-8, maxit=1000, mode=L.FL_MODE_MIXED | L.FL_PRECOND_AUTO,
                  raise_on_fail=True):
    """fl_solve_elliptic_batched over lists of plans and float64 CUDA tensors;
    returns (solutions, list of info dicts)."""
    import torch
    n = len(plans)
    us = []
    for p, f in zip(plans, fs):
        _check_tensor(f, torch.float64, p.N, "f")
        us.append(torch.empty_like(f))
    hp = (ctypes.c_void_p * n)(*[p._h.value for p in plans])
    fp = (ctypes.c_void_p * n)(*[f.data_ptr() for f in fs])
    up = (ctypes.c_void_p * n)(*[u.data_ptr() for u in us])
    infos = (L.FlSolveInfo * n)()
    st = L.load().fl_solve_elliptic_batched(hp, n, fp, up, float(tol), int(maxit), int(mode), infos)
    if raise_on_fail:
        L.check(st, "fl_solve_elliptic_batched")
    return us, [infos[i].as_dict() for i in range(n)]


class Plan:
    """Operator plan: fl_plan_create(d, n, h, alpha, mask) on the current
    device and torch stream (or the given one)."""

    def __init__(self, d, n, h, alpha, mask=None, rho=0.0, stream=None, inner_tol=0.0,
                 max_outer=0):
        import torch
        lib = L.load()
        n = [int(v) for v in np.broadcast_to(np.asarray(n), (d,))]
        self.d, self.n = d, tuple(n)
        self.N = int(np.prod(n))
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        opts = L.FlOpts(float(rho), ctypes.c_void_p(stream.cuda_stream), float(inner_tol),
                        int(max_outer))
        narr = (ctypes.c_int64 * d)(*n)
        mptr = None
        if mask is not None:
            m = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8).reshape(-1))
            if m.size != self.N:
                raise ValueError("mask must have prod(n) entries")
            self._mask = m
            mptr = m.ctypes.data_as(ctypes.c_void_p)
        handle = ctypes.c_void_p()
        L.check(lib.fl_plan_create(int(d), narr, float(h), float(alpha), mptr,
                                   ctypes.byref(opts), ctypes.byref(handle)), "fl_plan_create")
        self._h = handle
        self._lib = lib

    def close(self):
        if getattr(self, "_h", None):
            self._lib.fl_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def describe(self):
        d = L.FlPlanDesc()
        L.check(self._lib.fl_plan_describe(self._h, ctypes.byref(d)), "fl_plan_describe")
        return {"d": d.d, "n": tuple(d.n[: d.d]), "fft_len": tuple(d.fft_len[: d.d]),
                "h": d.h, "alpha": d.alpha, "rho": d.rho, "c_alpha_d": d.c_alpha_d,
                "lattice_zeta": d.lattice_zeta, "window_corr": d.window_corr,
                "kernel0": d.kernel0, "workspace_bytes": d.workspace_bytes}

    # -- operator ------------------------------------------------------------
    def apply(self, u, out=None):
        import torch
        f32 = u.dtype == torch.float32
        dt = torch.float32 if f32 else torch.float64
        _check_tensor(u, dt, self.N, "u")
        y = torch.empty_like(u) if out is None else out
        _check_tensor(y, dt, self.N, "out")
        fn = self._lib.fl_apply_f32 if f32 else self._lib.fl_apply
        L.check(fn(self._h, _ptr(u), _ptr(y)), "fl_apply")
        return y

    def precond(self, r, shift=0.0, scale=1.0, out=None):
        import torch
        f32 = r.dtype == torch.float32
        dt = torch.float32 if f32 else torch.float64
        _check_tensor(r, dt, self.N, "r")
        z = torch.empty_like(r) if out is None else out
        _check_tensor(z, dt, self.N, "out")
        fn = self._lib.fl_precond_f32 if f32 else self._lib.fl_precond
        L.check(fn(self._h, float(shift), float(scale), _ptr(r), _ptr(z)), "fl_precond")
        return z

    def set_tiles(self, tx):
        """Column-tile widths of the strided passes: six ints (FP32 axes 0..2,
        FP64 axes 0..2; 0 = the widest tile)."""
        arr = (ctypes.c_int * 6)(*[int(v) for v in tx])
        L.check(self._lib.fl_plan_set_tiles(self._h, arr), "fl_plan_set_tiles")

    def autotune(self):
        """Time the candidate column tiles on the GPU and keep the fastest;
        returns the six chosen widths (0 for axes without a strided pass)."""
        arr = (ctypes.c_int * 6)()
        L.check(self._lib.fl_plan_autotune(self._h, arr), "fl_plan_autotune")
        return list(arr)

    def set_row_shape(self, shape):
        """CTA shape of the FP32 row passes: 0 = 128 x 16, 1 = 256 x 8."""
        L.check(self._lib.fl_plan_set_row_shape(self._h, int(shape)), "fl_plan_set_row_shape")

    def row_shape(self):
        return int(self._lib.fl_plan_row_shape(self._h))

    def precond_params(self, mode, shift=0.0, scale=1.0):
        """(pshift, pscale) of the preconditioner (pshift I + pscale C h^d L)^-1
        that a solve in `mode` uses for shift I + scale M; (0, 0) for none."""
        ps, sc = ctypes.c_double(), ctypes.c_double()
        L.check(self._lib.fl_precond_params(self._h, int(mode), float(shift), float(scale),
                                            ctypes.byref(ps), ctypes.byref(sc)), "fl_precond_params")
        return ps.value, sc.value

    # -- solves ----------------------------------------------------------------
    def solve(self, f, u=None, tol=1e-8, maxit=1000, mode=L.FL_MODE_MIXED, raise_on_fail=True):
        """Solve M u = f; returns (u, info dict)."""
        import torch
        _check_tensor(f, torch.float64, self.N, "f")
        x0 = u is not None
        if u is None:
            u = torch.zeros_like(f)
        _check_tensor(u, torch.float64, self.N, "u")
        info = L.FlSolveInfo()
        st = self._lib.fl_solve_elliptic(self._h, _ptr(f), _ptr(u), int(x0), float(tol),
                                         int(maxit), int(mode), ctypes.byref(info))
        if raise_on_fail:
            L.check(st, "fl_solve_elliptic")
        return u, info.as_dict()

    def solve_host(self, f, tol=1e-8, maxit=1000, mode=L.FL_MODE_MIXED):
        """The same solve on host arrays (numpy float64, C order)."""
        f = np.ascontiguousarray(f, dtype=np.float64)
        if f.size != self.N:
            raise ValueError("f must have prod(n) entries")
        u = np.empty_like(f)
        info = L.FlSolveInfo()
        st = self._lib.fl_solve_elliptic_host(self._h, f.ctypes.data_as(ctypes.c_void_p),
                                              u.ctypes.data_as(ctypes.c_void_p), float(tol),
                                              int(maxit), int(mode), ctypes.byref(info))
        L.check(st, "fl_solve_elliptic_host")
        return u, info.as_dict()

    def time_step(self, u_prev, dt, theta=1.0, f_prev=None, f_next=None, out=None, tol=1e-8,
                  maxit=1000, mode=L.FL_MODE_MIXED):
        import torch
        _check_tensor(u_prev, torch.float64, self.N, "u_prev")
        u_next = torch.empty_like(u_prev) if out is None else out
        info = L.FlSolveInfo()
        fp = _ptr(f_prev) if f_prev is not None else None
        fn = _ptr(f_next) if f_next is not None else None
        st = self._lib.fl_time_step(self._h, float(dt), float(theta), _ptr(u_prev), fp, fn,
                                    _ptr(u_next), float(tol), int(maxit), int(mode),
                                    ctypes.byref(info))
        L.check(st, "fl_time_step")
        return u_next, info.as_dict()

    def training_pair(self, f, u_star, x):
        """fl_net_training_pair: features [3, N] and target [N] (float32 CUDA
        tensors) of the pair (r = f - M x, e = u* - x)."""
        import torch
        for t, name in ((f, "f"), (u_star, "u_star"), (x, "x")):
            _check_tensor(t, torch.float64, self.N, name)
        feat = torch.empty(3 * self.N, dtype=torch.float32, device=f.device)
        target = torch.empty(self.N, dtype=torch.float32, device=f.device)
        L.check(self._lib.fl_net_training_pair(self._h, _ptr(f), _ptr(u_star), _ptr(x), _ptr(feat),
                                               _ptr(target)), "fl_net_training_pair")
        return feat.view(3, self.N), target

    def attach_net(self, net):
        """Use `net` (api.Net, or None to detach) for FL_MODE_LEARNED solves."""
        L.check(self._lib.fl_plan_attach_net(self._h, net._h if net is not None else None),
                "fl_plan_attach_net")
        self._net = net

    def profile(self, enable=True):
        L.check(self._lib.fl_profile_enable(self._h, int(enable)), "fl_profile_enable")

    def profile_read(self):
        """{kernel name: (launches, total ms)} since profiling was enabled."""
        buf = (L.FlKernelStat * 64)()
        n = self._lib.fl_profile_read(self._h, buf, 64)
        return {buf[i].name.decode(): (buf[i].launches, buf[i].total_ms) for i in range(min(n, 64))}

    def sync(self):
        L.check(self._lib.fl_sync(self._h), "fl_sync")
