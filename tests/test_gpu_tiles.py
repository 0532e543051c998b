"""Column tiles of the strided passes and the FP32 row-pass shape
(fl_plan_set_tiles, fl_plan_set_row_shape, fl_plan_autotune).

Each line of a strided pass is transformed by the same arithmetic whatever
the tile width, so every width must give bit-identical applies and
preconditioner solves (FP32 and FP64); the second row-pass shape (256 x 8,
radix-8 stages) must agree with the oracle to FP32 rounding; the tuner must
return widths in range, and solves after it must still converge (it
discards the plan's captured CG graphs)."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.operator import Plan as OPlan  # noqa: E402
from paper_1802_03770_gb300 import _lib, inputs  # noqa: E402
from paper_1802_03770_gb300.api import Plan  # noqa: E402

DEV = "cuda:0"


def widths(L, f32):
    """Candidate widths of a strided pass along an axis of padded length L:
    the widest tile of a CTA (8192 FP32 / 4096 FP64 complex values, <= 64)
    halved down to 16 bytes of line element."""
    w = min(64, (8192 if f32 else 4096) // L)
    out = []
    while w >= (2 if f32 else 1):
        out.append(w)
        w //= 2
    return out


def outputs(p, fields):
    u32, u64, r32, r64 = fields
    res = [p.apply(u32), p.apply(u64), p.precond(r32), p.precond(r64),
           p.precond(r32, 1.0, 0.01), p.precond(r64, 1.0, 0.01)]
    torch.cuda.synchronize()
    return res


def _fields(N, seed):
    g = torch.Generator(device="cpu").manual_seed(seed)
    u = torch.randn(N, generator=g, dtype=torch.float64)
    r = torch.randn(N, generator=g, dtype=torch.float64)
    return (u.float().to(DEV), u.to(DEV), r.float().to(DEV), r.to(DEV))


def _l_shape(n):
    m = np.ones(n, bool)
    m[n[0] // 2:, n[1] // 2:] = False
    return m


@pytest.mark.parametrize("d,n,alpha,masked", [
    (2, (300, 257), 1.3, False),
    (2, (130, 97), 0.7, True),
    (3, (40, 33, 24), 0.8, False),
])
def test_every_tile_width_gives_identical_results(d, n, alpha, masked):
    mask = _l_shape(n) if masked else None
    p = Plan(d, n, 1.0 / (max(n) + 1), alpha, mask=mask)
    fields = _fields(int(np.prod(n)), 5)
    ref = outputs(p, fields)
    L = p.describe()["fft_len"]
    axes = [0] if d == 2 else [0, 1]
    w32 = [widths(L[a], True) for a in axes]
    w64 = [widths(L[a], False) for a in axes]
    k = max(len(w) for w in w32 + w64)
    for i in range(k):
        tx = [0] * 6
        for j, a in enumerate(axes):
            tx[a] = w32[j][min(i, len(w32[j]) - 1)]
            tx[3 + a] = w64[j][min(i, len(w64[j]) - 1)]
        p.set_tiles(tx)
        got = outputs(p, fields)
        for a, b in zip(got, ref):
            assert torch.equal(a, b), tx
    p.set_tiles([0] * 6)


def test_set_tiles_rejects_bad_widths():
    p = Plan(2, (300, 257), 1.0 / 301, 1.3)     # axis 0: L = 1024, FP32 8..2, FP64 4..1
    for tx in ([3, 0, 0, 0, 0, 0], [16, 0, 0, 0, 0, 0], [1, 0, 0, 0, 0, 0], [0, 0, 0, 8, 0, 0]):
        with pytest.raises(RuntimeError):
            p.set_tiles(tx)
    p.set_tiles([2, 0, 0, 1, 0, 0])
    p.set_tiles([8, 5, 7, 4, 9, 9])             # axes 1, 2 have no strided pass: ignored


@pytest.mark.parametrize("d,n", [(2, (255, 255)), (3, (48, 40, 32))])
def test_autotune_keeps_results_and_solves(d, n):
    h = 1.0 / (max(n) + 1)
    p = Plan(d, n, h, 1.25)
    fields = _fields(int(np.prod(n)), 9)
    ref = outputs(p, fields)
    f = torch.tensor(inputs.gaussian_mixture(max(n), d, 8, 2)[tuple(slice(0, m) for m in n)],
                     dtype=torch.float64, device=DEV).reshape(-1).contiguous()
    _, info0 = p.solve(f, tol=1e-9)               # captures the CG graphs
    tx = p.autotune()
    L = p.describe()["fft_len"]
    axes = [0] if d == 2 else [0, 1]
    for a in range(3):
        if a in axes:
            assert tx[a] in widths(L[a], True) and tx[3 + a] in widths(L[a], False)
        else:
            assert tx[a] == 0 and tx[3 + a] == 0
    # the column widths alone change no result: compare bit for bit in the
    # default row shape (the tuned row shape agrees to FP32 rounding only,
    # test_row_shape_256x8_matches_oracle), then solve in the tuned shape
    shape = p.row_shape()
    assert shape in (0, 1)
    p.set_row_shape(0)
    got = outputs(p, fields)
    for a, b in zip(got, ref):
        assert torch.equal(a, b)
    p.set_row_shape(shape)
    u, info = p.solve(f, tol=1e-9)
    assert info["converged"] == 1
    assert abs(info["iterations"] - info0["iterations"]) <= (0 if shape == 0 else 2)
    op = OPlan(d, n, h, 1.25)
    fh = f.cpu().numpy().reshape(n)
    res = op.apply(u.cpu().numpy().reshape(n)) - fh
    assert np.linalg.norm(res) <= 1.05e-9 * np.linalg.norm(fh)
    print(f"{d}D {n}: tuned column tiles {tx}, row shape {shape}")


@pytest.mark.parametrize("n", [(96, 96), (200, 130), (1024, 1024)])
def test_row_shape_256x8_matches_oracle(n):
    """The FP32 row passes in the 256 x 8 CTA shape (radix-8 stages): apply
    and FD preconditioner solve within the FP32 tolerance (2e-5) of the FP64
    oracle, and a mixed solve to 1e-8 in the oracle's residual."""
    from oracle import precond as oprec
    h = 1.0 / (max(n) + 1)
    alpha = 1.3
    p = Plan(2, n, h, alpha)
    p.set_row_shape(1)
    assert p.row_shape() == 1
    op = OPlan(2, n, h, alpha)
    rng = np.random.default_rng(81)
    u = rng.standard_normal(n).astype(np.float32).astype(np.float64)
    y = p.apply(torch.tensor(u.ravel(), dtype=torch.float32, device=DEV)).cpu().numpy()
    ref = op.apply(u).ravel()
    assert np.linalg.norm(y - ref) <= 2e-5 * np.linalg.norm(ref)
    z = p.precond(torch.tensor(u.ravel(), dtype=torch.float32, device=DEV)).cpu().numpy()
    zref = oprec.solve_box(op, u).ravel()
    assert np.linalg.norm(z - zref) <= 2e-5 * np.linalg.norm(zref)
    f = inputs.gaussian_mixture(n, 2, 16, 82)
    us, info = p.solve(torch.tensor(f, dtype=torch.float64, device=DEV).view(-1), tol=1e-8,
                       mode=_lib.FL_MODE_MIXED | _lib.FL_PRECOND_FD)
    assert info["converged"] == 1, info
    res = np.linalg.norm(op.apply(us.cpu().numpy().reshape(n)) - f) / np.linalg.norm(f)
    assert res <= 1.05e-8, res


def test_row_shape_rejected_outside_its_lengths_and_tuned():
    p = Plan(2, (50, 50), 1.0 / 51, 1.0)               # rows pad to 128 points
    with pytest.raises(_lib.FracLapError, match="INVALID_ARG"):
        p.set_row_shape(1)
    with pytest.raises(_lib.FracLapError, match="INVALID_ARG"):
        p.set_row_shape(2)
    q = Plan(2, (160, 160), 1.0 / 161, 1.0)             # rows pad to 512 points
    q.autotune()
    assert q.row_shape() in (0, 1)
    f = inputs.gaussian_mixture(160, 2, 16, 83)
    _, info = q.solve(torch.tensor(f, dtype=torch.float64, device=DEV).view(-1), tol=1e-8,
                      mode=_lib.FL_MODE_MIXED | _lib.FL_PRECOND_FD)
    assert info["converged"] == 1, info
