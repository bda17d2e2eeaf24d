"""The free residual monitor (apc_monitor) against the FP64 residual, and
apc_solve's use of it, through the C ABI.

Every x_i solves its block (App. A), so block i's residual of xbar is
D_i^{-1} R_i'^T Q_i^T (xbar - x_i), from the coefficients the iteration kernel
keeps for its next pass.  Its error is set by the stored bases and by z: the
FP32 products of n terms leave about sqrt(n) u ||xbar - x_i|| in z, a few 1e-6
of ||b|| at these sizes, and FP64 about 1e-13."""
import numpy as np
import pytest

from oracle import apc_oracle as O
from paper_1708_01413_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _env():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1708_01413_gb300 import apc, build
    build.build()
    return apc, torch.device("cuda:0")


@pytest.mark.parametrize("prec,rtol,atol", [("f64", 1e-8, 1e-13), ("f32", 1e-2, 1e-5)])
def test_monitor_tracks_fp64_residual(prec, rtol, atol):
    apc, dev = _env()
    n, N, m = 1536, 1728, 9  # tall system, blocks of 192 rows
    A, _, b = inputs.gaussian_system(n, 81, N=N)
    offs = inputs.even_offsets(N, m)
    bl = O.partition(A, b, offs)
    lo, hi = O.mu_bounds([O.block_qr(Ai)[0] for Ai, _ in bl])
    g, e, _ = O.optimal_params(lo, hi)
    ctx = apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(b, device=dev), offs, precision=prec)
    r2 = torch.tensor(np.random.default_rng(3).standard_normal(N), device=dev)
    seen = []
    for rhs in (None, r2):  # the stored b, then another right-hand side (as in refinement sweeps)
        ctx.reset(rhs)
        for k in (0, 1, 10, 50, 200, 400):
            if k:
                ctx.iterate(g, e, k)
            mon = ctx.monitor()
            res = ctx.residual(ctx.xbar(), rhs=rhs)
            assert abs(mon - res) <= rtol * res + atol, (prec, k, mon, res)
            seen.append(res)
    assert min(seen) < 1e-2 * max(seen)  # the checks spanned a real decrease of the residual


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
def test_solve_checks_with_the_monitor(prec):
    # FP32/FP64: checks by the monitor, an FP64 residual only to confirm;
    # BF16: FP64 residuals; every mode ends on an FP64 residual below tol
    apc, dev = _env()
    n, N, m = 1024, 1152, 9
    A, _, b = inputs.gaussian_system(n, 82, N=N)
    offs = inputs.even_offsets(N, m)
    bl = O.partition(A, b, offs)
    lo, hi = O.mu_bounds([O.block_qr(Ai)[0] for Ai, _ in bl])
    g, e, _ = O.optimal_params(lo, hi)
    ctx = apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(b, device=dev), offs, precision=prec)
    tol = 1e-10 if prec == "f64" else 1e-9
    x, st = ctx.solve(g, e, tol=tol, max_iters=200000, check_every=20, refine=prec != "f64")
    assert O.relative_residual(A, b, x.cpu().numpy()) <= tol
    if prec == "bf16":
        assert st["monitor_checks"] == 0
    else:
        assert st["monitor_checks"] > 0
        assert st["residual_checks"] < st["monitor_checks"]


def test_solve_rhs_solves_every_column_and_keeps_b():
    # k right-hand sides through apc_solve_rhs (columns of a wider matrix),
    # each to 1e-10 with FP32 + refinement; the context's own b is unchanged
    apc, dev = _env()
    n, N, m, k = 768, 864, 9, 3
    A, _, b = inputs.gaussian_system(n, 83, N=N)
    offs = inputs.even_offsets(N, m)
    bl = O.partition(A, b, offs)
    g, e, _ = O.optimal_params(*O.mu_bounds([O.block_qr(Ai)[0] for Ai, _ in bl]))
    Bw = A @ np.random.default_rng(9).standard_normal((n, k + 2))  # consistent: the system is tall
    ctx = apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(b, device=dev), offs, precision="f32")
    X, st = ctx.solve_rhs(torch.tensor(Bw, device=dev)[:, :k], g, e, tol=1e-10, max_iters=400000, check_every=20,
                          refine=True)
    Xh = X.cpu().numpy()
    for j in range(k):
        assert O.relative_residual(A, Bw[:, j], Xh[:, j]) <= 1e-10
    assert st["rel_residual"] <= 1e-10
    x, _ = ctx.solve(g, e, tol=1e-10, max_iters=400000, check_every=20, refine=True)
    assert O.relative_residual(A, b, x.cpu().numpy()) <= 1e-10


def test_monitor_needs_a_forward_state():
    # after a reverse sweep the state holds adjoints: the monitor refuses
    apc, dev = _env()
    A, _, b = inputs.gaussian_system(128, 84)
    offs = inputs.even_offsets(128, 4)
    ctx = apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(b, device=dev), offs, precision="f64")
    ctx.backward(torch.ones(128, dtype=torch.float64, device=dev), 3, 1.0, 1.5)
    with pytest.raises(apc.ApcError) as ei:
        ctx.monitor()
    assert ei.value.name == "INVALID_ARG"
    ctx.reset()
    assert ctx.monitor() == pytest.approx(ctx.residual(ctx.xbar()), rel=1e-8, abs=1e-13)
