"""GPU parity for partitions whose blocks are arbitrary row sets (apc_setup_rows)
on a tall system (N > n), against the oracle's ``partition_rows``."""
import numpy as np
import pytest

from oracle import apc_oracle as O
from paper_1708_01413_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _apc():
    from paper_1708_01413_gb300 import apc, build
    build.build()
    return apc


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch.device("cuda:0")


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _case(seed=51, n=200, N=450):
    A, x_true, b = inputs.gaussian_system(n, seed, N=N)
    rng = np.random.default_rng(seed)
    perm = rng.permutation(N)
    cuts = np.sort(rng.choice(np.arange(20, N - 20), size=5, replace=False))
    sets = np.split(perm, cuts)  # 6 uneven, scattered row sets
    blocks = O.partition_rows(A, b, sets)
    QR = [O.block_qr(Ai) for Ai, _ in blocks]
    Qs, Rs = [q for q, _ in QR], [r for _, r in QR]
    g, e, _ = O.optimal_params(*O.mu_bounds(Qs))
    return A, x_true, b, sets, blocks, Qs, Rs, g, e


def _oracle_run(blocks, Qs, Rs, g, e, T):
    xs = [O.least_norm_init(Q, R, bi) for Q, R, (_, bi) in zip(Qs, Rs, blocks)]
    xbar = sum(xs) / len(xs)
    for _ in range(T):
        xs, xbar = O.apc_step(xs, xbar, Qs, g, e)
    return xbar


def test_row_sets_trajectory_residual_and_reset_match_oracle():
    apc, dev = _apc(), _dev()
    A, x_true, b, sets, blocks, Qs, Rs, g, e = _case()
    ctx = apc.apc_setup_rows(torch.tensor(A, device=dev), torch.tensor(b, device=dev), sets, precision="f64")
    T = 150
    ctx.reset()
    ctx.iterate(g, e, T)
    xb = ctx.xbar().cpu().numpy()
    assert _rel(xb, _oracle_run(blocks, Qs, Rs, g, e, T)) <= 1e-10
    # residual vector and right-hand side in the caller's row order
    b2 = np.random.default_rng(3).standard_normal(A.shape[0])
    r_out = torch.empty(A.shape[0], dtype=torch.float64, device=dev)
    rel = ctx.residual(torch.tensor(xb, device=dev), torch.tensor(b2, device=dev), r_out)
    want = b2 - A @ xb
    assert np.allclose(r_out.cpu().numpy(), want, rtol=0, atol=1e-10 * np.abs(want).max())
    assert rel == pytest.approx(np.linalg.norm(want) / np.linalg.norm(b2), rel=1e-10)
    # a new right-hand side through reset (caller's order)
    ctx.reset(torch.tensor(b2, device=dev))
    ctx.iterate(g, e, T)
    blocks2 = O.partition_rows(A, b2, sets)
    assert _rel(ctx.xbar().cpu().numpy(), _oracle_run(blocks2, Qs, Rs, g, e, T)) <= 1e-10


def test_row_sets_solve_and_backward_order():
    apc, dev = _apc(), _dev()
    A, x_true, b, sets, blocks, Qs, Rs, g, e = _case(seed=52)
    ctx = apc.apc_setup_rows(torch.tensor(A, device=dev), torch.tensor(b, device=dev), sets, precision="f64")
    x, st = ctx.solve(g, e, tol=1e-10, max_iters=500000, check_every=200)
    assert O.relative_residual(A, b, x.cpu().numpy()) <= 1e-10
    # dL/db comes back in the caller's row order
    T = 40
    gT = np.random.default_rng(7).standard_normal(A.shape[1])
    db = ctx.backward(torch.tensor(gT, device=dev), T, g, e).cpu().numpy()
    per_block = O.apc_adjoint(blocks, Qs, Rs, g, e, T, gT)[0]
    ref = np.zeros(A.shape[0])
    for r, d in zip(sets, per_block):
        ref[r] = d
    assert _rel(db, ref) <= 1e-10


def test_row_sets_must_be_a_permutation():
    apc, dev = _apc(), _dev()
    A, _, b = inputs.gaussian_system(40, 53, N=60)
    with pytest.raises(apc.ApcError) as ei:
        apc.apc_setup_rows(torch.tensor(A, device=dev), torch.tensor(b, device=dev),
                           [np.arange(0, 30), np.arange(29, 59)])
    assert ei.value.name == "INVALID_ARG"
