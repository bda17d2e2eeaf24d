"""k right-hand sides in one call (apc_forward_rhs / apc_backward_rhs) and the
batched reverse sweep (apc_batch_backward), through the C ABI, against the
FP64 oracle.

The tensor-core form (BF16 context, square system, 2 <= k <= 32) computes the
affine form of App. A on the BF16-stored bases, so its references are the
oracle's ``apc_run_affine`` and ``apc_adjoint_affine`` on ``round_bf16`` of
the oracle's own bases (the same rounding decision on both sides).  Operands
enter the BF16 tensor cores as sums of BF16 planes (xbar' and mu: 3 planes,
24 bits; z and v: 2 planes, 16 bits), so the tolerance is the batched path's
1e-4 relative (a NumPy model of 2-plane v over 200 reverse steps: 2e-5)."""
import numpy as np
import pytest
import scipy.linalg as sla

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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _oracle_system(A, offs):
    bl = O.partition(A, np.zeros(A.shape[0]), offs)
    QR = [O.block_qr(Ai) for Ai, _ in bl]
    return [q for q, _ in QR], [r for _, r in QR]


def _affine_forward(Qs, Rs, offs, B, g, e, T):
    Qt = [O.round_bf16(Q) for Q in Qs]
    cs = [O.block_coefficients(Q, R, B[offs[i]:offs[i + 1]]) for i, (Q, R) in enumerate(zip(Qs, Rs))]
    return O.apc_run_affine(Qt, cs, g, e, T)[1]


def _affine_backward(Qs, Rs, G, g, e, T):
    dc = O.apc_adjoint_affine([O.round_bf16(Q) for Q in Qs], g, e, T, G)
    return np.concatenate([sla.solve_triangular(R, d, lower=False) for R, d in zip(Rs, dc)])


@pytest.mark.parametrize("k,T", [(4, 0), (4, 1), (4, 30), (24, 30)])
def test_batch_backward_matches_affine_oracle(k, T):
    # three uneven systems advanced together; dL/dB of each against the
    # oracle's reverse sweep through the affine form on the BF16 bases
    apc, dev = _env()
    rng = np.random.default_rng(11)
    systems = []
    for n_s in (90, 150, 300):
        A_s = rng.standard_normal((n_s, n_s)) + 0.5 * np.sqrt(n_s) * np.eye(n_s)
        systems.append((A_s, rng.standard_normal((n_s, k)), inputs.uneven_offsets(n_s, 16, 64, rng)))
    bt = apc.apc_batch_setup([torch.tensor(A_s, device=dev) for A_s, _, _ in systems],
                             [torch.tensor(B_s, device=dev) for _, B_s, _ in systems], [o for _, _, o in systems])
    params = [(1.0, 1.0), (1.2, 1.5), (0.9, 2.5)]
    bt.set_params([p[0] for p in params], [p[1] for p in params])
    Gs = [rng.standard_normal((A_s.shape[0], k)) for A_s, _, _ in systems]
    DB = bt.backward([torch.tensor(G, device=dev) for G in Gs], T)
    for (A_s, B_s, o), (g, e), G, db in zip(systems, params, Gs, DB):
        Qs, Rs = _oracle_system(A_s, o)
        want = _affine_backward(Qs, Rs, G, g, e, T)
        assert _rel(db.cpu().numpy(), want) <= 1e-4, (A_s.shape[0], T)
    # the batch still iterates after a reset
    X = bt.forward(10)
    for (A_s, B_s, o), (g, e), x in zip(systems, params, X):
        Qs, Rs = _oracle_system(A_s, o)
        assert _rel(x.cpu().numpy(), _affine_forward(Qs, Rs, o, B_s, g, e, 10)) <= 1e-4


@pytest.mark.parametrize("prec", ["bf16", "f64"])
def test_forward_and_backward_rhs_in_one_call(prec):
    # BF16 square context: the tensor-core form (App. A) against the oracle's
    # affine run and reverse sweep on the rounded bases; FP64 context: the
    # column loop against Eq. (cons) and its reverse sweep, with B and G given
    # as column slices of wider matrices (leading dimension > k)
    apc, dev = _env()
    n, m, k, T = 640, 5, 6, 25
    A, _, _ = inputs.gaussian_system(n, 61)
    rng = np.random.default_rng(12)
    Bw = rng.standard_normal((n, k + 3))
    Gw = rng.standard_normal((n, k + 2))
    offs = inputs.even_offsets(n, m)
    Qs, Rs = _oracle_system(A, offs)
    g, e, _ = O.optimal_params(*O.mu_bounds(Qs))
    ctx = apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(Bw[:, 0].copy(), device=dev), offs, precision=prec)
    Bt = torch.tensor(Bw, device=dev)[:, :k]
    Gt = torch.tensor(Gw, device=dev)[:, :k]
    X = ctx.forward_rhs(Bt, T, g, e).cpu().numpy()
    DB = ctx.backward_rhs(Gt, T, g, e).cpu().numpy()
    B, G = Bw[:, :k], Gw[:, :k]
    if prec == "bf16":
        assert _rel(X, _affine_forward(Qs, Rs, offs, B, g, e, T)) <= 1e-4
        assert _rel(DB, _affine_backward(Qs, Rs, G, g, e, T)) <= 1e-4
    else:
        bl = O.partition(A, B, offs)
        ref = O.apc_run(A, B, offs, g, e, max_iters=T, Qs=Qs, Rs=Rs)
        assert _rel(X, ref.xbar) <= 1e-10
        want = np.concatenate(O.apc_adjoint(bl, Qs, Rs, g, e, T, G)[0])
        assert _rel(DB, want) <= 1e-10


def test_rhs_parameters_change_between_calls():
    # one BF16 context, calls with (gamma1, eta1), then (gamma2, eta2), then
    # (gamma1, eta1) again: every call follows its own parameters (the batch's
    # parameters are uploaded again only when they change), forward and reverse
    apc, dev = _env()
    n, m, k, T = 512, 4, 5, 20
    A, _, _ = inputs.gaussian_system(n, 63)
    rng = np.random.default_rng(14)
    B = rng.standard_normal((n, k))
    G = rng.standard_normal((n, k))
    offs = inputs.even_offsets(n, m)
    Qs, Rs = _oracle_system(A, offs)
    g1, e1, _ = O.optimal_params(*O.mu_bounds(Qs))
    g2, e2 = 0.8, 1.3
    ctx = apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(B[:, 0].copy(), device=dev), offs, precision="bf16")
    Bt, Gt = torch.tensor(B, device=dev), torch.tensor(G, device=dev)
    for g, e in ((g1, e1), (g2, e2), (g2, e2), (g1, e1)):
        X = ctx.forward_rhs(Bt, T, g, e).cpu().numpy()
        DB = ctx.backward_rhs(Gt, T, g, e).cpu().numpy()
        assert _rel(X, _affine_forward(Qs, Rs, offs, B, g, e, T)) <= 1e-4
        assert _rel(DB, _affine_backward(Qs, Rs, G, g, e, T)) <= 1e-4


def test_differentiation_workload_on_tensor_cores_full_size():
    # The differentiation workload (A 8192 x 8192 Gaussian, m = 32 blocks of
    # 256, k = 16, T = 200) through APCSolveFn on a BF16 context: one call per
    # direction on the tensor cores.  The gradient of L = 0.5 ||xbar_T - x_t||^2
    # with respect to B against the oracle's reverse sweep through the affine
    # form on the BF16 bases (FP64, all 8192 x 16 entries), the forward against
    # the oracle's affine run, and the dot-product test of the GPU's own
    # forward and reverse maps.
    apc, dev = _env()
    n, m, k, T = 8192, 32, 16, 200
    A, _, _ = inputs.gaussian_system_torch(n, 77, dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(78)
    B = torch.randn((n, k), generator=gen, device=dev, dtype=torch.float64)
    xt = torch.randn((n, k), generator=gen, device=dev, dtype=torch.float64)
    offs = inputs.even_offsets(n, m)
    ctx = apc.apc_setup(A, B[:, 0].contiguous(), offs, precision="bf16")
    lo, hi = ctx.spectral_bounds(steps=60, seed=5)
    gam, eta, _ = apc.apc_optimal_params(0.5 * lo, min(1.0, 1.01 * hi))
    bt = B.clone().requires_grad_(True)
    x = apc.APCSolveFn.apply(bt, ctx, gam, eta, T)
    loss = 0.5 * ((x - xt) ** 2).sum()
    loss.backward()
    Qs, Rs = _oracle_system(A.cpu().numpy(), offs)
    Bh = B.cpu().numpy()
    xf = _affine_forward(Qs, Rs, offs, Bh, gam, eta, T)
    assert _rel(x.detach().cpu().numpy(), xf) <= 1e-4
    want = _affine_backward(Qs, Rs, xf - xt.cpu().numpy(), gam, eta, T)
    assert _rel(bt.grad.cpu().numpy(), want) <= 1e-4
    V = torch.randn((n, k), generator=gen, device=dev, dtype=torch.float64)
    W = torch.randn((n, k), generator=gen, device=dev, dtype=torch.float64)
    JV, JTW = ctx.forward_rhs(V, T, gam, eta), ctx.backward_rhs(W, T, gam, eta)
    lhs, rhs = float((JV * W).sum()), float((V * JTW).sum())
    # a dot product of n k terms of both signs: its rounding scales with the
    # norms of its factors, not with its value
    scale = max(float(torch.linalg.norm(JV) * torch.linalg.norm(W)), float(torch.linalg.norm(V) * torch.linalg.norm(JTW)))
    assert abs(lhs - rhs) <= 1e-4 * scale


@pytest.mark.parametrize("k", [1, 40])
def test_rhs_column_loop_on_bf16_context(k):
    # k = 1 and k > 32 on a BF16 context take the columns one after another
    # through the iteration kernel (Eq. (cons)), checked against the oracle on
    # the BF16-rounded bases at the rounding bound
    apc, dev = _env()
    n, m, T = 384, 3, 12
    A, _, _ = inputs.gaussian_system(n, 62)
    B = np.random.default_rng(13).standard_normal((n, k))
    offs = inputs.even_offsets(n, m)
    Qs, Rs = _oracle_system(A, offs)
    g, e = 1.0, 1.5
    ctx = apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(B[:, 0].copy(), device=dev), offs, precision="bf16")
    X = ctx.forward_rhs(torch.tensor(B, device=dev), T, g, e).cpu().numpy()
    Qt = [O.round_bf16(Q) for Q in Qs]
    for j in (0, k - 1):
        xs0 = [Q @ O.block_coefficients(Q0, R, B[offs[i]:offs[i + 1], j]) for i, (Q, Q0, R) in enumerate(zip(Qt, Qs, Rs))]
        ref = O.apc_run(A, B[:, j], offs, g, e, max_iters=T, Qs=Qt, xs0=xs0)
        assert _rel(X[:, j], ref.xbar) <= 1e-5, j
