"""GPU parity of the CUDA path against the FP64 oracle, through the C ABI.

Tolerances.  FP64: both sides compute Eq. (cons) in float64 with different
summation orders; after T iterations the difference is a few hundred ulps
times the iteration's transient gain, so 1e-10 relative is a safe bound.

FP32 and BF16: the oracle runs on the bases the GPU stores, rounded the same
way from its own QR (FP32, or BF16 by ``round_bf16``; the QR with a positive
diagonal of R is unique, so both sides hold the same basis up to column
signs, which Eq. (cons) does not see), so only the arithmetic's rounding
separates the two trajectories.  The machines' iterates are FP32 (unit
roundoff u = 2^-24).  Each step the master forms
(eta/m) sum_i x_i + (1 - eta) xbar, two terms of about eta |xbar| each, so the
rounding of the machines' values reaches xbar amplified by eta, and on the
early iterations (spectral radius close to 1) these errors add up rather than
decay: after T steps the relative difference is at most about eta T u.  The
tests use ``rounding_bound`` = max(1e-5, |eta| T u) (measured: about a
quarter of it with Theorem 1's parameters, where eta ~ m; below 1e-6 with
eta = 1.5 over 100 iterations, which is where the 1e-5 bar of the
single-precision path is checked)."""
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


def _case(n, m, seed, N=None, offs=None):
    A, x_true, b = inputs.gaussian_system(n, seed, N=N)
    offs = inputs.even_offsets(A.shape[0], m) if offs is None else offs
    blocks = O.partition(A, b, offs)
    QR = [O.block_qr(Ai) for Ai, _ in blocks]
    Qs, Rs = [q for q, _ in QR], [r for _, r in QR]
    lo, hi = O.mu_bounds(Qs)
    g, e, rho = O.optimal_params(lo, hi)
    return A, x_true, b, offs, blocks, Qs, Rs, g, e


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def rounding_bound(eta, T):
    """max(1e-5, |eta| T u), u = 2^-24: see the module docstring."""
    return max(1e-5, abs(eta) * T * 2.0 ** -24)


def _f32(q):
    return q.astype(np.float32).astype(np.float64)


def _stored_basis_run(Qs, Rs, blocks, rnd, g, e, T):
    """Oracle trajectory (Eq. (cons), Algorithm 1) on the bases as the GPU
    stores them: Q_i rounded by `rnd`, x_i(0) = Q_i c_i (the least-norm start
    computed with the stored basis), xbar(0) their mean."""
    Qr = [rnd(Q) for Q in Qs]
    xs0 = [Q @ O.block_coefficients(Q0, R, bi) for Q, Q0, R, (_, bi) in zip(Qr, Qs, Rs, blocks)]
    A = np.concatenate([Ai for Ai, _ in blocks])
    b = np.concatenate([bi for _, bi in blocks])
    offs = np.concatenate([[0], np.cumsum([Ai.shape[0] for Ai, _ in blocks])])
    return O.apc_run(A, b, offs, g, e, max_iters=T, Qs=Qr, xs0=xs0)


@pytest.mark.parametrize("n,m,p_desc", [(500, 10, "c1 50-row blocks"), (333, 7, "ragged 47/48-row"),
                                        (640, 5, "128-row blocks")])
def test_f64_least_norm_init_matches_oracle(n, m, p_desc):
    apc, dev = _apc(), _dev()
    A, x_true, b, offs, blocks, Qs, Rs, g, e = _case(n, m, 1)
    ctx = apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(b, device=dev), offs, precision="f64")
    ctx.reset()
    X = ctx.x().cpu().numpy()
    for i, (Q, R, (_, bi)) in enumerate(zip(Qs, Rs, blocks)):
        ref = O.least_norm_init(Q, R, bi)
        assert _rel(X[i], ref) <= 1e-11, i
    xs = [O.least_norm_init(Q, R, bi) for Q, R, (_, bi) in zip(Qs, Rs, blocks)]
    assert _rel(ctx.xbar().cpu().numpy(), sum(xs) / m) <= 1e-11


@pytest.mark.parametrize("n,m,T", [(500, 10, 300), (257, 3, 200), (1000, 40, 100), (96, 1, 5)])
def test_f64_trajectory_matches_oracle(n, m, T):
    apc, dev = _apc(), _dev()
    A, x_true, b, offs, blocks, Qs, Rs, g, e = _case(n, m, 2) if m > 1 else _case(n, 1, 2)
    if m == 1:
        g, e = 1.0, 1.0
    ref = O.apc_run(A, b, offs, g, e, max_iters=T, Qs=Qs, Rs=Rs)
    ctx = apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(b, device=dev), offs, precision="f64")
    ctx.reset()
    # split the T iterations over several launches to cover the z-buffer hand-off
    done = 0
    for k in (1, T // 3, T):
        k = min(k, T - done)
        if k > 0:
            ctx.iterate(g, e, k)
            done += k
    assert _rel(ctx.xbar().cpu().numpy(), ref.xbar) <= 1e-10
    X = ctx.x().cpu().numpy()
    for i in range(m):
        assert _rel(X[i], ref.xs[i]) <= 1e-10


@pytest.mark.parametrize("n,offs", [(1, [0, 1]), (2, [0, 1, 2]), (3, [0, 1, 2, 3]), (5, [0, 2, 5]),
                                    (64, [0, 1, 2, 10, 11, 40, 64]), (70, [0, 70]), (256, [0, 256])])
def test_degenerate_shapes_f64(n, offs):
    # 1 x 1 to 5 x 5 systems (fewer rows than one pipeline group per cluster,
    # a one-row last group), 1-row blocks, and a single block holding the
    # whole square system (P_1 = 0: the least-norm start is the solution and
    # the iteration leaves it there); zero iterations change nothing
    apc, dev = _apc(), _dev()
    offs = np.asarray(offs, dtype=np.int64)
    A, x_true, b, offs, blocks, Qs, Rs, g, e = _case(n, len(offs) - 1, 12, offs=offs)
    ctx = apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(b, device=dev), offs, precision="f64")
    ctx.reset()
    x0 = ctx.xbar().cpu().numpy()
    ref0 = sum(O.least_norm_init(Q, R, bi) for Q, R, (_, bi) in zip(Qs, Rs, blocks)) / len(blocks)
    assert _rel(x0, ref0) <= 1e-12
    ctx.iterate(g, e, 0)
    assert np.array_equal(ctx.xbar().cpu().numpy(), x0)
    T = 40
    ref = O.apc_run(A, b, offs, g, e, max_iters=T, Qs=Qs, Rs=Rs)
    ctx.iterate(g, e, T)
    assert _rel(ctx.xbar().cpu().numpy(), ref.xbar) <= 1e-10
    if len(offs) == 2:
        assert _rel(ctx.xbar().cpu().numpy(), x_true) <= 1e-9


def test_block_wider_than_256_rows_is_unsupported():
    apc, dev = _apc(), _dev()
    A, _, b = inputs.gaussian_system(300, 13)
    with pytest.raises(apc.ApcError) as ei:
        apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(b, device=dev), [0, 257, 300], precision="f64")
    assert ei.value.name == "UNSUPPORTED"
    with pytest.raises(apc.ApcError) as ei:  # more rows than unknowns: rank-deficient block
        Bt, _, bt = inputs.gaussian_system(40, 13, N=90)
        apc.apc_setup(torch.tensor(Bt, device=dev), torch.tensor(bt, device=dev), [0, 45, 90], precision="f64")
    assert ei.value.name == "SINGULAR_BLOCK"


def test_f64_solve_config1_reaches_lu_solution():
    # 500 x 500 Gaussian, m = 10 blocks of 50 rows, optimal (gamma, eta), tol 1e-10
    apc, dev = _apc(), _dev()
    A, x_true, b, offs, blocks, Qs, Rs, g, e = _case(500, 10, 0)
    ctx = apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(b, device=dev), offs, precision="f64")
    x, st = ctx.solve(g, e, tol=1e-10, max_iters=400000, check_every=500)
    x = x.cpu().numpy()
    assert st["rel_residual"] <= 1e-10
    assert O.relative_residual(A, b, x) <= 1e-10
    x_star = np.linalg.solve(A, b)
    assert _rel(x, x_star) <= 1e-10 * np.linalg.cond(A)


@pytest.mark.parametrize("n,m,T", [(2048, 8, 60), (1500, 6, 100), (4000, 16, 100), (2048, 8, 120)])
def test_f32_trajectory_matches_oracle(n, m, T):
    # Theorem 1's parameters; the oracle on the FP32-rounded bases; the
    # machines' iterates as well as xbar, at the rounding bound
    apc, dev = _apc(), _dev()
    A, x_true, b, offs, blocks, Qs, Rs, g, e = _case(n, m, 4)
    ref = _stored_basis_run(Qs, Rs, blocks, _f32, g, e, T)
    ctx = apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(b, device=dev), offs, precision="f32")
    ctx.reset()
    ctx.iterate(g, e, T)
    tol = rounding_bound(e, T)
    assert _rel(ctx.xbar().cpu().numpy(), ref.xbar) <= tol
    X = ctx.x().cpu().numpy()
    assert max(_rel(X[i], ref.xs[i]) for i in range(m)) <= tol
    # against the exact-basis trajectory too (the FP32 basis moves it by ~1e-7)
    ex = O.apc_run(A, b, offs, g, e, max_iters=T, Qs=Qs, Rs=Rs)
    assert _rel(ctx.xbar().cpu().numpy(), ex.xbar) <= tol


@pytest.mark.parametrize("cs,wpw", [(1, 1), (1, 2), (2, 2), (4, 1), (4, 2), (8, 2), (1, 4), (2, 4), (4, 4)])
def test_cluster_sizes_agree(cs, wpw):
    # the same problem under every cluster size / workers per warp gives the oracle's trajectory
    apc, dev = _apc(), _dev()
    n, m, T = 1200, 16, 30
    A, x_true, b, offs, blocks, Qs, Rs, g, e = _case(n, m, 5)
    ref = O.apc_run(A, b, offs, g, e, max_iters=T, Qs=Qs, Rs=Rs)
    ctx = apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(b, device=dev), offs, precision="f32",
                        cluster_size=cs, workers_per_warp=wpw)
    assert ctx.info()["cluster_size"] == cs
    ctx.reset()
    ctx.iterate(g, e, T)
    assert _rel(ctx.xbar().cpu().numpy(), ref.xbar) <= 1e-5


@pytest.mark.parametrize("cs,m", [(3, 16), (5, 18), (6, 22), (7, 26), (0, 144)])
def test_cluster_sizes_not_powers_of_two(cs, m):
    # clusters of 3, 5, 6 and 7 CTAs (the last CTA of each holds fewer
    # workers), and the automatic choice for m = 144 blocks (5 CTAs of <= 30
    # worker slots) give the oracle's trajectory.  FP64 path (the same kernel
    # template), so that an exchange error cannot hide under FP32 rounding,
    # which at m = 144 (eta ~ 145) already moves the trajectory by ~5e-5.
    apc, dev = _apc(), _dev()
    n, T = (2304 if m == 144 else 1200), 30
    A, x_true, b, offs, blocks, Qs, Rs, g, e = _case(n, m, 5)
    ref = O.apc_run(A, b, offs, g, e, max_iters=T, Qs=Qs, Rs=Rs)
    ctx = apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(b, device=dev), offs, precision="f64",
                        cluster_size=cs)
    assert ctx.info()["cluster_size"] == (cs if cs else 5)
    ctx.reset()
    ctx.iterate(g, e, T)
    assert _rel(ctx.xbar().cpu().numpy(), ref.xbar) <= 1e-10


@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32", 1e-5)])
@pytest.mark.parametrize("rg,cs", [(1, 0), (1, 2), (1, 4), (2, 0), (2, 4)])
def test_rows_per_group_agree(prec, tol, rg, cs):
    # one or two rows of Q per pipeline step (2 or 4 control warps, a full or a
    # transposed butterfly for the first product) give the oracle's trajectory
    apc, dev = _apc(), _dev()
    n, m, T = 1201, 16, 30
    A, x_true, b, offs, blocks, Qs, Rs, g, e = _case(n, m, 7)
    ref = O.apc_run(A, b, offs, g, e, max_iters=T, Qs=Qs, Rs=Rs)
    ctx = apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(b, device=dev), offs, precision=prec,
                        cluster_size=cs, rows_per_group=rg)
    info = ctx.info()
    assert info["rows_per_group"] == rg and (cs == 0 or info["cluster_size"] == cs)
    ctx.reset()
    ctx.iterate(g, e, T)
    assert _rel(ctx.xbar().cpu().numpy(), ref.xbar) <= tol


@pytest.mark.parametrize("prec,n,m,want", [("bf16", 16640, 128, (4, 2)), ("f32", 16640, 128, (4, 1)),
                                           ("f32", 8192, 32, (1, 1)), ("bf16", 8192, 32, (1, 2))])
def test_automatic_configuration(prec, n, m, want):
    # blocks of 130 / 256 rows (width 256): the smallest cluster whose CTAs hold
    # <= 32 workers, two rows per step where the ring still has >= 5 stages of
    # two rows (BF16), one row otherwise (FP32 stages are twice as large)
    apc, dev = _apc(), _dev()
    A, _, b = inputs.gaussian_system_torch(n, 3, dev)
    ctx = apc.apc_setup(A, b, inputs.even_offsets(n, m), precision=prec)
    info = ctx.info()
    assert (info["cluster_size"], info["rows_per_group"]) == want, info
    assert info["width"] == 256


def _headline_shape(n, seed):
    # m = 128 blocks with one block of 256 rows: width 256 and 32 worker
    # slots per CTA in 4-CTA clusters, as at n = 32768 (blocks of 256), at a
    # size the oracle runs in seconds
    A, x_true, b = inputs.gaussian_system(n, seed)
    offs = np.concatenate([[0], 256 + inputs.even_offsets(n - 256, 127)]).astype(np.int64)
    return A, x_true, b, offs


@pytest.mark.parametrize("shape,params,T", [("m128", "fixed", 100), ("m128", "theorem1", 60),
                                            ("m32", "fixed", 100), ("m32", "theorem1", 100)])
def test_bf16_headline_launch_configuration_matches_stored_basis_oracle(shape, params, T):
    # The benchmark's launch configuration (BF16 Q, blocks of width 256, 4-CTA
    # clusters, two rows of Q per pipeline step) against Eq. (cons) on the
    # BF16-rounded bases, element by element: xbar and every x_i.  With
    # (gamma, eta) = (1, 1.5) the single-precision bar of 1e-5 holds over 100
    # iterations; with Theorem 1's parameters the rounding bound applies.
    apc, dev = _apc(), _dev()
    if shape == "m128":
        A, x_true, b, offs = _headline_shape(4096, 31)
    else:
        A, x_true, b = inputs.gaussian_system(8192, 32)
        offs = inputs.even_offsets(8192, 32)
    blocks = O.partition(A, b, offs)
    QR = [O.block_qr(Ai) for Ai, _ in blocks]
    Qs, Rs = [q for q, _ in QR], [r for _, r in QR]
    if params == "fixed":
        g, e = 1.0, 1.5
    else:
        g, e, _ = O.optimal_params(*O.mu_bounds(Qs))
    ref = _stored_basis_run(Qs, Rs, blocks, O.round_bf16, g, e, T)
    m = len(offs) - 1
    ctx = apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(b, device=dev), offs, precision="bf16",
                        cluster_size=4, rows_per_group=2)
    info = ctx.info()
    assert (info["width"], info["cluster_size"], info["rows_per_group"]) == (256, 4, 2), info
    ctx.reset()
    ctx.iterate(g, e, T // 3)
    ctx.iterate(g, e, T - T // 3)
    tol = 1e-5 if params == "fixed" else rounding_bound(e, T)
    assert _rel(ctx.xbar().cpu().numpy(), ref.xbar) <= tol
    X = ctx.x().cpu().numpy()
    assert max(_rel(X[i], ref.xs[i]) for i in range(m)) <= tol


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_refinement_reaches_1e10(prec):
    apc, dev = _apc(), _dev()
    n, m = 512, 8
    A, x_true, b, offs, blocks, Qs, Rs, g, e = _case(n, m, 7)
    ctx = apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(b, device=dev), offs, precision=prec)
    x, st = ctx.solve(g, e, tol=1e-10, max_iters=2_000_000, check_every=200, refine=True)
    x = x.cpu().numpy()
    assert O.relative_residual(A, b, x) <= 1e-10
    assert st["sweeps"] >= 2


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_refinement_on_tall_scaled_family(prec):
    # The headline's family A = D_r G D_c made tall (N = 1.125 n), D_c narrowed
    # to half a decade each way (kappa(X) ~ 6e3): parameters from the GPU
    # Lanczos bounds, refinement to 1e-10 checked by the oracle's residual.
    apc, dev = _apc(), _dev()
    n, N = 2048, 2304
    A, x_true, b = inputs.scaled_system(n, 21, N=N, col_decades=0.5)
    offs = inputs.even_offsets(N, 9)
    ctx = apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(b, device=dev), offs, precision=prec)
    lo, hi = ctx.spectral_bounds(steps=100)
    assert 1e3 < hi / lo < 1e5
    g, e, _ = apc.apc_optimal_params(0.98 * lo, min(1.0, 1.01 * hi))
    x, st = ctx.solve(g, e, tol=1e-10, max_iters=20000, check_every=50, refine=True)
    x = x.cpu().numpy()
    assert st["rc"] == 0
    assert O.relative_residual(A, b, x) <= 1e-10


def test_tall_uneven_blocks_f64():
    # N > n (Sec. 2) with uneven contiguous blocks whose widths are not multiples of 32
    apc, dev = _apc(), _dev()
    rng = np.random.default_rng(8)
    A, x_true, b = inputs.gaussian_system(200, 8, N=450)
    offs = inputs.uneven_offsets(450, 17, 70, rng)
    blocks = O.partition(A, b, offs)
    QR = [O.block_qr(Ai) for Ai, _ in blocks]
    Qs, Rs = [q for q, _ in QR], [r for _, r in QR]
    lo, hi = O.mu_bounds(Qs)
    g, e, _ = O.optimal_params(lo, hi)
    T = 150
    ref = O.apc_run(A, b, offs, g, e, max_iters=T, Qs=Qs, Rs=Rs)
    ctx = apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(b, device=dev), offs, precision="f64")
    ctx.reset()
    ctx.iterate(g, e, T)
    assert _rel(ctx.xbar().cpu().numpy(), ref.xbar) <= 1e-10


def test_errors_reported():
    apc, dev = _apc(), _dev()
    A, _, b = inputs.gaussian_system(64, 9)
    offs = inputs.even_offsets(64, 4)
    A2 = A.copy()
    A2[1] = A2[0]
    with pytest.raises(apc.ApcError) as ei:
        apc.apc_setup(torch.tensor(A2, device=dev), torch.tensor(b, device=dev), offs, precision="f64")
    assert ei.value.name == "SINGULAR_BLOCK"
    b2 = b.copy()
    b2[5] = np.nan
    with pytest.raises(apc.ApcError) as ei:
        apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(b2, device=dev), offs, precision="f32")
    assert ei.value.name == "NONFINITE"
    with pytest.raises(apc.ApcError) as ei:
        apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(b, device=dev), [0, 10, 10, 64])
    assert ei.value.name == "INVALID_ARG"
    with pytest.raises(apc.ApcError) as ei:
        apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(b, device=dev), offs, rows_per_group=3)
    assert ei.value.name == "INVALID_ARG"
    ctx = apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(b, device=dev), offs, precision="f32")
    ctx.reset()
    with pytest.raises(apc.ApcError) as ei:
        ctx.iterate(2.5, 1.0, 3)
    assert ei.value.name == "PARAMS"
    x, st = ctx.solve(1.0, 1.0, tol=1e-14, max_iters=20, check_every=10, raise_on_error=False)
    assert apc.ERRORS[st["rc"]] == "NOT_CONVERGED"


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-6), ("bf16", 1e-2)])
def test_basis_spans_row_space_and_projector_matches(prec, tol):
    # Sec. 3.1/3.3: Q_i orthonormal, A_i P_i = 0, and I - Q_i Q_i^T equals the oracle's projector
    apc, dev = _apc(), _dev()
    rng = np.random.default_rng(10)
    A, x_true, b = inputs.gaussian_system(150, 10)
    offs = inputs.uneven_offsets(150, 20, 45, rng)
    ctx = apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(b, device=dev), offs, precision=prec)
    for i, (Ai, _) in enumerate(O.partition(A, b, offs)):
        Q = ctx.basis(i).cpu().numpy()
        assert Q.shape == (150, Ai.shape[0])
        assert np.abs(Q.T @ Q - np.eye(Q.shape[1])).max() <= 4 * tol
        P = np.eye(150) - Q @ Q.T
        assert np.abs(P - O.projector(Ai)).max() <= 4 * tol
        assert np.abs(Ai @ P).max() <= 4 * tol * np.abs(Ai).max() * np.sqrt(150)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32", 1e-4)])
def test_backward_matches_oracle_adjoint(prec, tol):
    # dL/db through T unrolled iterations (transpose of Eq. (cons)) against the FP64 oracle sweep
    apc, dev = _apc(), _dev()
    n, m, T = 600, 6, 40
    A, x_true, b, offs, blocks, Qs, Rs, g, e = _case(n, m, 12)
    xt = inputs.target_vector(n, 12)
    xbar, _, _ = O.apc_forward_linear(blocks, Qs, Rs, g, e, T)
    gT = xbar - xt
    ref = np.concatenate(O.apc_adjoint(blocks, Qs, Rs, g, e, T, gT)[0])
    ctx = apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(b, device=dev), offs, precision=prec)
    db = ctx.backward(torch.tensor(gT, device=dev), T, g, e).cpu().numpy()
    assert _rel(db, ref) <= tol
    # the reverse sweep leaves the context usable for a fresh forward solve
    ctx.reset()
    ctx.iterate(g, e, 5)


def test_backward_with_four_workers_per_warp():
    # the reverse sweep's generic pass modes with 32 blocks in one CTA and four
    # workers per element warp (FP32 context), against the FP64 oracle sweep
    apc, dev = _apc(), _dev()
    n, m, T = 2048, 32, 30
    A, x_true, b, offs, blocks, Qs, Rs, g, e = _case(n, m, 16)
    gT = inputs.target_vector(n, 16)
    ref = np.concatenate(O.apc_adjoint(blocks, Qs, Rs, g, e, T, gT)[0])
    ctx = apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(b, device=dev), offs, precision="f32",
                        workers_per_warp=4)
    db = ctx.backward(torch.tensor(gT, device=dev), T, g, e).cpu().numpy()
    assert _rel(db, ref) <= 1e-4


@pytest.mark.parametrize("prec,ck,tol", [("f64", 1, 1e-9), ("f64", 7, 1e-9), ("f64", 0, 1e-9), ("f64", 40, 1e-9),
                                         ("f32", 0, 2e-3)])
def test_backward_params_match_oracle(prec, ck, tol):
    # dL/dgamma and dL/deta through T iterations, from forward states recomputed
    # out of checkpoints every ck iterations (0 = 20; 7 leaves a short last
    # segment), and dL/db, against the FP64 oracle sweep, for a right-hand side
    # other than the one given at set-up (the forward trajectory depends on it)
    apc, dev = _apc(), _dev()
    n, m, T = 600, 6, 40
    A, x_true, b, offs, blocks, Qs, Rs, g, e = _case(n, m, 12)
    b2 = np.random.default_rng(5).standard_normal(n)
    blocks2 = O.partition(A, b2, offs)
    xt = inputs.target_vector(n, 12)
    xbar, _, states = O.apc_forward_linear(blocks2, Qs, Rs, g, e, T)
    gT = xbar - xt
    db_ref, dg_ref, de_ref = O.apc_adjoint(blocks2, Qs, Rs, g, e, T, gT, states=states)
    ctx = apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(b, device=dev), offs, precision=prec)
    db, dg, de = ctx.backward_params(torch.tensor(gT, device=dev), T, g, e, b=torch.tensor(b2, device=dev),
                                     ckpt_every=ck)
    assert _rel(db.cpu().numpy(), np.concatenate(db_ref)) <= (1e-10 if prec == "f64" else 1e-4)
    assert dg == pytest.approx(dg_ref, rel=tol), (dg, dg_ref)
    assert de == pytest.approx(de_ref, rel=tol), (de, de_ref)
    # zero iterations: no parameter dependence; the context stays usable
    db0, dg0, de0 = ctx.backward_params(torch.tensor(gT, device=dev), 0, g, e)
    assert dg0 == 0.0 and de0 == 0.0
    ctx.reset()
    ctx.iterate(g, e, 5)


def test_backward_params_full_size_central_difference():
    # the differentiation workload's sizes (n = 8192, m = 32 blocks of 256,
    # T = 200, checkpoints every 20), FP64 path: dL/dgamma and dL/deta of
    # L = 0.5 ||xbar(T) - x_target||^2 against central differences of L
    # through the forward iteration, and the FP32 path against the FP64 one
    apc, dev = _apc(), _dev()
    n, m, T, g, e = 8192, 32, 200, 1.0, 1.0
    A, _, b = inputs.gaussian_system_torch(n, 78, dev)
    offs = inputs.even_offsets(n, m)
    xt = torch.tensor(inputs.target_vector(n, 78), device=dev)
    ctx = apc.apc_setup(A, b, offs, precision="f64")

    def loss(gg, ee):
        ctx.reset()
        ctx.iterate(gg, ee, T)
        return 0.5 * float(torch.sum((ctx.xbar() - xt) ** 2))

    ctx.reset()
    ctx.iterate(g, e, T)
    gT = ctx.xbar() - xt
    _, dg, de = ctx.backward_params(gT, T, g, e, ckpt_every=20)
    h = 1e-5
    fdg = (loss(g + h, e) - loss(g - h, e)) / (2 * h)
    fde = (loss(g, e + h) - loss(g, e - h)) / (2 * h)
    assert dg == pytest.approx(fdg, rel=1e-5), (dg, fdg)
    assert de == pytest.approx(fde, rel=1e-5), (de, fde)
    c32 = apc.apc_setup(A, b, offs, precision="f32")
    _, dg32, de32 = c32.backward_params(gT, T, g, e, ckpt_every=20)
    assert dg32 == pytest.approx(dg, rel=1e-3) and de32 == pytest.approx(de, rel=1e-3), (dg32, dg, de32, de)


def test_autograd_grad_b_matches_central_difference():
    # L = 0.5 ||xbar_T - x_target||^2 is quadratic in b: central differences of the
    # FP64 oracle forward are exact up to rounding (spec bar: 1e-4 relative)
    apc, dev = _apc(), _dev()
    n, m, T, k = 512, 8, 40, 3
    A, _, B = inputs.gaussian_system(n, 13, k=k)
    offs = inputs.even_offsets(n, m)
    blocks = O.partition(A, B, offs)
    QR = [O.block_qr(Ai) for Ai, _ in blocks]
    Qs, Rs = [q for q, _ in QR], [r for _, r in QR]
    lo, hi = O.mu_bounds(Qs)
    g, e, _ = O.optimal_params(lo, hi)
    xt = inputs.target_vector(n, 13, k=k)
    ctx = apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(B[:, 0].copy(), device=dev), offs, precision="f32")
    bt = torch.tensor(B, device=dev, requires_grad=True)
    x = apc.APCSolveFn.apply(bt, ctx, g, e, T)
    loss = 0.5 * ((x - torch.tensor(xt, device=dev)) ** 2).sum()
    loss.backward()
    grad = bt.grad.cpu().numpy()

    def L(Bv):
        xb, _, _ = O.apc_forward_linear(O.partition(A, Bv, offs), Qs, Rs, g, e, T)
        return 0.5 * float(np.sum((xb - xt) ** 2))

    rng = np.random.default_rng(3)
    for _ in range(3):
        d = rng.standard_normal(B.shape)
        h = 1e-2 * np.linalg.norm(B)
        fd = (L(B + h * d) - L(B - h * d)) / (2 * h)
        assert float(np.sum(grad * d)) == pytest.approx(fd, rel=1e-4)


def test_autograd_gamma_eta_two_columns_match_oracle():
    # torch.autograd through APCSolveFn with gamma and eta as tensors: the
    # gradients sum over the k = 2 columns, each from its own forward
    # trajectory (checkpoints every 9 iterations), against the oracle
    apc, dev = _apc(), _dev()
    n, m, T = 400, 5, 30
    A, x_true, b, offs, blocks, Qs, Rs, g, e = _case(n, m, 21)
    Bm = np.random.default_rng(6).standard_normal((n, 2))
    Xt = np.random.default_rng(7).standard_normal((n, 2))
    dg_ref = de_ref = 0.0
    db_ref = []
    for j in range(2):
        bl = O.partition(A, Bm[:, j], offs)
        xbar, _, states = O.apc_forward_linear(bl, Qs, Rs, g, e, T)
        dbj, dgj, dej = O.apc_adjoint(bl, Qs, Rs, g, e, T, xbar - Xt[:, j], states=states)
        dg_ref, de_ref = dg_ref + dgj, de_ref + dej
        db_ref.append(np.concatenate(dbj))
    ctx = apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(b, device=dev), offs, precision="f64")
    bt = torch.tensor(Bm, device=dev, requires_grad=True)
    gt = torch.tensor(g, dtype=torch.float64, requires_grad=True)
    et = torch.tensor(e, dtype=torch.float64, requires_grad=True)
    x = apc.APCSolveFn.apply(bt, ctx, gt, et, T, 9)
    loss = 0.5 * torch.sum((x - torch.tensor(Xt, device=dev)) ** 2)
    loss.backward()
    assert float(gt.grad) == pytest.approx(dg_ref, rel=1e-9)
    assert float(et.grad) == pytest.approx(de_ref, rel=1e-9)
    assert _rel(bt.grad.cpu().numpy(), np.stack(db_ref, axis=1)) <= 1e-10


def test_backward_tends_to_inverse_transpose_at_convergence():
    apc, dev = _apc(), _dev()
    n, m = 200, 4
    A, x_true, b, offs, blocks, Qs, Rs, g, e = _case(n, m, 14)
    tr = O.apc_run(A, b, offs, g, e, tol=1e-13, max_iters=200000, record_every=50, Qs=Qs, Rs=Rs)
    gT = inputs.target_vector(n, 14)
    ctx = apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(b, device=dev), offs, precision="f64")
    db = ctx.backward(torch.tensor(gT, device=dev), tr.iters, g, e).cpu().numpy()
    ref = np.linalg.solve(A.T, gT)
    assert _rel(db, ref) <= 1e-8


def test_device_wait_timeout_is_reported_and_context_recovers():
    # Failure detection without a GPU fault: the test hook makes every grid barrier
    # wait for one CTA more than exists; the bounded wait runs out, the kernel
    # returns, the host reports TIMEOUT, and the context still solves afterwards.
    apc, dev = _apc(), _dev()
    n, m, T = 400, 8, 20
    A, x_true, b, offs, blocks, Qs, Rs, g, e = _case(n, m, 15)
    ctx = apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(b, device=dev), offs, precision="f32")
    ctx.reset()
    ctx.set_test_hooks(grid_barrier_skew=1, timeout_s=0.2)
    import time
    t0 = time.time()
    with pytest.raises(apc.ApcError) as ei:
        ctx.iterate(g, e, 3)
    assert ei.value.name == "TIMEOUT"
    assert "grid barrier" in str(ei.value)
    assert time.time() - t0 < 10
    ctx.set_test_hooks(grid_barrier_skew=0, timeout_s=2.0)
    ctx.reset()
    ctx.iterate(g, e, T)
    ref = O.apc_run(A, b, offs, g, e, max_iters=T, Qs=Qs, Rs=Rs)
    assert _rel(ctx.xbar().cpu().numpy(), ref.xbar) <= 1e-5


def test_differentiation_workload_full_size():
    # A 8192 x 8192 Gaussian, m = 32 blocks of 256, k = 16 right-hand sides,
    # L = 0.5 ||xbar_T - x_target||^2 through T = 200 unrolled iterations.
    # The map b -> xbar_T is linear and L quadratic, so central differences of
    # the FP64 forward are exact up to rounding: the FP32 autograd gradient is
    # checked against them (1e-4), and the FP64 forward / reverse sweep pass the
    # dot-product test <J v, w> = <v, J^T w>.  (gamma, eta) from the GPU
    # spectral estimates.
    apc, dev = _apc(), _dev()
    n, m, k, T = 8192, 32, 16, 200
    A, _, _ = inputs.gaussian_system_torch(n, 77, dev)
    g_ = torch.Generator(device=dev)
    g_.manual_seed(78)
    B = torch.randn((n, k), generator=g_, device=dev, dtype=torch.float64)
    xt = torch.randn((n, k), generator=g_, device=dev, dtype=torch.float64)
    offs = inputs.even_offsets(n, m)
    c64 = apc.apc_setup(A, B[:, 0].contiguous(), offs, precision="f64")
    c32 = apc.apc_setup(A, B[:, 0].contiguous(), offs, precision="f32")
    lo, hi = c64.spectral_bounds(steps=60, seed=5)
    gam, eta, _ = apc.apc_optimal_params(0.5 * lo, min(1.0, 1.01 * hi))

    def forward(ctx, Bm):
        cols = []
        for j in range(Bm.shape[1]):
            ctx.reset(Bm[:, j].contiguous())
            ctx.iterate(gam, eta, T)
            cols.append(ctx.xbar().clone())
        return torch.stack(cols, dim=1)

    bt = B.clone().requires_grad_(True)
    x = apc.APCSolveFn.apply(bt, c32, gam, eta, T)
    loss = 0.5 * ((x - xt) ** 2).sum()
    loss.backward()
    grad = bt.grad
    D = torch.randn((n, k), generator=g_, device=dev, dtype=torch.float64)
    h = 1e-2 * float(torch.linalg.norm(B))

    def L(Bm):
        return 0.5 * float(((forward(c64, Bm) - xt) ** 2).sum())

    fd = (L(B + h * D) - L(B - h * D)) / (2 * h)
    assert float((grad * D).sum()) == pytest.approx(fd, rel=1e-4)
    # dot-product test of the FP64 forward and reverse sweeps (one column)
    v = torch.randn(n, generator=g_, device=dev, dtype=torch.float64)
    w = torch.randn(n, generator=g_, device=dev, dtype=torch.float64)
    Jv = forward(c64, v.unsqueeze(1))[:, 0]
    JTw = c64.backward(w, T, gam, eta)
    lhs, rhs = float(Jv @ w), float(v @ JTw)
    assert abs(lhs - rhs) <= 1e-10 * max(abs(lhs), abs(rhs))


@pytest.mark.parametrize("name,n,m,prec", [("scaled 32768, BF16", 32768, 128, "bf16"),
                                           ("Gaussian 16384, FP32", 16384, 64, "f32")])
def test_full_size_workloads_match_stored_basis_oracle(name, n, m, prec):
    # The benchmark's workloads in its launch configuration (automatic: 4-CTA
    # clusters and two rows per step for BF16 at m = 128; 2-CTA clusters, one
    # row per step, for FP32 at m = 64), element by element against the
    # oracle's Eq. (cons) on the bases as stored (its own QR of every block,
    # rounded like the GPU's): xbar(0) and xbar(20) over all n rows and the
    # iterates of six machines.  Then, one step later, properties that hold at
    # any size: the master's update (Eq. (cons2)) recomputed in FP64 from the
    # machines' iterates, and every machine's step lying in the nullspace of
    # its block (Sec. 3.1: A_i (x_i(t+1) - x_i(t)) = gamma A_i P_i (...) = 0)
    # up to the precision of the stored basis.
    apc, dev = _apc(), _dev()
    if prec == "bf16":
        A, _, b = inputs.scaled_system_torch(n, 1234, dev)
        rnd = O.round_bf16
    else:
        A, _, b = inputs.gaussian_system_torch(n, 1235, dev)
        rnd = _f32
    offs = inputs.even_offsets(n, m)
    gam, eta, T = 1.0, 1.5, 20
    Ah, bh = A.cpu().numpy(), b.cpu().numpy()
    blocks = O.partition(Ah, bh, offs)
    QR = [O.block_qr(Ai) for Ai, _ in blocks]
    ref0 = _stored_basis_run([q for q, _ in QR], [r for _, r in QR], blocks, rnd, gam, eta, 0)
    ref = _stored_basis_run([q for q, _ in QR], [r for _, r in QR], blocks, rnd, gam, eta, T)
    del QR, blocks
    ctx = apc.apc_setup(A, b, offs, precision=prec)
    ctx.reset()
    assert _rel(ctx.xbar().cpu().numpy(), ref0.xbar) <= 1e-6, name
    ctx.iterate(gam, eta, T)
    assert _rel(ctx.xbar().cpu().numpy(), ref.xbar) <= 1e-5, name
    rng = np.random.default_rng(5)
    X = ctx.x().cpu().numpy()
    for i in rng.choice(m, 6, replace=False):
        assert _rel(X[i], ref.xs[i]) <= 1e-5, (name, int(i))
    del X, ref, ref0, Ah
    xs0, xb0 = ctx.x(), ctx.xbar().clone()
    ctx.iterate(gam, eta, 1)
    xs1, xb1 = ctx.x(), ctx.xbar()
    master = eta / m * xs1.sum(dim=0) + (1.0 - eta) * xb0
    assert float(torch.linalg.norm(xb1 - master) / torch.linalg.norm(xb1)) <= 1e-6, name
    tol = 2e-2 if prec == "bf16" else 1e-5
    for i in rng.choice(m, 6, replace=False):
        Ai = A[offs[i]:offs[i + 1]]
        dx = xs1[i] - xs0[i]
        ratio = float(torch.linalg.norm(Ai @ dx) / (torch.linalg.norm(Ai) * torch.linalg.norm(dx)))
        assert ratio <= tol, (name, int(i), ratio)


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
def test_setup_passes_and_orthogonality(prec):
    # FP64 contexts take both Cholesky-QR passes; FP32 / BF16 contexts keep a
    # first pass that the probe finds orthonormal far below their rounding,
    # and the stored basis is still orthonormal and spans the blocks' rows;
    # an ill-conditioned block (rows nearly dependent) makes the probe fail
    # and the second pass run
    apc, dev = _apc(), _dev()
    n, m = 600, 4
    A, _, b = inputs.gaussian_system(n, 71)
    offs = inputs.even_offsets(n, m)
    ctx = apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(b, device=dev), offs, precision=prec)
    rep = ctx.setup_report()
    if prec == "f64":
        assert rep["qr_passes"] == 2 and rep["orth_probe"] == -1.0
    else:
        assert rep["qr_passes"] == 1 and 0.0 <= rep["orth_probe"] <= 1e-11
    tol = {"f64": 1e-12, "f32": 1e-6, "bf16": 1e-2}[prec]
    for i, (Ai, _) in enumerate(O.partition(A, b, offs)):
        Q = ctx.basis(i).cpu().numpy()
        assert np.abs(Q.T @ Q - np.eye(Q.shape[1])).max() <= 4 * tol
        assert np.abs(np.eye(n) - Q @ Q.T - O.projector(Ai)).max() <= 4 * tol
    # nearly dependent rows: kappa(A_1) ~ 1e6, the first pass loses orthogonality
    A2 = A.copy()
    A2[1] = A2[0] + 1e-6 * A2[1]
    c2 = apc.apc_setup(torch.tensor(A2, device=dev), torch.tensor(b, device=dev), offs, precision=prec)
    if prec != "f64":
        assert c2.setup_report()["qr_passes"] == 2
    Q = c2.basis(0).cpu().numpy()
    assert np.abs(Q.T @ Q - np.eye(Q.shape[1])).max() <= 4 * tol
