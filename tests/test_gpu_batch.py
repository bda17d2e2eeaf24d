"""GPU parity of the batched solver (include/apc_batch.h) against the FP64 oracle.

The batched kernel stores every basis Q_i in BF16 and computes the machines'
update in the form of App. A (x_i <- x_i + gamma (xbar - x_i - Q_i (Q_i^T xbar
- c_i))).  The oracle therefore runs ``apc_run_affine`` on the BF16-rounded
bases of its own FP64 QR (``round_bf16``), with the coefficients c_i in FP64.

Tolerance.  A vectorised model of the kernel's rounding (FP32 iterates, BF16
operand planes holding 16 / 24 significant bits, double-float master) differs
from that FP64 trajectory by 5e-6 .. 1.2e-5 (relative, Frobenius) after 20-40
iterations on these workloads (n 257..1000, k 4..32, optimal parameters); the
tests allow 1e-4.  Against the exact-basis trajectory of Eq. (cons) the BF16
rounding of Q_i (relative 2^-8) dominates, checked at 5e-2 like the
single-system BF16 path.
"""
import numpy as np
import pytest

from oracle import apc_oracle as O
from paper_1708_01413_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-4


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


def _oracle_system(A, B, offs):
    blocks = O.partition(A, B, offs)
    QR = [O.block_qr(Ai) for Ai, _ in blocks]
    Qs, Rs = [q for q, _ in QR], [r for _, r in QR]
    cs = [O.block_coefficients(Q, R, bi) for Q, R, (_, bi) in zip(Qs, Rs, blocks)]
    return Qs, Rs, cs


def _systems(sizes, k, seed, p_lo=16, p_hi=128):
    rng = np.random.default_rng(seed)
    out = []
    for n in sizes:
        A = rng.standard_normal((n, n)) + 0.5 * np.sqrt(n) * np.eye(n)
        B = rng.standard_normal((n, k))
        offs = inputs.uneven_offsets(n, min(p_lo, n - 1), min(p_hi, n - 1), rng)
        out.append((A, B, offs))
    return out


# sizes: n < 32 (one padded tile), a single 16-row block remainder, several
# 256-row sweep-A units, several 512-column sweep-B units; k covers one and two
# 16-wide right-hand-side tiles and a ragged count
@pytest.mark.parametrize("k", [5, 20, 32])
def test_batch_matches_affine_oracle_on_bf16_bases(k):
    apc, dev = _apc(), _dev()
    systems = _systems([20, 77, 300, 613], k, seed=10 + k)
    params, refs = [], []
    T = 20
    for A, B, offs in systems:
        Qs, Rs, cs = _oracle_system(A, B, offs)
        g, e, _ = O.optimal_params(*O.mu_bounds(Qs))
        params.append((g, e))
        refs.append(O.apc_run_affine([O.round_bf16(Q) for Q in Qs], cs, g, e, T))
    bt = apc.apc_batch_setup([torch.tensor(A, device=dev) for A, _, _ in systems],
                             [torch.tensor(B, device=dev) for _, B, _ in systems],
                             [offs for _, _, offs in systems])
    bt.set_params([p[0] for p in params], [p[1] for p in params])
    bt.reset()
    # the initialisation alone: x_i(0) = Q_i c_i and their mean
    for s, (A, B, offs) in enumerate(systems):
        Qs, Rs, cs = _oracle_system(A, B, offs)
        Qr = [O.round_bf16(Q) for Q in Qs]
        x0 = sum(Q @ c for Q, c in zip(Qr, cs)) / len(Qr)
        assert _rel(bt.xbar(s).cpu().numpy(), x0) <= 1e-5
    bt.iterate(T)
    for s, (xs_ref, xbar_ref) in enumerate(refs):
        assert _rel(bt.xbar(s).cpu().numpy(), xbar_ref) <= TOL, s
        for i in (0, len(xs_ref) - 1):
            assert _rel(bt.x(s, i).cpu().numpy(), xs_ref[i]) <= TOL, (s, i)


def test_batch_close_to_exact_basis_trajectory():
    # Eq. (cons) with the FP64 bases: the BF16 rounding of Q_i dominates
    apc, dev = _apc(), _dev()
    systems = _systems([200, 350], 8, seed=3)
    refs, params = [], []
    T = 20
    for A, B, offs in systems:
        Qs, Rs, _ = _oracle_system(A, B, offs)
        g, e, _ = O.optimal_params(*O.mu_bounds(Qs))
        params.append((g, e))
        refs.append(O.apc_run(A, B, offs, g, e, max_iters=T, Qs=Qs, Rs=Rs).xbar)
    bt = apc.apc_batch_setup([torch.tensor(A, device=dev) for A, _, _ in systems],
                             [torch.tensor(B, device=dev) for _, B, _ in systems],
                             [offs for _, _, offs in systems])
    bt.set_params([p[0] for p in params], [p[1] for p in params])
    bt.reset()
    bt.iterate(T)
    for s, ref in enumerate(refs):
        assert _rel(bt.xbar(s).cpu().numpy(), ref) <= 5e-2


def test_batch_converges_to_the_bf16_fixed_point():
    # The limit of the affine iteration on BF16 bases solves
    # (sum_i Q_i Q_i^T) x = sum_i Q_i c_i (closed form, solved on the host).
    apc, dev = _apc(), _dev()
    rng = np.random.default_rng(21)
    n, k = 96, 3
    A = rng.standard_normal((n, n)) + 2.0 * np.sqrt(n) * np.eye(n)
    B = rng.standard_normal((n, k))
    offs = inputs.uneven_offsets(n, 16, 40, rng)
    Qs, Rs, cs = _oracle_system(A, B, offs)
    Qr = [O.round_bf16(Q) for Q in Qs]
    x_fp = np.linalg.solve(sum(Q @ Q.T for Q in Qr), sum(Q @ c for Q, c in zip(Qr, cs)))
    g, e, rho = O.optimal_params(*O.mu_bounds(Qs))
    T = int(np.ceil(np.log(1e-9) / np.log(rho))) + 50
    bt = apc.apc_batch_setup([torch.tensor(A, device=dev)], [torch.tensor(B, device=dev)], [offs])
    bt.set_params([g], [e])
    bt.reset()
    bt.iterate(T)
    assert _rel(bt.xbar(0).cpu().numpy(), x_fp) <= 1e-5


def test_batch_graph_replay_is_deterministic():
    # no atomics on the path: 10 iterations at once equal 5 + 5, bit for bit
    apc, dev = _apc(), _dev()
    systems = _systems([150, 400], 32, seed=4)
    As = [torch.tensor(A, device=dev) for A, _, _ in systems]
    Bs = [torch.tensor(B, device=dev) for _, B, _ in systems]
    bt = apc.apc_batch_setup(As, Bs, [o for _, _, o in systems])
    bt.set_params([1.2, 1.1], [1.5, 2.0])
    bt.reset()
    bt.iterate(10)
    a = [bt.xbar(s).cpu() for s in range(2)]
    bt.reset()
    bt.iterate(5)
    bt.iterate(5)
    b = [bt.xbar(s).cpu() for s in range(2)]
    for u, v in zip(a, b):
        assert torch.equal(u, v)
    # new right-hand sides through reset
    Bs2 = [2.0 * B for B in Bs]
    bt.reset(Bs2)
    bt.iterate(10)
    for s in range(2):
        assert torch.allclose(bt.xbar(s).cpu(), 2.0 * a[s], rtol=1e-5, atol=1e-6)


def test_batch_timeout_hook_reports_and_recovers():
    apc, dev = _apc(), _dev()
    systems = _systems([100, 64], 4, seed=5)
    bt = apc.apc_batch_setup([torch.tensor(A, device=dev) for A, _, _ in systems],
                             [torch.tensor(B, device=dev) for _, B, _ in systems],
                             [o for _, _, o in systems])
    bt.set_params([1.0, 1.0], [1.0, 1.0])
    bt.reset()
    bt.iterate(3)
    good = [bt.xbar(s).cpu() for s in range(2)]
    bt.set_test_hooks(grid_barrier_skew=1, timeout_s=0.2)
    with pytest.raises(apc.ApcError) as ei:
        bt.iterate(3)
    assert ei.value.name == "TIMEOUT"
    bt.set_test_hooks(0, 0.0)
    bt.reset()
    bt.iterate(3)
    for s in range(2):
        assert torch.equal(bt.xbar(s).cpu(), good[s])


def test_batch_errors_reported():
    apc, dev = _apc(), _dev()
    A, B, offs = _systems([64], 4, seed=6)[0]
    At, Bt = torch.tensor(A, device=dev), torch.tensor(B, device=dev)
    with pytest.raises(apc.ApcError) as ei:
        apc.apc_batch_setup([At], [torch.zeros((64, 33), dtype=torch.float64, device=dev)], [offs])
    assert ei.value.name == "UNSUPPORTED"
    with pytest.raises(apc.ApcError) as ei:
        apc.apc_batch_setup([At], [Bt], [[0, 10, 60]])
    assert ei.value.name == "INVALID_ARG"
    A2 = A.copy()
    A2[1] = A2[0]
    with pytest.raises(apc.ApcError) as ei:
        apc.apc_batch_setup([torch.tensor(A2, device=dev)], [Bt], [offs])
    assert ei.value.name == "SINGULAR_BLOCK"
    bt = apc.apc_batch_setup([At], [Bt], [offs])
    bt.reset()
    with pytest.raises(apc.ApcError) as ei:
        bt.iterate(2)
    assert ei.value.name == "PARAMS"
    with pytest.raises(apc.ApcError) as ei:
        bt.set_params([2.5], [1.0])
    assert ei.value.name == "PARAMS"


def test_batch_full_workload_sampled_parity():
    # 256 systems, n uniform in [256, 4096], blocks p_i uniform in [16, 128],
    # k = 32: built on the device; a few systems are copied back and checked
    # against the oracle.  (gamma, eta) = (1, 1) lies in the set S of
    # Theorem 1 for every system.
    apc, dev = _apc(), _dev()
    specs = inputs.batch_specs(256, seed=2024)
    As, Bs, offs = inputs.batch_systems_torch(specs, seed=2024, device=dev)
    bt = apc.apc_batch_setup(As, Bs, offs)
    info = bt.info()
    assert info["nsys"] == 256 and info["k"] == 32
    bt.set_params([1.0] * 256, [1.0] * 256)
    bt.reset()
    T = 8
    bt.iterate(T)
    ns = [n for n, _ in specs]
    sample = sorted({int(np.argmin(ns)), int(np.argmax(ns)), int(np.argsort(ns)[len(ns) // 2])})
    for s in sample:
        A, B = As[s].cpu().numpy(), Bs[s].cpu().numpy()
        Qs, Rs, cs = _oracle_system(A, B, offs[s])
        _, ref = O.apc_run_affine([O.round_bf16(Q) for Q in Qs], cs, 1.0, 1.0, T)
        assert _rel(bt.xbar(s).cpu().numpy(), ref) <= TOL, s


@pytest.mark.parametrize("k", [5, 20])
def test_batch_heavy_ball_matches_oracle_dhbm(k):
    # Sec. 6 preconditioned D-HBM: gradient sum_i Q_i (Q_i^T x - c_i) on the
    # BF16 bases, started from xbar(0) with zero momentum
    apc, dev = _apc(), _dev()
    systems = _systems([90, 300], k, seed=40 + k)
    T = 20
    refs, params = [], []
    for A, B, offs in systems:
        Qs, Rs, cs = _oracle_system(A, B, offs)
        lo, hi = O.mu_bounds(Qs)
        alpha, beta, _ = O.hb_optimal_params(len(Qs) * lo, len(Qs) * hi)
        params.append((alpha, beta))
        Qr = [O.round_bf16(Q) for Q in Qs]
        x0 = sum(Q @ c for Q, c in zip(Qr, cs)) / len(Qr)
        refs.append(O.dhbm_run([(Q.T, c) for Q, c in zip(Qr, cs)], x0, alpha, beta, T))
    bt = apc.apc_batch_setup([torch.tensor(A, device=dev) for A, _, _ in systems],
                             [torch.tensor(B, device=dev) for _, B, _ in systems],
                             [offs for _, _, offs in systems])
    bt.set_hb_params([p[0] for p in params], [p[1] for p in params])
    bt.reset()
    bt.iterate(T)
    for s, ref in enumerate(refs):
        assert _rel(bt.xbar(s).cpu().numpy(), ref) <= TOL, s
    # back to APC: the same batch reproduces the APC trajectory
    refs_apc = []
    for (A, B, offs) in systems:
        Qs, Rs, cs = _oracle_system(A, B, offs)
        g, e, _ = O.optimal_params(*O.mu_bounds(Qs))
        refs_apc.append((g, e, O.apc_run_affine([O.round_bf16(Q) for Q in Qs], cs, g, e, T)[1]))
    bt.set_params([r[0] for r in refs_apc], [r[1] for r in refs_apc])
    bt.reset()
    bt.iterate(T)
    for s, (_, _, ref) in enumerate(refs_apc):
        assert _rel(bt.xbar(s).cpu().numpy(), ref) <= TOL, s


def test_batch_heavy_ball_reaches_the_bf16_fixed_point():
    # heavy ball on C x = d with C_i = Q_i^T, d_i = c_i solves the normal
    # equations (sum_i Q_i Q_i^T) x = sum_i Q_i c_i: the same limit as APC
    apc, dev = _apc(), _dev()
    rng = np.random.default_rng(22)
    n, k = 96, 3
    A = rng.standard_normal((n, n)) + 2.0 * np.sqrt(n) * np.eye(n)
    B = rng.standard_normal((n, k))
    offs = inputs.uneven_offsets(n, 16, 40, rng)
    Qs, Rs, cs = _oracle_system(A, B, offs)
    Qr = [O.round_bf16(Q) for Q in Qs]
    x_fp = np.linalg.solve(sum(Q @ Q.T for Q in Qr), sum(Q @ c for Q, c in zip(Qr, cs)))
    lo, hi = O.mu_bounds(Qs)
    alpha, beta, rho = apc.apc_hb_optimal_params(lo, hi, len(Qs))
    T = int(np.ceil(np.log(1e-9) / np.log(rho))) + 100
    bt = apc.apc_batch_setup([torch.tensor(A, device=dev)], [torch.tensor(B, device=dev)], [offs])
    bt.set_hb_params([alpha], [beta])
    bt.reset()
    bt.iterate(T)
    assert _rel(bt.xbar(0).cpu().numpy(), x_fp) <= 1e-5


@pytest.mark.parametrize("seed", [101, 102, 103])
def test_batch_random_shapes_match_oracle(seed):
    # random mixes: tiny and mid-size systems, blocks from 1 row up to 128 rows
    # (widths that are and are not multiples of 8 and 16), ragged k
    apc, dev = _apc(), _dev()
    rng = np.random.default_rng(seed)
    k = int(rng.choice([1, 3, 16, 17, 32]))
    systems = []
    for _ in range(int(rng.integers(2, 6))):
        n = int(rng.integers(17, 700))
        A = rng.standard_normal((n, n)) + np.sqrt(n) * np.eye(n)
        B = rng.standard_normal((n, k))
        offs = inputs.uneven_offsets(n, 1, min(128, n - 1), rng)
        systems.append((A, B, offs))
    T = 10
    refs, params = [], []
    for A, B, offs in systems:
        Qs, Rs, cs = _oracle_system(A, B, offs)
        g, e, _ = O.optimal_params(*O.mu_bounds(Qs))
        params.append((g, e))
        refs.append(O.apc_run_affine([O.round_bf16(Q) for Q in Qs], cs, g, e, T)[1])
    bt = apc.apc_batch_setup([torch.tensor(A, device=dev) for A, _, _ in systems],
                             [torch.tensor(B, device=dev) for _, B, _ in systems],
                             [offs for _, _, offs in systems])
    bt.set_params([p[0] for p in params], [p[1] for p in params])
    bt.reset()
    bt.iterate(T)
    for s, ref in enumerate(refs):
        assert _rel(bt.xbar(s).cpu().numpy().reshape(ref.shape), ref) <= TOL, (s, k)


def test_batch_results_independent_of_batch_composition():
    # A unit computes from its own system's data only, in a fixed order, so a
    # system's iterates are bit-identical whether it runs alone, in a batch,
    # or in the same batch listed in reverse order.  The claim order, the
    # CTAs that take each unit and the waits between units all change with
    # the batch; a unit that read an input before the units writing it had
    # completed would break the equality.
    apc, dev = _apc(), _dev()
    rng = np.random.default_rng(77)
    sizes = [int(x) for x in rng.integers(17, 900, size=24)]
    systems = _systems(sizes, 7, seed=78)
    T = 12

    def run(idx):
        bt = apc.apc_batch_setup([torch.tensor(systems[i][0], device=dev) for i in idx],
                                 [torch.tensor(systems[i][1], device=dev) for i in idx],
                                 [systems[i][2] for i in idx])
        bt.set_params([1.0] * len(idx), [1.0] * len(idx))
        bt.reset()
        bt.iterate(T)
        out = {i: bt.xbar(j).cpu() for j, i in enumerate(idx)}
        bt.close()
        return out

    fwd = run(list(range(len(systems))))
    rev = run(list(reversed(range(len(systems)))))
    for i in range(len(systems)):
        assert torch.isfinite(fwd[i]).all(), i
        assert torch.equal(fwd[i], rev[i]), i
    for i in (0, 11, 23):
        assert torch.equal(run([i])[i], fwd[i]), i
