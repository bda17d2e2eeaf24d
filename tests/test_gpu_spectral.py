"""GPU Lanczos estimates of the extreme eigenvalues of X = (1/m) sum_i Q_i Q_i^T
(Eq. 3), checked against the oracle's exact eigenvalues (``numpy.linalg.eigvalsh``
of the oracle's own X)."""
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


def _bases(A, b, offs):
    return [O.block_qr(Ai)[0] for Ai, _ in O.partition(A, b, offs)]


def test_lanczos_recovers_both_ends_when_steps_reach_n():
    # k = n steps: the Ritz values are the whole spectrum up to rounding
    apc, dev = _apc(), _dev()
    A, _, b = inputs.gaussian_system(120, 31)
    offs = inputs.even_offsets(120, 4)
    lo, hi = O.mu_bounds(_bases(A, b, offs))
    ctx = apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(b, device=dev), offs, precision="f64")
    e_lo, e_hi = ctx.spectral_bounds(steps=120, seed=3)
    assert abs(e_hi - hi) <= 1e-9 * hi
    assert abs(e_lo - lo) <= 1e-6 * lo


def test_lanczos_ritz_values_lie_inside_and_mu_max_converges():
    apc, dev = _apc(), _dev()
    A, _, b = inputs.gaussian_system(1000, 32)
    offs = inputs.even_offsets(1000, 8)
    lo, hi = O.mu_bounds(_bases(A, b, offs))
    ctx = apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(b, device=dev), offs, precision="f64")
    e_lo, e_hi = ctx.spectral_bounds(steps=80, seed=5)
    assert e_hi <= hi * (1 + 1e-12)
    assert abs(e_hi - hi) <= 1e-8 * hi
    assert e_lo >= lo * (1 - 1e-9)
    assert e_lo < 0.5 * e_hi


def test_lanczos_on_bf16_bases_estimates_the_bf16_X():
    # the passes apply X built from the stored BF16 bases
    apc, dev = _apc(), _dev()
    A, _, b = inputs.gaussian_system(300, 33)
    offs = inputs.even_offsets(300, 6)
    Qr = [O.round_bf16(Q) for Q in _bases(A, b, offs)]
    mu = np.linalg.eigvalsh(sum(Q @ Q.T for Q in Qr) / len(Qr))
    ctx = apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(b, device=dev), offs, precision="bf16")
    e_lo, e_hi = ctx.spectral_bounds(steps=120, seed=7)
    # FP32 passes apply X with ~1e-7 absolute error
    assert abs(e_hi - mu[-1]) <= 1e-5 * mu[-1]
    assert e_lo >= mu[0] - 1e-6


def test_gpu_bounds_drive_a_solve_to_1e10():
    # Theorem 1's parameters from the GPU estimates (mu_min lowered by a
    # margin, mu_max raised, capped at 1) reach the tolerance
    apc, dev = _apc(), _dev()
    n, N, m = 512, 576, 9
    A, x_true, b = inputs.gaussian_system(n, 34, N=N)
    offs = inputs.even_offsets(N, m)
    At, bt = torch.tensor(A, device=dev), torch.tensor(b, device=dev)
    ctx = apc.apc_setup(At, bt, offs, precision="f64")
    e_lo, e_hi = ctx.spectral_bounds(steps=100, seed=9)
    g, e, rho = apc.apc_optimal_params(0.5 * e_lo, min(1.0, 1.01 * e_hi))
    x, st = ctx.solve(g, e, tol=1e-10, max_iters=200000, check_every=100)
    assert O.relative_residual(A, b, x.cpu().numpy()) <= 1e-10
    # against the oracle's exact parameters: at most a few times more iterations
    lo, hi = O.mu_bounds(_bases(A, b, offs))
    g0, e0, _ = O.optimal_params(lo, hi)
    x0, st0 = ctx.solve(g0, e0, tol=1e-10, max_iters=200000, check_every=100)
    assert st["iterations"] <= 4 * st0["iterations"] + 200


@pytest.mark.parametrize("prec", ["bf16", "f32"])
def test_lanczos_with_four_workers_per_warp(prec):
    # 32 blocks in one CTA with four workers per element warp (the automatic
    # choice for FP32/BF16 at 16 or more workers per CTA): the seed and power
    # passes of the generic pass modes against the exact spectrum of the X that
    # the stored bases define
    apc, dev = _apc(), _dev()
    n, m = 2048, 32
    A, _, b = inputs.gaussian_system(n, 35)
    offs = inputs.even_offsets(n, m)
    ctx = apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(b, device=dev), offs, precision=prec,
                        workers_per_warp=4)
    Qs = [ctx.basis(i).cpu().numpy() for i in range(m)]
    mu = np.linalg.eigvalsh(sum(Q @ Q.T for Q in Qs) / m)
    e_lo, e_hi = ctx.spectral_bounds(steps=150, seed=11)
    assert abs(e_hi - mu[-1]) <= 1e-5 * mu[-1]
    assert e_lo >= mu[0] - 1e-6  # inside the spectrum (the square system's mu_min converges slowly)
