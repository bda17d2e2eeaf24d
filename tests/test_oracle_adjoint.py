"""Pins for the oracle's reverse sweep through T unrolled iterations of Eq. (cons).

b -> xbar(T) is linear, so for L = 0.5 ||xbar(T) - x_target||^2 a central
finite difference in b is exact up to rounding for any step; at convergence
the gradient tends to A^{-T}(xbar - x_target)."""
import numpy as np
import pytest

from oracle import apc_oracle as O
from paper_1708_01413_gb300 import inputs


def _setup(n, m, seed, k=1):
    A, _, b = inputs.gaussian_system(n, seed, k=k)
    offs = inputs.even_offsets(n, m)
    blocks = O.partition(A, b, offs)
    QR = [O.block_qr(A_i) for A_i, _ in blocks]
    Qs, Rs = [q for q, _ in QR], [r for _, r in QR]
    mus = np.linalg.eigvalsh(O.x_matrix(Qs))
    g, e, rho = O.optimal_params(mus[0], mus[-1])
    return A, b, offs, blocks, Qs, Rs, g, e


def _loss(A, b, offs, Qs, Rs, g, e, T, xt):
    blocks = O.partition(A, b, offs)
    xbar, _, _ = O.apc_forward_linear(blocks, Qs, Rs, g, e, T)
    return 0.5 * float(np.sum((xbar - xt) ** 2))


@pytest.mark.parametrize("k", [1, 3])
def test_grad_b_matches_central_difference(k):
    A, b, offs, blocks, Qs, Rs, g, e = _setup(30, 5, 1, k=k)
    T = 40
    xt = inputs.target_vector(30, 1, k=k)
    xbar, _, states = O.apc_forward_linear(blocks, Qs, Rs, g, e, T)
    db, _, _ = O.apc_adjoint(blocks, Qs, Rs, g, e, T, xbar - xt)
    db = np.concatenate(db)
    rng = np.random.default_rng(5)
    for _ in range(3):
        d = rng.standard_normal(b.shape)
        h = 1e-2 * np.linalg.norm(b)
        fd = (_loss(A, b + h * d, offs, Qs, Rs, g, e, T, xt) - _loss(A, b - h * d, offs, Qs, Rs, g, e, T, xt)) / (2 * h)
        assert float(np.sum(db * d)) == pytest.approx(fd, rel=1e-9, abs=1e-12)


def test_adjoint_is_transpose_dot_product():
    # <J db, w> = <db, J^T w> for the linear map b -> xbar(T)
    A, b, offs, blocks, Qs, Rs, g, e = _setup(24, 4, 2)
    T = 25
    rng = np.random.default_rng(3)
    v = rng.standard_normal(24)
    w = rng.standard_normal(24)
    Jv, _, _ = O.apc_forward_linear(O.partition(A, v, offs), Qs, Rs, g, e, T)
    JTw, _, _ = O.apc_adjoint(blocks, Qs, Rs, g, e, T, w)
    assert float(Jv @ w) == pytest.approx(float(np.concatenate(JTw) @ v), rel=1e-11)


def test_grad_gamma_eta_match_central_difference():
    A, b, offs, blocks, Qs, Rs, g, e = _setup(20, 4, 3)
    T = 30
    xt = inputs.target_vector(20, 3)
    xbar, _, states = O.apc_forward_linear(blocks, Qs, Rs, g, e, T)
    _, dg, de = O.apc_adjoint(blocks, Qs, Rs, g, e, T, xbar - xt, states=states)
    h = 1e-6
    fdg = (_loss(A, b, offs, Qs, Rs, g + h, e, T, xt) - _loss(A, b, offs, Qs, Rs, g - h, e, T, xt)) / (2 * h)
    fde = (_loss(A, b, offs, Qs, Rs, g, e + h, T, xt) - _loss(A, b, offs, Qs, Rs, g, e - h, T, xt)) / (2 * h)
    assert dg == pytest.approx(fdg, rel=1e-5)
    assert de == pytest.approx(fde, rel=1e-5)


def test_grad_b_tends_to_inverse_transpose_at_convergence():
    A, b, offs, blocks, Qs, Rs, g, e = _setup(40, 4, 4)
    tr = O.apc_run(A, b, offs, g, e, tol=1e-13, max_iters=100000, record_every=20, Qs=Qs, Rs=Rs)
    T = tr.iters
    xt = inputs.target_vector(40, 4)
    xbar, _, _ = O.apc_forward_linear(blocks, Qs, Rs, g, e, T)
    gT = xbar - xt
    db, _, _ = O.apc_adjoint(blocks, Qs, Rs, g, e, T, gT)
    ref = np.linalg.solve(A.T, gT)
    assert np.linalg.norm(np.concatenate(db) - ref) <= 1e-7 * np.linalg.norm(ref)
