"""Pins of the distributed-preconditioned heavy-ball method (Sec. 4.3 update,
Sec. 6 preconditioning) in the oracle."""
import numpy as np
import pytest

from oracle import apc_oracle as O
from paper_1708_01413_gb300 import inputs


def _case(n=80, m=4, seed=61):
    A, x_true, b = inputs.gaussian_system(n, seed)
    offs = inputs.even_offsets(n, m)
    blocks = O.partition(A, b, offs)
    QR = [O.block_qr(Ai) for Ai, _ in blocks]
    return A, x_true, b, offs, blocks, [q for q, _ in QR], [r for _, r in QR]


def test_preconditioned_rows_are_orthonormal_and_CtC_is_mX():
    A, x_true, b, offs, blocks, Qs, Rs = _case()
    pb = O.precondition_blocks(blocks)
    for C_i, _ in pb:
        assert np.allclose(C_i @ C_i.T, np.eye(C_i.shape[0]), atol=1e-10)
    CtC = sum(C.T @ C for C, _ in pb)
    assert np.allclose(CtC, len(pb) * O.x_matrix(Qs), atol=1e-10)


def test_preconditioned_gradient_equals_the_basis_form():
    # C_i^T (C_i x - d_i) = Q_i (Q_i^T x - c_i): any orthonormal basis of the
    # row space gives the same gradient (Sec. 6 premultiplies by (A_i A_i^T)^{-1/2})
    A, x_true, b, offs, blocks, Qs, Rs = _case(seed=62)
    pb = O.precondition_blocks(blocks)
    x = np.random.default_rng(1).standard_normal(A.shape[1])
    for (C, d), Q, R, (_, bi) in zip(pb, Qs, Rs, blocks):
        c = O.block_coefficients(Q, R, bi)
        assert np.allclose(C.T @ (C @ x - d), Q @ (Q.T @ x - c), atol=1e-9 * np.linalg.norm(x))


def test_hb_parameters_give_rate_rho_on_every_eigenvalue():
    # brute force: the 2 x 2 iteration matrix of heavy ball on one eigen-direction
    L_min, L_max = 0.03, 2.5
    alpha, beta, rho = O.hb_optimal_params(L_min, L_max)
    radii = []
    for lam in np.linspace(L_min, L_max, 401):
        M = np.array([[1.0 + beta - alpha * lam, -beta], [1.0, 0.0]])
        radii.append(np.abs(np.linalg.eigvals(M)).max())
    assert max(radii) == pytest.approx(rho, rel=1e-6)
    k = L_max / L_min
    assert rho == pytest.approx((np.sqrt(k) - 1) / (np.sqrt(k) + 1), rel=1e-12)


def test_dhbm_converges_at_the_apc_rate():
    # Sec. 6: the preconditioned D-HBM attains (sqrt(kappa(X)) - 1)/(sqrt(kappa(X)) + 1)
    A, x_true, b, offs, blocks, Qs, Rs = _case(n=60, m=3, seed=63)
    pb = O.precondition_blocks(blocks)
    lo, hi = O.mu_bounds(Qs)
    m = len(Qs)
    alpha, beta, rho = O.hb_optimal_params(m * lo, m * hi)
    g, e, rho_apc = O.optimal_params(lo, hi)
    assert rho == pytest.approx(rho_apc, rel=1e-10)
    x = np.zeros(A.shape[1])
    z = np.zeros_like(x)
    errs = []
    for t in range(6000):
        x, z = O.dhbm_step(pb, x, z, alpha, beta)
        errs.append(np.linalg.norm(x - x_true) / np.linalg.norm(x_true))
        if errs[-1] < 1e-11:
            break
    assert errs[-1] < 1e-10
    # tail rate against rho (the double root makes early decay slower)
    t1 = len(errs) - 1
    t0 = t1 // 2
    obs = (errs[t1] / errs[t0]) ** (1.0 / (t1 - t0))
    assert 0.8 <= np.log(obs) / np.log(rho) <= 1.1
    # the same limit as APC
    tr = O.apc_run(A, b, offs, g, e, max_iters=200000, tol=1e-12)
    assert np.linalg.norm(tr.xbar - x) <= 1e-9 * np.linalg.norm(x_true)


def test_dhbm_basis_form_gives_the_same_iterates():
    A, x_true, b, offs, blocks, Qs, Rs = _case(seed=64)
    pb = O.precondition_blocks(blocks)
    qb = [(Q.T, O.block_coefficients(Q, R, bi)) for Q, R, (_, bi) in zip(Qs, Rs, blocks)]
    x0 = np.random.default_rng(2).standard_normal(A.shape[1])
    lo, hi = O.mu_bounds(Qs)
    alpha, beta, _ = O.hb_optimal_params(len(Qs) * lo, len(Qs) * hi)
    xa = O.dhbm_run(pb, x0, alpha, beta, 50)
    xq = O.dhbm_run(qb, x0, alpha, beta, 50)
    assert np.linalg.norm(xa - xq) <= 1e-9 * np.linalg.norm(xa)
