"""Pins for the oracle's setup steps: partition, QR, projector, X, least-norm init.

Each check reaches the quantity by a second route (the paper's explicit
formula, a different LAPACK routine) or tests a property the paper states."""
import numpy as np
import pytest

from oracle import apc_oracle as O
from paper_1708_01413_gb300 import inputs


def _blocks(n=40, m=5, seed=0, N=None):
    A, x, b = inputs.gaussian_system(n, seed, N=N)
    offs = inputs.even_offsets(A.shape[0], m)
    return A, x, b, offs, O.partition(A, b, offs)


def test_partition_covers_rows_in_order():
    A, _, b, offs, blocks = _blocks(n=23, m=4)
    assert np.array_equal(np.vstack([a for a, _ in blocks]), A)
    assert np.array_equal(np.concatenate([bb for _, bb in blocks]), b)
    with pytest.raises(ValueError):
        O.partition(A, b, [0, 5, 5, 23])
    with pytest.raises(ValueError):
        O.partition(A, b, [0, 5, 22])


def test_projector_properties_sec31():
    # A_i P_i = 0 and P_i^2 = P_i (Sec. 3.1); P_i symmetric (orthogonal projector)
    _, _, _, _, blocks = _blocks()
    for A_i, _ in blocks:
        P = O.projector(A_i)
        assert np.abs(A_i @ P).max() <= 1e-12 * np.abs(A_i).max()
        assert np.abs(P @ P - P).max() <= 1e-12
        assert np.abs(P - P.T).max() <= 1e-13


def test_qr_route_equals_explicit_projector():
    _, _, _, _, blocks = _blocks(n=37, m=3, seed=3)
    for A_i, _ in blocks:
        Q, R = O.block_qr(A_i)
        assert np.abs(Q.T @ Q - np.eye(Q.shape[1])).max() <= 1e-13
        assert np.abs(np.eye(A_i.shape[1]) - Q @ Q.T - O.projector(A_i)).max() <= 1e-12
        assert np.abs(Q @ R - A_i.T).max() <= 1e-12 * np.abs(A_i).max()


def test_rank_deficient_block_rejected():
    A, _, b, offs, _ = _blocks(n=20, m=4)
    A = A.copy()
    A[1] = A[0]  # duplicate row inside block 0
    with pytest.raises(np.linalg.LinAlgError):
        O.block_qr(O.partition(A, b, offs)[0][0])


def test_least_norm_init_matches_lstsq():
    _, _, _, _, blocks = _blocks(n=31, m=4, seed=5)
    for A_i, b_i in blocks:
        Q, R = O.block_qr(A_i)
        x0 = O.least_norm_init(Q, R, b_i)
        ref = np.linalg.lstsq(A_i, b_i, rcond=None)[0]  # minimum-norm solution (SVD route)
        assert np.abs(x0 - ref).max() <= 1e-12 * np.abs(ref).max()
        assert np.abs(A_i @ x0 - b_i).max() <= 1e-12 * np.abs(b_i).max()


def test_x_matrix_identity_and_spectrum_sec32():
    # (1/m) sum_i P_i = I - X and 0 <= mu_min <= mu_max <= 1 (Sec. 3.2)
    _, _, _, _, blocks = _blocks(n=30, m=6, seed=2)
    QR = [O.block_qr(A_i) for A_i, _ in blocks]
    X = O.x_matrix([q for q, _ in QR])
    Pbar = sum(O.projector(A_i) for A_i, _ in blocks) / len(blocks)
    assert np.abs(Pbar - (np.eye(30) - X)).max() <= 1e-12
    # X also equals the definition with (A_i A_i^T)^{-1}
    Xdef = sum(A_i.T @ np.linalg.solve(A_i @ A_i.T, A_i) for A_i, _ in blocks) / len(blocks)
    assert np.abs(X - Xdef).max() <= 1e-12
    mu = np.linalg.eigvalsh(X)
    assert mu[0] >= -1e-14 and mu[-1] <= 1 + 1e-12
    lo, hi = O.mu_bounds([q for q, _ in QR])
    assert lo == pytest.approx(mu[0]) and hi == pytest.approx(mu[-1])


def test_one_block_gives_x_equal_identity():
    # m = 1 with a square nonsingular A: P_1 = 0, X = I
    A, _, b = inputs.gaussian_system(12, 9)
    Q, _ = O.block_qr(A)
    assert np.abs(O.x_matrix([Q]) - np.eye(12)).max() <= 1e-12


def test_power_mu_max_matches_eigvalsh():
    _, _, _, _, blocks = _blocks(n=40, m=5, seed=4)
    Qs = [O.block_qr(A_i)[0] for A_i, _ in blocks]
    lo, hi = O.mu_bounds(Qs)
    est = O.power_mu_max(Qs, np.random.default_rng(1).standard_normal(40), 400)
    assert est == pytest.approx(hi, rel=1e-6)


def test_partition_rows_arbitrary_sets():
    # Sec. 2: any assignment of the equations to machines; the APC limit is the
    # same solution (the method never uses the row order), and each block's
    # projector depends only on its set of rows
    import numpy as np
    from oracle import apc_oracle as O
    from paper_1708_01413_gb300 import inputs
    A, x_true, b = inputs.gaussian_system(60, 41)
    sets = [np.arange(i, 60, 4) for i in range(4)]  # round-robin, 15 rows each
    blocks = O.partition_rows(A, b, sets)
    for (Ai, bi), r in zip(blocks, sets):
        assert np.array_equal(Ai, A[r]) and np.array_equal(bi, b[r])
    # permuting the rows inside a set leaves the projector unchanged
    P1 = O.projector(blocks[0][0])
    P2 = O.projector(A[sets[0][::-1]])
    assert np.allclose(P1, P2, atol=1e-12)
    Qs = [O.block_qr(Ai)[0] for Ai, _ in blocks]
    g, e, _ = O.optimal_params(*O.mu_bounds(Qs))
    # gather the rows block by block and run on the contiguous system
    order = np.concatenate(sets)
    offs = np.concatenate([[0], np.cumsum([len(r) for r in sets])])
    tr = O.apc_run(A[order], b[order], offs, g, e, max_iters=20000, tol=1e-12)
    assert tr.converged
    assert np.linalg.norm(tr.xbar - x_true) <= 1e-9 * np.linalg.norm(x_true)
    with pytest.raises(ValueError):
        O.partition_rows(A, b, [np.arange(0, 30), np.arange(29, 60)])
