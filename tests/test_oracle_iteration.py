"""Pins for the oracle's iteration (Eq. (cons), Algorithm 1), its analysis
(Theorem 1, App. A) and Proposition 1."""
import math

import numpy as np
import pytest
import scipy.optimize as so

from oracle import apc_oracle as O
from paper_1708_01413_gb300 import inputs


def _setup(n, m, seed, N=None):
    A, x_true, b = inputs.gaussian_system(n, seed, N=N)
    offs = inputs.even_offsets(A.shape[0], m)
    blocks = O.partition(A, b, offs)
    QR = [O.block_qr(A_i) for A_i, _ in blocks]
    return A, x_true, b, offs, blocks, [q for q, _ in QR], [r for _, r in QR]


def test_step_is_the_block_iteration_matrix_appA():
    # In error coordinates the step is the (m+1)n matrix of Eq. (matrix_recursion).
    A, _, b, offs, blocks, Qs, Rs = _setup(9, 3, 1)
    x_star = np.linalg.solve(A, b)
    g, e = 1.3, 4.2
    rng = np.random.default_rng(0)
    # feasible x_i (A_i x_i = b_i) and an arbitrary xbar
    xs = [x_star + (np.eye(9) - Q @ Q.T) @ rng.standard_normal(9) for Q in Qs]
    xbar = rng.standard_normal(9)
    new_xs, new_xbar = O.apc_step(xs, xbar, Qs, g, e)
    T = O.iteration_matrix([O.projector(A_i) for A_i, _ in blocks], g, e)
    err = np.concatenate([x - x_star for x in xs] + [xbar - x_star])
    pred = T @ err
    got = np.concatenate([x - x_star for x in new_xs] + [new_xbar - x_star])
    assert np.abs(pred - got).max() <= 1e-12 * np.abs(pred).max()


def test_brute_force_spectrum_matches_appA():
    # eigenvalues: 1-gamma with multiplicity (m-1)n, plus the roots of p_i (Eq. 5)
    A, _, b, offs, blocks, Qs, Rs = _setup(8, 3, 2)
    g, e = 1.15, 3.7
    T = O.iteration_matrix([O.projector(A_i) for A_i, _ in blocks], g, e)
    ev = np.sort_complex(np.linalg.eigvals(T))
    mus = np.linalg.eigvalsh(O.x_matrix(Qs))
    pred = [1 - g] * ((3 - 1) * 8)
    for mu in mus:
        pred += list(O.char_roots(mu, g, e))
    pred = np.sort_complex(np.array(pred, dtype=complex))
    # match as multisets
    used = np.zeros(len(pred), bool)
    for z in ev:
        d = np.abs(pred - z) + used * 1e9
        j = int(np.argmin(d))
        assert d[j] < 1e-6
        used[j] = True
    assert max(abs(ev)) == pytest.approx(O.apc_spectral_radius(mus, g, e, 3), rel=1e-8)


def test_invariant_every_iterate_solves_its_block():
    A, _, b, offs, blocks, Qs, Rs = _setup(60, 6, 3)
    mu_lo, mu_hi = O.mu_bounds(Qs)
    g, e, _ = O.optimal_params(mu_lo, mu_hi)
    tr = O.apc_run(A, b, offs, g, e, max_iters=300, record_every=50, Qs=Qs, Rs=Rs)
    assert max(h[3] for h in tr.history) <= 1e-12


def test_argmin_form_kkt_sec31():
    # x_i(t+1) = argmin ||x - xbar||^2 + (1-g)/g ||x - x_i(t)||^2 s.t. A_i x = b_i
    A, _, b, offs, blocks, Qs, Rs = _setup(14, 2, 4)
    rng = np.random.default_rng(7)
    for g in (0.6, 1.0, 1.7):
        xs = [O.least_norm_init(Q, R, bb) for Q, R, (_, bb) in zip(Qs, Rs, blocks)]
        xbar = rng.standard_normal(14)
        new_xs, _ = O.apc_step(xs, xbar, Qs, g, 2.0)
        c = (1 - g) / g
        for (A_i, b_i), x_i, new in zip(blocks, xs, new_xs):
            p = A_i.shape[0]
            K = np.block([[2 * (1 + c) * np.eye(14), A_i.T], [A_i, np.zeros((p, p))]])
            rhs = np.concatenate([2 * xbar + 2 * c * x_i, b_i])
            sol = np.linalg.solve(K, rhs)[:14]
            assert np.abs(sol - new).max() <= 1e-10 * np.abs(sol).max()


def test_prop1_cimmino_is_gamma_one():
    # Proposition 1: APC with gamma = 1, eta = m*nu reproduces block Cimmino
    A, _, b, offs, blocks, Qs, Rs = _setup(30, 5, 5)
    nu = 0.3
    tr_c = O.cimmino_run(A, b, offs, nu, np.zeros(30), 1)
    xs = [O.least_norm_init(Q, R, bb) for Q, R, (_, bb) in zip(Qs, Rs, blocks)]
    xbar = np.zeros(30)
    cims = O.cimmino_run(A, b, offs, nu, xbar, 25)
    for t in range(25):
        xs, xbar = O.apc_step(xs, xbar, Qs, 1.0, 5 * nu)
        assert np.abs(xbar - cims[t + 1]).max() <= 1e-11 * max(1.0, np.abs(cims[t + 1]).max())
    assert len(tr_c) == 2


def test_consensus_rate_gamma_eta_one():
    # gamma = eta = 1: rate 1 - mu_min (Table 1, "Consensus")
    A, _, b, offs, blocks, Qs, Rs = _setup(20, 4, 6)
    mus = np.linalg.eigvalsh(O.x_matrix(Qs))
    r = O.apc_spectral_radius(mus, 1.0, 1.0, 4)
    assert r == pytest.approx(O.rate_consensus(mus[0]), rel=1e-12)


def test_optimal_params_closed_form_vs_numeric_min():
    A, _, b, offs, blocks, Qs, Rs = _setup(12, 3, 7)
    mus = np.linalg.eigvalsh(O.x_matrix(Qs))
    g, e, rho = O.optimal_params(mus[0], mus[-1])
    # the optimality system of Theorem 1 holds
    r = math.sqrt((g - 1) * (e - 1))
    assert mus[-1] * e * g == pytest.approx((1 + r) ** 2, rel=1e-12)
    assert mus[0] * e * g == pytest.approx((1 - r) ** 2, rel=1e-10)
    assert rho == pytest.approx((math.sqrt(mus[-1] / mus[0]) - 1) / (math.sqrt(mus[-1] / mus[0]) + 1), rel=1e-12)
    assert 0 <= g <= 2
    # the spectral radius at the optimum is rho ...
    assert O.apc_spectral_radius(mus, g, e, 3) == pytest.approx(rho, rel=1e-6)
    # ... and no nearby (gamma, eta) does better (numeric minimisation from several starts)
    f = lambda v: O.apc_spectral_radius(mus, v[0], v[1], 3)
    best = min(so.minimize(f, x0, method="Nelder-Mead", options=dict(xatol=1e-10, fatol=1e-12, maxiter=4000)).fun
               for x0 in ([1.0, 2.0], [1.2, e * 0.8], [0.8, e * 1.3]))
    assert best >= rho - 1e-6


def test_swapped_params_leave_S():
    A, _, b, offs, blocks, Qs, Rs = _setup(12, 3, 8)
    mus = np.linalg.eigvalsh(O.x_matrix(Qs))
    g, e, rho = O.optimal_params(mus[0], mus[-1])
    assert O.apc_spectral_radius(mus, e, g, 3) > 1.0


def test_converges_to_lu_solution_and_observed_rate():
    # Algorithm 1 at the optimum reaches the LU solution; tail rate ~ rho (Theorem 1)
    n, m = 120, 6
    A, x_true, b, offs, blocks, Qs, Rs = _setup(n, m, 11)
    mus = np.linalg.eigvalsh(O.x_matrix(Qs))
    g, e, rho = O.optimal_params(mus[0], mus[-1])
    x_star = np.linalg.solve(A, b)
    tr = O.apc_run(A, b, offs, g, e, tol=1e-10, max_iters=200000, record_every=25,
                   x_star=x_star, Qs=Qs, Rs=Rs)
    assert tr.converged
    assert O.relative_residual(A, b, tr.xbar) <= 1e-10
    assert O.relative_error(tr.xbar, x_star) <= 1e-10 * np.linalg.cond(A)
    # fit the decay of the relative error over the second half of the run
    hist = [(t, re) for t, _, re, _ in tr.history if t >= tr.iters // 2 and re > 0]
    ts, es = np.array([h[0] for h in hist]), np.log([h[1] for h in hist])
    slope = np.polyfit(ts, es, 1)[0]
    ratio = slope / math.log(rho)
    assert 0.8 <= ratio <= 1.1


def test_general_params_in_S_converge_outside_diverge():
    A, _, b, offs, blocks, Qs, Rs = _setup(24, 4, 12)
    mus = np.linalg.eigvalsh(O.x_matrix(Qs))
    x_star = np.linalg.solve(A, b)
    for g, e in ((0.9, 1.5), (1.5, 3.0)):
        r = O.apc_spectral_radius(mus, g, e, 4)
        tr = O.apc_run(A, b, offs, g, e, max_iters=400, Qs=Qs, Rs=Rs)
        err = O.relative_error(tr.xbar, x_star)
        if r < 0.95:
            assert err < 1e-3
    # gamma outside [0, 2]: the (m-1)n-fold eigenvalue 1 - gamma (App. A) has
    # modulus 1.5.  Its eigenvectors have ebar = 0 and sum_i e_i = 0, so in exact
    # arithmetic they never reach xbar; the machines' iterates x_i blow up.
    tr = O.apc_run(A, b, offs, 2.5, 1.0, max_iters=120, Qs=Qs, Rs=Rs)
    assert max(O.relative_error(x, x_star) for x in tr.xs) > 1e3


def test_tall_system_and_uneven_blocks():
    # N > n (Sec. 2) with uneven contiguous blocks still converges to the solution
    rng = np.random.default_rng(3)
    A, x_true, b = inputs.gaussian_system(40, 13, N=90)
    offs = inputs.uneven_offsets(90, 8, 20, rng)
    blocks = O.partition(A, b, offs)
    Qs = [O.block_qr(A_i)[0] for A_i, _ in blocks]
    mus = np.linalg.eigvalsh(O.x_matrix(Qs))
    g, e, rho = O.optimal_params(mus[0], mus[-1])
    tr = O.apc_run(A, b, offs, g, e, tol=1e-10, max_iters=20000, record_every=10)
    assert tr.converged
    assert O.relative_error(tr.xbar, x_true) <= 1e-8


def test_initialisation_does_not_change_limit():
    # Sec. 5 remark: any feasible x_i(0) works; xbar(0) = 0 also works
    A, x_true, b, offs, blocks, Qs, Rs = _setup(40, 4, 14)
    mus = np.linalg.eigvalsh(O.x_matrix(Qs))
    g, e, _ = O.optimal_params(mus[0], mus[-1])
    rng = np.random.default_rng(2)
    xs0 = [O.least_norm_init(Q, R, bb) + (np.eye(40) - Q @ Q.T) @ rng.standard_normal(40)
           for Q, R, (_, bb) in zip(Qs, Rs, blocks)]
    tr = O.apc_run(A, b, offs, g, e, tol=1e-10, max_iters=50000, record_every=10, xs0=xs0,
                   xbar0=np.zeros(40), Qs=Qs, Rs=Rs)
    assert tr.converged and O.relative_error(tr.xbar, x_true) <= 1e-8
