"""Pins of the rate formulas of Table 1 (Sec. 4) used to reproduce the synthetic
rows of Table 2 (Sec. 5), and of the modified ADMM of Sec. 4.4."""
import math

import numpy as np
import pytest

from oracle import apc_oracle as O
from paper_1708_01413_gb300 import inputs


def _radius(M):
    return float(np.abs(np.linalg.eigvals(M)).max())


def test_dgd_rate_is_the_spectral_radius_at_the_optimal_step():
    rng = np.random.default_rng(71)
    A = rng.standard_normal((40, 12))
    H = A.T @ A
    lam = np.linalg.eigvalsh(H)
    alpha = 2.0 / (lam[0] + lam[-1])
    assert _radius(np.eye(12) - alpha * H) == pytest.approx(O.rate_dgd(lam[-1] / lam[0]), rel=1e-9)


def test_dnag_rate_is_the_worst_two_by_two_radius():
    # per eigenvalue lam the D-NAG update of Sec. 4.2 acts on (y(t+1), y(t)) as
    # [[(1 - a lam)(1 + b), -(1 - a lam) b], [1, 0]]; with the tuning
    # a = 4/(3L + l), b = (sqrt(3 kappa + 1) - 2)/(sqrt(3 kappa + 1) + 2)
    # the worst radius over [l, L] is the rate Sec. 4.2 quotes
    l, L = 0.02, 3.0
    k = L / l
    a = 4.0 / (3.0 * L + l)
    q = math.sqrt(3.0 * k + 1.0)
    b = (q - 2.0) / (q + 2.0)
    worst = max(_radius(np.array([[(1 - a * x) * (1 + b), -(1 - a * x) * b], [1.0, 0.0]]))
                for x in np.linspace(l, L, 2001))
    assert worst == pytest.approx(O.rate_dnag(k), rel=1e-4)


def test_dhbm_rate_formula_equals_the_heavy_ball_radius():
    l, L = 0.05, 2.0
    _, _, rho = O.hb_optimal_params(l, L)
    assert O.rate_dhbm(L / l) == pytest.approx(rho, rel=1e-12)


def test_madmm_rate_matches_its_iteration_and_the_optimum():
    A, x_true, b = inputs.gaussian_system(30, 72)
    offs = inputs.even_offsets(30, 3)
    blocks = O.partition(A, b, offs)
    xi = 5.0
    r = O.madmm_rate(blocks, xi)
    xbar = np.zeros(30)
    errs = []
    for _ in range(400):
        xbar = O.madmm_step(blocks, xbar, xi)
        errs.append(np.linalg.norm(xbar - x_true))
    obs = (errs[-1] / errs[199]) ** (1.0 / 200)
    assert obs == pytest.approx(r, rel=1e-3)
    # the rate grows with xi and tends to the consensus rate 1 - mu_min(X)
    rates = [O.madmm_rate(blocks, 10.0 ** e) for e in (-3, -1, 0, 1, 3)]
    assert all(r1 <= r2 + 1e-12 for r1, r2 in zip(rates, rates[1:]))
    Qs = [O.block_qr(Ai)[0] for Ai, _ in blocks]
    mu_lo, _ = O.mu_bounds(Qs)
    xi_opt, r_opt = O.madmm_optimal_rate(blocks)
    assert r_opt == pytest.approx(O.rate_consensus(mu_lo), abs=1e-8)


def test_table2_synthetic_row_claims():
    # "Standard Gaussian (500 x 500)" of Table 2 with m = 10 blocks of 50 (the
    # paper does not state m): APC has the smallest convergence time, block
    # Cimmino's is about 2 T_APC^2, and T_APC is of the order the paper prints
    A, _, b = inputs.gaussian_system(500, 0)
    row = O.table2_row(A, b, inputs.even_offsets(500, 10))
    methods = ("DGD", "D-NAG", "D-HBM", "M-ADMM", "B-Cimmino", "APC")
    assert min(methods, key=lambda k: row[k]) == "APC"
    assert row["B-Cimmino"] == pytest.approx(2.0 * row["APC"] ** 2, rel=0.01)
    assert 0.3 <= row["APC"] / 2.70e3 <= 3.0


def _paper_row(name):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "table2_convergence_times.txt")
    for line in open(path):
        if line.startswith(name):
            return [float(v) for v in line.split()[1:]]
    raise KeyError(name)


def test_table2_tall_gaussian_row_matches_the_printed_values():
    # "Standard Tall Gaussian (1000 x 500)": the spectra of a tall Gaussian
    # concentrate, so one instance (m = 10 blocks of 100) reproduces every
    # printed convergence time of the row within 10 %
    A, _, b = inputs.gaussian_system(500, 0, N=1000)
    row = O.table2_row(A, b, inputs.even_offsets(1000, 10))
    printed = dict(zip(("DGD", "D-NAG", "D-HBM", "M-ADMM", "B-Cimmino", "APC"), _paper_row("Standard_Tall_Gaus")))
    for k, v in printed.items():
        assert row[k] == pytest.approx(v, rel=0.10), k
