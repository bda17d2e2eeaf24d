"""Pins of the oracle's BF16 rounding and of the affine (App. A) form of the
machines' update, which the batched solver computes on BF16-stored bases."""
import numpy as np
import pytest

from oracle import apc_oracle as O
from paper_1708_01413_gb300 import inputs


def test_round_bf16_exact_values_and_ties_to_even():
    exact = np.array([1.0, 1.5, -0.75, 1.25 * 2.0 ** -20, 3.0 * 2.0 ** 40, 0.0])
    assert np.array_equal(O.round_bf16(exact), exact)
    # 1 + 2^-8 lies half-way between 1 and 1 + 2^-7 (odd last bit): goes to 1
    assert O.round_bf16(1.0 + 2.0 ** -8) == 1.0
    assert O.round_bf16(-(1.0 + 2.0 ** -8)) == -1.0
    # 1 + 3 * 2^-8 lies half-way between 1 + 2^-7 (odd) and 1 + 2^-6 (even)
    assert O.round_bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    # just above a half-way point rounds up
    assert O.round_bf16(1.0 + 2.0 ** -8 + 2.0 ** -40) == 1.0 + 2.0 ** -7
    # carry into the exponent
    assert O.round_bf16(2.0 - 2.0 ** -9) == 2.0


def test_round_bf16_matches_bit_rounding_of_fp32_values():
    # second route: round-to-nearest-even on the bit pattern of an IEEE single
    rng = np.random.default_rng(0)
    v = (rng.standard_normal(20000) * 10.0 ** rng.uniform(-6, 6, 20000)).astype(np.float32)
    u = v.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    want = r.astype(np.uint32).view(np.float32).astype(np.float64)
    assert np.array_equal(O.round_bf16(v.astype(np.float64)), want)


def test_round_bf16_error_bound_and_monotone():
    rng = np.random.default_rng(1)
    a = np.sort(rng.standard_normal(50000) * 10.0 ** rng.uniform(-8, 8, 50000))
    r = O.round_bf16(a)
    # unit roundoff of 8 significant bits: 2^-8
    assert np.all(np.abs(r - a) <= 2.0 ** -8 * np.abs(a))
    assert np.all(np.diff(r) >= 0)


def _blocks(n, seed, k=1):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) + 0.5 * np.sqrt(n) * np.eye(n)
    B = rng.standard_normal((n, k)) if k > 1 else rng.standard_normal(n)
    offs = inputs.uneven_offsets(n, 16, 40, rng)
    blocks = O.partition(A, B, offs)
    QR = [O.block_qr(Ai) for Ai, _ in blocks]
    return A, B, offs, blocks, [q for q, _ in QR], [r for _, r in QR]


def test_block_coefficients_are_coordinates_of_every_block_solution():
    A, B, offs, blocks, Qs, Rs = _blocks(150, 2, k=3)
    x_star = np.linalg.solve(A, B)
    for (Ai, bi), Q, R in zip(blocks, Qs, Rs):
        c = O.block_coefficients(Q, R, bi)
        assert np.allclose(Q @ c, O.least_norm_init(Q, R, bi), rtol=0, atol=1e-12)
        # x* solves A_i x = b_i, so Q_i^T x* = c_i
        assert np.allclose(Q.T @ x_star, c, rtol=0, atol=1e-9 * np.abs(c).max())


@pytest.mark.parametrize("k", [1, 3])
def test_affine_form_equals_cons1_with_orthonormal_bases(k):
    # App. A: with Q_i orthonormal and A_i x_i = b_i the two forms coincide
    A, B, offs, blocks, Qs, Rs = _blocks(160, 3, k=k)
    g, e, _ = O.optimal_params(*O.mu_bounds(Qs))
    cs = [O.block_coefficients(Q, R, bi) for Q, R, (_, bi) in zip(Qs, Rs, blocks)]
    xs_a, xbar_a = O.apc_run_affine(Qs, cs, g, e, 40)
    ref = O.apc_run(A, B, offs, g, e, max_iters=40, Qs=Qs, Rs=Rs)
    scale = np.linalg.norm(ref.xbar)
    assert np.linalg.norm(xbar_a - ref.xbar) <= 1e-12 * scale * 40
    for xa, xr in zip(xs_a, ref.xs):
        assert np.linalg.norm(xa - xr) <= 1e-12 * scale * 40


def test_affine_form_differs_from_cons1_on_rounded_bases():
    A, B, offs, blocks, Qs, Rs = _blocks(160, 4)
    g, e, _ = O.optimal_params(*O.mu_bounds(Qs))
    cs = [O.block_coefficients(Q, R, bi) for Q, R, (_, bi) in zip(Qs, Rs, blocks)]
    Qr = [O.round_bf16(Q) for Q in Qs]
    _, xbar_a = O.apc_run_affine(Qr, cs, g, e, 10)
    xs0 = [Q @ c for Q, c in zip(Qr, cs)]
    ref = O.apc_run(A, B, offs, g, e, max_iters=10, Qs=Qr, Rs=Rs, xs0=xs0)
    assert np.linalg.norm(xbar_a - ref.xbar) > 1e-6 * np.linalg.norm(ref.xbar)


def test_affine_fixed_point_on_rounded_bases_closed_form():
    # The limit of the affine iteration satisfies x_i = P_i xbar + Q_i c_i and
    # xbar = mean_i x_i, i.e. (sum_i Q_i Q_i^T) xbar = sum_i Q_i c_i: solved
    # here directly and compared with 4000 iterations.
    A, B, offs, blocks, Qs, Rs = _blocks(120, 5)
    g, e, rho = O.optimal_params(*O.mu_bounds(Qs))
    cs = [O.block_coefficients(Q, R, bi) for Q, R, (_, bi) in zip(Qs, Rs, blocks)]
    Qr = [O.round_bf16(Q) for Q in Qs]
    M = sum(Q @ Q.T for Q in Qr)
    rhs = sum(Q @ c for Q, c in zip(Qr, cs))
    x_fp = np.linalg.solve(M, rhs)
    _, xbar = O.apc_run_affine(Qr, cs, g, e, 4000)
    assert np.linalg.norm(xbar - x_fp) <= 1e-9 * np.linalg.norm(x_fp)
    # and the rounded bases move the limit away from A^{-1} b by about the rounding
    x_star = np.linalg.solve(A, B)
    d = np.linalg.norm(x_fp - x_star) / np.linalg.norm(x_star)
    assert 1e-6 < d < 1e-1


def _affine_case(n, m, seed, k=1, bf16=True):
    A, _, B = inputs.gaussian_system(n, seed, k=k)
    offs = inputs.even_offsets(n, m)
    bl = O.partition(A, B, offs)
    QR = [O.block_qr(Ai) for Ai, _ in bl]
    Qs = [O.round_bf16(Q) if bf16 else Q for Q, _ in QR]
    Rs = [R for _, R in QR]
    cs = [O.block_coefficients(Q, R, bi) for (Q, R), (_, bi) in zip(QR, bl)]
    lo, hi = O.mu_bounds([Q for Q, _ in QR])
    g, e, _ = O.optimal_params(lo, hi)
    return A, B, offs, bl, Qs, Rs, cs, g, e


@pytest.mark.parametrize("k", [1, 3])
def test_affine_adjoint_matches_central_differences(k):
    # c -> xbar(T) is linear and L = 0.5 ||xbar(T) - x_t||^2 quadratic, so a
    # central difference in any direction equals <dL/dc, d> up to rounding
    n, m, T = 60, 4, 25
    A, B, offs, bl, Qs, Rs, cs, g, e = _affine_case(n, m, 41, k=k)
    rng = np.random.default_rng(2)
    xt = rng.standard_normal(B.shape)

    def L(cc):
        return 0.5 * float(np.sum((O.apc_run_affine(Qs, cc, g, e, T)[1] - xt) ** 2))

    gT = O.apc_run_affine(Qs, cs, g, e, T)[1] - xt
    dc = O.apc_adjoint_affine(Qs, g, e, T, gT)
    for _ in range(3):
        d = [rng.standard_normal(c.shape) for c in cs]
        h = 0.3
        fd = (L([c + h * di for c, di in zip(cs, d)]) - L([c - h * di for c, di in zip(cs, d)])) / (2 * h)
        an = sum(float(np.sum(a * di)) for a, di in zip(dc, d))
        assert an == pytest.approx(fd, rel=1e-9)


def test_affine_adjoint_dot_product_test():
    # <J v, w> = <v, J^T w> for the linear map J: (c_i) -> xbar(T)
    n, m, T = 50, 5, 30
    A, B, offs, bl, Qs, Rs, cs, g, e = _affine_case(n, m, 42)
    rng = np.random.default_rng(3)
    v = [rng.standard_normal(c.shape) for c in cs]
    w = rng.standard_normal(n)
    Jv = O.apc_run_affine(Qs, v, g, e, T)[1]
    JTw = O.apc_adjoint_affine(Qs, g, e, T, w)
    lhs, rhs = float(Jv @ w), sum(float(a @ b) for a, b in zip(v, JTw))
    assert abs(lhs - rhs) <= 1e-11 * max(abs(lhs), abs(rhs))


def test_affine_adjoint_equals_cons_adjoint_for_orthonormal_bases():
    # with exact (orthonormal) bases both forms give one map b -> xbar(T), so
    # R_i^{-1} dL/dc_i equals the Eq. (cons) sweep's dL/db_i (a different
    # recursion: per-machine lam_i carry Q_i Q_i^T terms there)
    import scipy.linalg as sla
    n, m, T = 48, 4, 20
    A, B, offs, bl, Qs, Rs, cs, g, e = _affine_case(n, m, 43, bf16=False)
    gT = np.random.default_rng(4).standard_normal(n)
    dc = O.apc_adjoint_affine(Qs, g, e, T, gT)
    db_aff = np.concatenate([sla.solve_triangular(R, d, lower=False) for R, d in zip(Rs, dc)])
    db_cons = np.concatenate(O.apc_adjoint(bl, Qs, Rs, g, e, T, gT)[0])
    assert np.linalg.norm(db_aff - db_cons) <= 1e-10 * np.linalg.norm(db_cons)


def test_affine_adjoint_tends_to_the_fixed_point_adjoint():
    # the affine iteration converges to x* = M^{-1} sum_i Q_i c_i with
    # M = sum_i Q_i Q_i^T (rounded bases included), so for many iterations
    # dL/dc_i tends to Q_i^T M^{-1} g (closed form, numpy.linalg.solve)
    n, m = 40, 4
    A, B, offs, bl, Qs, Rs, cs, g, e = _affine_case(n, m, 44)
    gT = np.random.default_rng(5).standard_normal(n)
    M = sum(Q @ Q.T for Q in Qs)
    want = [Q.T @ np.linalg.solve(M, gT) for Q in Qs]
    dc = O.apc_adjoint_affine(Qs, g, e, 3000, gT)
    err = max(np.linalg.norm(a - b) / np.linalg.norm(b) for a, b in zip(dc, want))
    assert err <= 1e-9
