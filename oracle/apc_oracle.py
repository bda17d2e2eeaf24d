"""Plain FP64 CPU oracle of Accelerated Projection-based Consensus (APC).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  The product path (the CUDA library and its Python binding) never calls
it, and this module imports nothing from the product package.

Everything here is float64 NumPy, written for a reader to check against the
paper (Azizan-Ruhi, Lahouti, Avestimehr, Hassibi, "Distributed Solution of
Large-Scale Linear Systems via Accelerated Projection-Based Consensus", 2017)
by eye: no blocking, fusion or reordering beyond what each cited passage
states.  Library primitives used as steps: ``numpy.linalg.qr`` (the paper's
"e.g. using QR factorization", Sec. 3.3), ``scipy.linalg.solve_triangular``,
``numpy.linalg.eigvalsh`` and ``numpy.linalg.solve``.

Notation follows the paper: ``A`` is N x n, the rows are split into m blocks
``A_i`` (p_i x n) with right-hand sides ``b_i``; ``x_i`` are the machines'
iterates, ``xbar`` the master's estimate, ``gamma`` / ``eta`` the two
momentum parameters, ``P_i`` the projector onto the nullspace of ``A_i`` and
``X = (1/m) sum_i A_i^T (A_i A_i^T)^{-1} A_i``.

Readings taken where the paper is silent or ambiguous (each is also listed in
the design notes):
  * ``xbar(0)`` is not defined by Algorithm 1: we take the mean of the
    ``x_i(0)``.
  * Algorithm 1 loops "for t = 1 to T" but updates t -> t+1: T iterations are
    T applications of Eq. (cons), t = 0 .. T-1.
  * ``x_i(0)`` is "a solution among infinitely many": we take the least-norm
    solution ``A_i^T (A_i A_i^T)^{-1} b_i``.
  * The optimality system of Theorem 1 is symmetric in gamma and eta; the set
    S requires gamma in [0, 2], so gamma is the smaller root.
  * Uneven blocks are allowed: no step of the analysis (Sec. 3.2, App. A)
    uses equal p.

Parity status: every function below is pinned by ``tests/test_oracle_*.py``
(closed forms, invariants, brute-force spectra, library routines reached by a
different route, and the values printed in Table 2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla

__all__ = [
    "partition", "block_qr", "least_norm_init", "projector", "x_matrix",
    "mu_bounds", "optimal_params", "char_roots", "apc_spectral_radius",
    "iteration_matrix", "apc_step", "apc_run", "cimmino_step", "cimmino_run",
    "relative_residual", "relative_error", "invariant_drift",
    "rate_apc", "rate_cimmino", "rate_consensus", "convergence_time",
    "apc_forward_linear", "apc_adjoint", "power_mu_max", "ApcTrace",
    "round_bf16", "block_coefficients", "apc_step_affine", "apc_run_affine", "apc_adjoint_affine",
    "partition_rows",
    "precondition_blocks", "hb_optimal_params", "dhbm_step", "dhbm_run",
    "rate_dgd", "rate_dnag", "rate_dhbm", "madmm_step", "madmm_rate", "madmm_optimal_rate", "table2_row",
]


# ---------------------------------------------------------------------------
# Setup (Sec. 2, Sec. 3.1, Sec. 3.3)
# ---------------------------------------------------------------------------

def partition(A: np.ndarray, b: np.ndarray, row_offsets) -> list[tuple[np.ndarray, np.ndarray]]:
    """Split [A, b] into the machines' blocks [A_i, b_i] (Sec. 2, the block
    form of Eq. (1)).  ``row_offsets`` has m+1 entries, 0 = o_0 < ... < o_m = N;
    block i holds rows o_i .. o_{i+1}-1.  ``b`` may be N or N x k."""
    offs = [int(o) for o in row_offsets]
    if offs[0] != 0 or offs[-1] != A.shape[0] or any(offs[i + 1] <= offs[i] for i in range(len(offs) - 1)):
        raise ValueError("row_offsets must be strictly increasing from 0 to N")
    return [(A[offs[i]:offs[i + 1], :], b[offs[i]:offs[i + 1]]) for i in range(len(offs) - 1)]


def partition_rows(A: np.ndarray, b: np.ndarray, row_sets) -> list[tuple[np.ndarray, np.ndarray]]:
    """The machines' blocks for an arbitrary (not necessarily contiguous)
    assignment of equations (Sec. 2 only asks that the m subsets of the N
    equations be given to m machines): block i holds the rows listed in
    ``row_sets[i]``, in that order.  The sets must cover every row exactly once."""
    rows = [np.asarray(r, dtype=np.int64) for r in row_sets]
    allr = np.concatenate(rows) if rows else np.zeros(0, dtype=np.int64)
    if allr.size != A.shape[0] or not np.array_equal(np.sort(allr), np.arange(A.shape[0])):
        raise ValueError("row_sets must cover every row exactly once")
    return [(A[r, :], b[r]) for r in rows]


def block_qr(A_i: np.ndarray, rank_tol: float | None = None) -> tuple[np.ndarray, np.ndarray]:
    """Thin QR of A_i^T = Q_i R_i (Sec. 3.3, "e.g. using QR factorization").

    Q_i (n x p) has orthonormal columns spanning the row space of A_i, so the
    nullspace projector of Sec. 3.1 is P_i = I - Q_i Q_i^T.  Raises if A_i is
    rank deficient (the paper needs (A_i A_i^T)^{-1} to exist)."""
    Q, R = np.linalg.qr(A_i.T, mode="reduced")
    d = np.abs(np.diag(R))
    tol = rank_tol if rank_tol is not None else max(A_i.shape) * np.finfo(np.float64).eps * d.max()
    if d.min() <= tol:
        raise np.linalg.LinAlgError("block has dependent rows: A_i A_i^T is singular")
    return Q, R


def least_norm_init(Q_i: np.ndarray, R_i: np.ndarray, b_i: np.ndarray) -> np.ndarray:
    """x_i(0) = A_i^T (A_i A_i^T)^{-1} b_i, the least-norm solution of
    A_i x = b_i (Sec. 3.1 / Algorithm 1 initialisation).  With A_i^T = Q_i R_i
    this is Q_i R_i^{-T} b_i."""
    c_i = sla.solve_triangular(R_i, b_i, trans="T", lower=False)
    return Q_i @ c_i


def projector(A_i: np.ndarray) -> np.ndarray:
    """P_i = I - A_i^T (A_i A_i^T)^{-1} A_i, written out as defined in Sec. 3.1
    (used by the tests as a second route to the projector)."""
    n = A_i.shape[1]
    return np.eye(n) - A_i.T @ np.linalg.solve(A_i @ A_i.T, A_i)


def x_matrix(Qs: list[np.ndarray]) -> np.ndarray:
    """X = (1/m) sum_i A_i^T (A_i A_i^T)^{-1} A_i  (Eq. 3, Sec. 3.2), which
    equals (1/m) sum_i Q_i Q_i^T."""
    m = len(Qs)
    return sum(Q @ Q.T for Q in Qs) / m


def mu_bounds(Qs: list[np.ndarray]) -> tuple[float, float]:
    """(mu_min, mu_max) of X (Eq. 4) by a dense symmetric eigensolve."""
    mu = np.linalg.eigvalsh(x_matrix(Qs))
    return float(mu[0]), float(mu[-1])


def optimal_params(mu_min: float, mu_max: float) -> tuple[float, float, float]:
    """Optimal (gamma*, eta*, rho) of Theorem 1.

    The two equations mu_max*eta*gamma = (1+r)^2 and mu_min*eta*gamma = (1-r)^2
    with r = sqrt((gamma-1)(eta-1)) give eta*gamma = s = 4/(sqrt(mu_max)+sqrt(mu_min))^2
    and r = rho = (sqrt(kappa)-1)/(sqrt(kappa)+1) (App. A).  Then
    gamma + eta = s + 1 - rho^2, so gamma and eta are the roots of
    z^2 - (s + 1 - rho^2) z + s.  The set S restricts gamma to [0, 2], which
    selects the smaller root for gamma."""
    if not (0.0 < mu_min <= mu_max <= 1.0 + 1e-12):
        raise ValueError("need 0 < mu_min <= mu_max <= 1")
    smin, smax = math.sqrt(mu_min), math.sqrt(mu_max)
    s = 4.0 / (smax + smin) ** 2
    rho = (smax - smin) / (smax + smin)
    tr = s + 1.0 - rho * rho
    disc = max(tr * tr - 4.0 * s, 0.0)
    gamma = (tr - math.sqrt(disc)) / 2.0
    eta = (tr + math.sqrt(disc)) / 2.0
    return gamma, eta, rho


def char_roots(mu: float, gamma: float, eta: float) -> np.ndarray:
    """Roots of p_i(lambda; gamma, eta) = lambda^2 + (-eta*gamma*(1-mu) + gamma - 1 + eta - 1) lambda
    + (gamma-1)(eta-1)  (Eq. 5)."""
    return np.roots([1.0, -eta * gamma * (1.0 - mu) + gamma - 1.0 + eta - 1.0, (gamma - 1.0) * (eta - 1.0)])


def apc_spectral_radius(mus, gamma: float, eta: float, m: int) -> float:
    """Spectral radius of the APC error recursion (App. A): the largest root
    modulus of p_i over the spectrum of X, together with the (m-1)n-fold
    eigenvalue 1 - gamma when m > 1."""
    r = max(float(np.max(np.abs(char_roots(mu, gamma, eta)))) for mu in mus)
    if m > 1:
        r = max(r, abs(1.0 - gamma))
    return r


def iteration_matrix(Ps: list[np.ndarray], gamma: float, eta: float) -> np.ndarray:
    """The (m+1)n x (m+1)n matrix of Eq. (matrix_recursion), App. A, acting on
    the stacked errors [e_1; ...; e_m; ebar]."""
    m = len(Ps)
    n = Ps[0].shape[0]
    M = eta * gamma / m * sum(Ps) + (1.0 - eta) * np.eye(n)
    T = np.zeros(((m + 1) * n, (m + 1) * n))
    for i in range(m):
        T[i * n:(i + 1) * n, i * n:(i + 1) * n] = (1.0 - gamma) * np.eye(n)
        T[i * n:(i + 1) * n, m * n:] = gamma * Ps[i]
        T[m * n:, i * n:(i + 1) * n] = eta * (1.0 - gamma) / m * np.eye(n)
    T[m * n:, m * n:] = M
    return T


# ---------------------------------------------------------------------------
# The iteration (Eq. (cons), Algorithm 1)
# ---------------------------------------------------------------------------

def apc_step(xs: list[np.ndarray], xbar: np.ndarray, Qs: list[np.ndarray], gamma: float, eta: float):
    """One APC iteration, Eq. (cons1)-(cons2) as printed:
        x_i(t+1) = x_i(t) + gamma * P_i (xbar(t) - x_i(t)),   i = 1..m
        xbar(t+1) = (eta/m) sum_i x_i(t+1) + (1 - eta) xbar(t)
    with P_i y = y - Q_i (Q_i^T y).  Works for n-vectors and n x k blocks."""
    m = len(xs)
    new_xs = []
    for x_i, Q_i in zip(xs, Qs):
        y = xbar - x_i
        P_y = y - Q_i @ (Q_i.T @ y)
        new_xs.append(x_i + gamma * P_y)
    new_xbar = (eta / m) * sum(new_xs) + (1.0 - eta) * xbar
    return new_xs, new_xbar


@dataclass
class ApcTrace:
    """What ``apc_run`` returns: the final state and a record every
    ``record_every`` iterations of (t, relative residual, relative error,
    invariant drift)."""
    xs: list
    xbar: np.ndarray
    iters: int
    history: list
    converged: bool


def relative_residual(A: np.ndarray, b: np.ndarray, x: np.ndarray) -> float:
    """||b - A x||_2 / ||b||_2 (Frobenius over columns when k > 1)."""
    return float(np.linalg.norm(b - A @ x) / np.linalg.norm(b))


def relative_error(x: np.ndarray, x_star: np.ndarray) -> float:
    """||x - x*|| / ||x*||, the error the paper plots in Fig. 2 (Sec. 5)."""
    return float(np.linalg.norm(x - x_star) / np.linalg.norm(x_star))


def invariant_drift(blocks, xs) -> float:
    """max_i ||A_i x_i - b_i|| / ||b||: every x_i(t) solves A_i x = b_i (App. A,
    the step from Eq. (e_i) to Eq. (e_i(t+1)))."""
    nb = math.sqrt(sum(float(np.linalg.norm(b_i)) ** 2 for _, b_i in blocks))
    return max(float(np.linalg.norm(A_i @ x_i - b_i)) for (A_i, b_i), x_i in zip(blocks, xs)) / nb


def apc_run(A, b, row_offsets, gamma, eta, *, max_iters=10**6, tol=None, x_star=None,
            record_every=0, xs0=None, xbar0=None, Qs=None, Rs=None) -> ApcTrace:
    """Algorithm 1 end to end in FP64.

    Initialisation: x_i(0) least-norm (unless ``xs0`` is given), xbar(0) the
    mean of the x_i(0) (unless ``xbar0`` is given).  Runs until the relative
    residual ||b - A xbar|| / ||b|| <= tol (checked every ``record_every``
    iterations, or every iteration when record_every == 0 and tol is set) or
    max_iters iterations."""
    blocks = partition(A, b, row_offsets)
    if Qs is None:
        QR = [block_qr(A_i) for A_i, _ in blocks]
        Qs = [q for q, _ in QR]
        Rs = [r for _, r in QR]
    if xs0 is None:
        xs = [least_norm_init(Q, R, b_i) for Q, R, (_, b_i) in zip(Qs, Rs, blocks)]
    else:
        xs = [np.array(x, dtype=np.float64, copy=True) for x in xs0]
    xbar = sum(xs) / len(xs) if xbar0 is None else np.array(xbar0, dtype=np.float64, copy=True)
    history = []
    every = record_every if record_every > 0 else (1 if tol is not None else 0)

    def record(t):
        rr = relative_residual(A, b, xbar)
        re = relative_error(xbar, x_star) if x_star is not None else float("nan")
        history.append((t, rr, re, invariant_drift(blocks, xs)))
        return rr

    converged = False
    t = 0
    if every and record(0) <= (tol if tol is not None else -1.0):
        converged = True
    while not converged and t < max_iters:
        xs, xbar = apc_step(xs, xbar, Qs, gamma, eta)
        t += 1
        if every and t % every == 0:
            if record(t) <= (tol if tol is not None else -1.0):
                converged = True
    return ApcTrace(xs=xs, xbar=xbar, iters=t, history=history, converged=converged)


# ---------------------------------------------------------------------------
# Block Cimmino (Sec. 4.5), used to check Proposition 1
# ---------------------------------------------------------------------------

def cimmino_step(blocks, xbar: np.ndarray, nu: float) -> np.ndarray:
    """Eq. (cimmino_1)-(cimmino_2): r_i = A_i^+ (b_i - A_i xbar),
    xbar <- xbar + nu * sum_i r_i, with A_i^+ = A_i^T (A_i A_i^T)^{-1}."""
    total = np.zeros_like(xbar)
    for A_i, b_i in blocks:
        total = total + A_i.T @ np.linalg.solve(A_i @ A_i.T, b_i - A_i @ xbar)
    return xbar + nu * total


def cimmino_run(A, b, row_offsets, nu, xbar0, iters):
    blocks = partition(A, b, row_offsets)
    xbar = np.array(xbar0, dtype=np.float64, copy=True)
    out = [xbar]
    for _ in range(iters):
        xbar = cimmino_step(blocks, xbar, nu)
        out.append(xbar)
    return out


# ---------------------------------------------------------------------------
# Rates (Table 1, Theorem 1, Sec. 4.5) and the convergence time of Table 2
# ---------------------------------------------------------------------------

def rate_apc(kappa_X: float) -> float:
    """Optimal APC rate (Theorem 1): (sqrt(kappa)-1)/(sqrt(kappa)+1)."""
    s = math.sqrt(kappa_X)
    return (s - 1.0) / (s + 1.0)


def rate_cimmino(kappa_X: float) -> float:
    """Optimal block Cimmino rate (Sec. 4.5): (kappa-1)/(kappa+1)."""
    return (kappa_X - 1.0) / (kappa_X + 1.0)


def rate_consensus(mu_min: float) -> float:
    """Standard projection consensus (gamma = eta = 1), Table 1: 1 - mu_min(X)."""
    return 1.0 - mu_min


def rate_dgd(kappa_AtA: float) -> float:
    """Distributed gradient descent, optimal step (Sec. 4.1): (kappa - 1)/(kappa + 1)."""
    return (kappa_AtA - 1.0) / (kappa_AtA + 1.0)


def rate_dnag(kappa_AtA: float) -> float:
    """Distributed Nesterov accelerated gradient, optimal tuning (Sec. 4.2):
    1 - 2 / sqrt(3 kappa + 1)."""
    return 1.0 - 2.0 / math.sqrt(3.0 * kappa_AtA + 1.0)


def rate_dhbm(kappa_AtA: float) -> float:
    """Distributed heavy ball, optimal tuning (Sec. 4.3): (sqrt(kappa) - 1)/(sqrt(kappa) + 1)."""
    s = math.sqrt(kappa_AtA)
    return (s - 1.0) / (s + 1.0)


def madmm_step(blocks, xbar: np.ndarray, xi: float) -> np.ndarray:
    """One iteration of the modified consensus ADMM of Sec. 4.4 (the y_i set to
    zero): x_i = (A_i^T A_i + xi I)^{-1} (A_i^T b_i + xi xbar), xbar' = mean_i x_i."""
    n = xbar.shape[0]
    xs = [np.linalg.solve(A_i.T @ A_i + xi * np.eye(n), A_i.T @ b_i + xi * xbar) for A_i, b_i in blocks]
    return sum(xs) / len(xs)


def madmm_rate(blocks, xi: float) -> float:
    """Rate of ``madmm_step``: the error map is e -> (1/m) sum_i xi (A_i^T A_i + xi I)^{-1} e
    (subtract the step at the solution), so the rate is its largest eigenvalue."""
    n = blocks[0][0].shape[1]
    M = sum(xi * np.linalg.inv(A_i.T @ A_i + xi * np.eye(n)) for A_i, _ in blocks) / len(blocks)
    return float(np.linalg.eigvalsh((M + M.T) / 2).max())


def madmm_optimal_rate(blocks, lo: float = -4.0, hi: float = 6.0, points: int = 41) -> tuple[float, float]:
    """The paper tunes every method to its best parameter (Sec. 5); Sec. 4.4
    gives no closed form for the modified ADMM, so scan ``madmm_rate`` over
    xi = 10^lo .. 10^hi (log grid) and return the best (xi, rate).  Each term
    xi (A_i^T A_i + xi I)^{-1} grows with xi in the Loewner order, so the best
    rate is approached as xi -> 0, where the error map tends to
    (1/m) sum_i P_i = I - X (Sec. 3.2): the consensus rate 1 - mu_min(X).
    (Below xi ~ 1e-4 the inverse of A_i^T A_i + xi I is too ill-conditioned for
    FP64 to resolve the rate; the default grid stops there.)"""
    best = (0.0, 2.0)
    for e in np.linspace(lo, hi, points):
        r = madmm_rate(blocks, 10.0 ** e)
        if r < best[1]:
            best = (10.0 ** e, r)
    return best


def table2_row(A: np.ndarray, b: np.ndarray, row_offsets) -> dict:
    """Convergence times T = 1/(-log rho) of the methods compared in Table 2
    (Sec. 5) for one problem, from the rates of Table 1 (and ``madmm_optimal_rate``):
    the spectra of A^T A = sum_i A_i^T A_i and of X decide them all."""
    blocks = partition(A, b, row_offsets)
    Qs = [block_qr(A_i)[0] for A_i, _ in blocks]
    mu_lo, mu_hi = mu_bounds(Qs)
    sv = np.linalg.svd(A, compute_uv=False)
    k_ata = float((sv.max() / sv.min()) ** 2)
    k_x = mu_hi / mu_lo
    _, r_admm = madmm_optimal_rate(blocks)
    rates = {"DGD": rate_dgd(k_ata), "D-NAG": rate_dnag(k_ata), "D-HBM": rate_dhbm(k_ata), "M-ADMM": r_admm,
             "B-Cimmino": rate_cimmino(k_x), "APC": rate_apc(k_x), "Consensus": rate_consensus(mu_lo)}
    out = {k: convergence_time(r) for k, r in rates.items()}
    out.update(kappa_AtA=k_ata, kappa_X=k_x, mu_min=mu_lo, mu_max=mu_hi)
    return out


def convergence_time(rho: float) -> float:
    """T = 1 / (-log rho) (Table 2 caption)."""
    return 1.0 / (-math.log(rho))


# ---------------------------------------------------------------------------
# Differentiation through T unrolled iterations (transpose of Eq. (cons))
# ---------------------------------------------------------------------------

def apc_forward_linear(blocks, Qs, Rs, gamma, eta, T):
    """xbar(T) as a function of b: least-norm x_i(0), xbar(0) = mean, then T
    applications of Eq. (cons).  Returns (xbar(T), xs(T), states) where
    ``states[t] = (xs(t), xbar(t))`` for t = 0..T."""
    xs = [least_norm_init(Q, R, b_i) for Q, R, (_, b_i) in zip(Qs, Rs, blocks)]
    xbar = sum(xs) / len(xs)
    states = [(xs, xbar)]
    for _ in range(T):
        xs, xbar = apc_step(xs, xbar, Qs, gamma, eta)
        states.append((xs, xbar))
    return xbar, xs, states


def apc_adjoint(blocks, Qs, Rs, gamma, eta, T, g_T, states=None):
    """Reverse-mode sweep through T iterations of Eq. (cons).

    Given g_T = dL/dxbar(T), returns (dL/db as a list of per-block arrays,
    dL/dgamma, dL/deta).  The step t -> t+1 is linear in the state with
        dx_i(t+1)/dx_i(t) = I - gamma P_i,  dx_i(t+1)/dxbar(t) = gamma P_i,
        xbar(t+1) = (eta/m) sum_i x_i(t+1) + (1-eta) xbar(t),
    and P_i is symmetric (Sec. 3.1), so with mu_i = lam_i(t+1) + (eta/m) lbar(t+1):
        lam_i(t) = (I - gamma P_i) mu_i,
        lbar(t)  = gamma sum_i P_i mu_i + (1 - eta) lbar(t+1).
    At t = 0, x_i(0) = A_i^+ b_i and xbar(0) = mean_i x_i(0), so
        dL/db_i = (A_i^+)^T (lam_i(0) + lbar(0)/m) = R_i^{-1} Q_i^T (...).
    The gamma/eta derivatives need the forward states (``states`` from
    ``apc_forward_linear``); they are skipped (returned as None) without them."""
    m = len(Qs)
    lam = [np.zeros_like(g_T) for _ in range(m)]
    lbar = np.array(g_T, dtype=np.float64, copy=True)
    dgamma = 0.0 if states is not None else None
    deta = 0.0 if states is not None else None
    for t in range(T - 1, -1, -1):
        mus = [lam_i + (eta / m) * lbar for lam_i in lam]
        Pmus = [mu - Q @ (Q.T @ mu) for mu, Q in zip(mus, Qs)]
        if states is not None:
            xs_t, xbar_t = states[t]
            xs_t1, _ = states[t + 1]
            for mu, Q, x_i in zip(mus, Qs, xs_t):
                y = xbar_t - x_i
                dgamma += float(np.sum(mu * (y - Q @ (Q.T @ y))))
            deta += float(np.sum(lbar * (sum(xs_t1) / m - xbar_t)))
        new_lam = [mu - gamma * Pmu for mu, Pmu in zip(mus, Pmus)]
        lbar = gamma * sum(Pmus) + (1.0 - eta) * lbar
        lam = new_lam
    db = []
    for Q, R, lam_i in zip(Qs, Rs, lam):
        v = Q.T @ (lam_i + lbar / m)
        db.append(sla.solve_triangular(R, v, lower=False))
    return db, dgamma, deta


# ---------------------------------------------------------------------------
# Power iteration for mu_max(X) (used to pick safe parameters at large n)
# ---------------------------------------------------------------------------

def power_mu_max(Qs, v0: np.ndarray, iters: int) -> float:
    """Rayleigh quotient after ``iters`` steps of v <- X v / ||X v|| with
    X v = (1/m) sum_i Q_i (Q_i^T v) (Eq. 3)."""
    m = len(Qs)
    v = v0 / np.linalg.norm(v0)
    for _ in range(iters):
        w = sum(Q @ (Q.T @ v) for Q in Qs) / m
        v = w / np.linalg.norm(w)
    w = sum(Q @ (Q.T @ v) for Q in Qs) / m
    return float(v @ w)


# ---------------------------------------------------------------------------
# The affine form of the machines' update (App. A), used with stored bases
# ---------------------------------------------------------------------------

def round_bf16(a) -> np.ndarray:
    """Round float64 values to the nearest bfloat16 (8 significant bits, the
    exponent range of IEEE single), ties to even, and return them as float64.

    Definition written out: a = f * 2^e with 0.5 <= |f| < 1 (``frexp``); the
    nearest value with 8 significant bits is rint(f * 2^8) * 2^(e - 8), where
    ``rint`` rounds half-way cases to the even integer.  Values here are far
    from the overflow and subnormal ranges, which this definition does not
    treat."""
    a = np.asarray(a, dtype=np.float64)
    f, e = np.frexp(a)
    return np.ldexp(np.rint(np.ldexp(f, 8)), e - 8)


def block_coefficients(Q_i: np.ndarray, R_i: np.ndarray, b_i: np.ndarray) -> np.ndarray:
    """c_i = R_i^{-T} b_i, the coordinates of the least-norm solution in the
    basis Q_i: x_i(0) = Q_i c_i and Q_i^T x = c_i for every solution x of
    A_i x = b_i (A_i^T = Q_i R_i, Sec. 3.3).  Works for k right-hand sides."""
    return sla.solve_triangular(R_i, b_i, trans="T", lower=False)


def apc_step_affine(xs, xbar, Qs, cs, gamma: float, eta: float):
    """One iteration in the form of App. A, Eq. (e_i(t+1)) written for x:
        x_i(t+1) = (1 - gamma) x_i(t) + gamma (P_i xbar(t) + Q_i c_i),
        xbar(t+1) = (eta/m) sum_i x_i(t+1) + (1 - eta) xbar(t),
    with P_i y = y - Q_i (Q_i^T y).  App. A derives it from Eq. (cons1) using
    only that x_i(t) solves A_i x = b_i, i.e. P_i x_i = x_i - Q_i c_i; so with an
    orthonormal Q_i and iterates that keep that invariant the two forms give
    the same sequence.  With a rounded (not exactly orthonormal) basis they
    differ, and this is the form to compare against."""
    m = len(xs)
    new_xs = []
    for x_i, Q_i, c_i in zip(xs, Qs, cs):
        P_xbar = xbar - Q_i @ (Q_i.T @ xbar)
        new_xs.append((1.0 - gamma) * x_i + gamma * (P_xbar + Q_i @ c_i))
    new_xbar = (eta / m) * sum(new_xs) + (1.0 - eta) * xbar
    return new_xs, new_xbar


def apc_run_affine(Qs, cs, gamma: float, eta: float, T: int):
    """Algorithm 1 with the affine step: x_i(0) = Q_i c_i, xbar(0) the mean of
    the x_i(0), then T applications of ``apc_step_affine``.  Returns
    (xs(T), xbar(T))."""
    xs = [Q @ c for Q, c in zip(Qs, cs)]
    xbar = sum(xs) / len(xs)
    for _ in range(T):
        xs, xbar = apc_step_affine(xs, xbar, Qs, cs, gamma, eta)
    return xs, xbar


def apc_adjoint_affine(Qs, gamma: float, eta: float, T: int, g_T):
    """Reverse-mode sweep through ``apc_run_affine``: the derivatives of a
    loss L with respect to the block coefficients c_i, given g_T = dL/dxbar(T).

    ``apc_run_affine`` is linear in (c_1..c_m): x_i(0) = Q_i c_i, xbar(0) the
    mean, then T steps of the affine update of App. A.  Written as the plain
    transpose of that step (P_i symmetric, Sec. 3.1), with per-machine adjoints
    lam_i of x_i and lbar of xbar, and mu_i = lam_i(t+1) + (eta/m) lbar(t+1):
        lam_i(t) = (1 - gamma) mu_i,
        lbar(t)  = (1 - eta) lbar(t+1) + gamma sum_i P_i mu_i,
        dL/dc_i += gamma Q_i^T mu_i,
    starting from lam_i(T) = 0, lbar(T) = g_T; at t = 0 the initialisation adds
    dL/dc_i += Q_i^T (lam_i(0) + lbar(0)/m).  With c_i = R_i^{-T} b_i
    (``block_coefficients``) the derivative with respect to b_i is
    R_i^{-1} dL/dc_i.  Works for n-vectors and n x k blocks.  Returns the list
    of dL/dc_i."""
    m = len(Qs)
    lam = [np.zeros_like(g_T, dtype=np.float64) for _ in range(m)]
    lbar = np.array(g_T, dtype=np.float64, copy=True)
    dc = [np.zeros((Q.shape[1],) + np.shape(g_T)[1:]) for Q in Qs]
    for _ in range(T):
        mus = [lam_i + (eta / m) * lbar for lam_i in lam]
        Pmus = [mu - Q @ (Q.T @ mu) for mu, Q in zip(mus, Qs)]
        for i, (mu, Q) in enumerate(zip(mus, Qs)):
            dc[i] = dc[i] + gamma * (Q.T @ mu)
        lam = [(1.0 - gamma) * mu for mu in mus]
        lbar = (1.0 - eta) * lbar + gamma * sum(Pmus)
    for i, (Q, lam_i) in enumerate(zip(Qs, lam)):
        dc[i] = dc[i] + Q.T @ (lam_i + lbar / m)
    return dc


# ---------------------------------------------------------------------------
# Distributed heavy-ball method with the distributed preconditioning of Sec. 6
# ---------------------------------------------------------------------------

def precondition_blocks(blocks):
    """Sec. 6: machine i premultiplies [A_i, b_i] by (A_i A_i^T)^{-1/2}, giving
    [C_i, d_i].  The inverse square root is formed from the eigendecomposition
    of the symmetric positive definite A_i A_i^T (no QR involved)."""
    out = []
    for A_i, b_i in blocks:
        lam, V = np.linalg.eigh(A_i @ A_i.T)
        if lam.min() <= 0:
            raise np.linalg.LinAlgError("A_i A_i^T is singular")
        S = (V / np.sqrt(lam)) @ V.T
        out.append((S @ A_i, S @ b_i))
    return out


def hb_optimal_params(L_min: float, L_max: float) -> tuple[float, float, float]:
    """Step size alpha and momentum beta of the heavy-ball method (the D-HBM
    update of Sec. 4.3) for a quadratic whose Hessian has spectrum in [L_min, L_max]:
    alpha = 4 / (sqrt(L_max) + sqrt(L_min))^2,
    beta = ((sqrt(L_max) - sqrt(L_min)) / (sqrt(L_max) + sqrt(L_min)))^2, which
    attain the rate (sqrt(kappa) - 1) / (sqrt(kappa) + 1) that Sec. 4.3 quotes
    (Polyak's choice; the paper states only the rate).  Returns (alpha, beta, rho)."""
    if not (0.0 < L_min <= L_max):
        raise ValueError("need 0 < L_min <= L_max")
    a, c = math.sqrt(L_max), math.sqrt(L_min)
    return 4.0 / (a + c) ** 2, ((a - c) / (a + c)) ** 2, (a - c) / (a + c)


def dhbm_step(pblocks, x: np.ndarray, z: np.ndarray, alpha: float, beta: float):
    """One D-HBM iteration (Sec. 4.3) on the blocks [C_i, d_i]:
        z(t+1) = beta z(t) + sum_i C_i^T (C_i x(t) - d_i),
        x(t+1) = x(t) - alpha z(t+1)."""
    g = sum(C_i.T @ (C_i @ x - d_i) for C_i, d_i in pblocks)
    z = beta * z + g
    return x - alpha * z, z


def dhbm_run(pblocks, x0: np.ndarray, alpha: float, beta: float, T: int):
    """T iterations of ``dhbm_step`` from x0 with z(0) = 0; returns x(T)."""
    x = np.array(x0, dtype=np.float64, copy=True)
    z = np.zeros_like(x)
    for _ in range(T):
        x, z = dhbm_step(pblocks, x, z, alpha, beta)
    return x
