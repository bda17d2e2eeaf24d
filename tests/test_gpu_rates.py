"""Convergence rates measured on the GPU against Table 1 / Theorem 1 (the
oracle's spectra): APC on the synthetic rows of Table 2, and the preconditioned
heavy-ball method of Sec. 6 reaching APC's rate."""
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


def _tail_rate(ts, errs, floor):
    """Per-iteration decay fitted (least squares on log error) over the second
    half of the samples above `floor` (the optimum's double root makes the early
    decay slower)."""
    ts, errs = np.asarray(ts, float), np.asarray(errs, float)
    keep = errs > floor
    ts, errs = ts[keep], errs[keep]
    h = len(ts) // 2
    slope = np.polyfit(ts[h:], np.log(errs[h:]), 1)[0]
    return float(np.exp(slope))


@pytest.mark.parametrize("N,chunk,total", [(1000, 2, 80), (500, 1000, 40000)])
def test_apc_observed_rate_matches_theorem1_on_table2_rows(N, chunk, total):
    # "Standard Tall Gaussian (1000 x 500)" and "Standard Gaussian (500 x 500)",
    # m = 10 contiguous blocks, FP64 path
    apc, dev = _apc(), _dev()
    n, m = 500, 10
    A, x_true, b = inputs.gaussian_system(n, 0, N=N)
    offs = inputs.even_offsets(N, m)
    Qs = [O.block_qr(Ai)[0] for Ai, _ in O.partition(A, b, offs)]
    lo, hi = O.mu_bounds(Qs)
    g, e, rho = O.optimal_params(lo, hi)
    x_star = np.linalg.lstsq(A, b, rcond=None)[0]
    ctx = apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(b, device=dev), offs, precision="f64")
    ctx.reset()
    ts, errs = [], []
    for t in range(chunk, total + 1, chunk):
        ctx.iterate(g, e, chunk)
        ts.append(t)
        errs.append(np.linalg.norm(ctx.xbar().cpu().numpy() - x_star) / np.linalg.norm(x_star))
        if errs[-1] < 1e-12:
            break
    obs = _tail_rate(ts, errs, 1e-11)
    assert 0.8 <= np.log(obs) / np.log(rho) <= 1.1, (obs, rho)


def test_preconditioned_heavy_ball_reaches_the_apc_rate_on_gpu():
    # Sec. 6: D-HBM on C x = d (C^T C = m X) converges at (sqrt(kappa(X)) - 1) /
    # (sqrt(kappa(X)) + 1), APC's optimal rate.  Batched path, BF16 bases: the
    # spectrum is that of the BF16 X and the limit the BF16 fixed point.  The
    # FP32 arithmetic stalls near kappa(X) * 6e-8 relative, so the system is
    # well conditioned (kappa(X) ~ 76) and the fit stops at 1e-4.
    apc, dev = _apc(), _dev()
    rng = np.random.default_rng(81)
    n, k = 256, 1
    A = rng.standard_normal((n, n)) + 1.5 * np.sqrt(n) * np.eye(n)
    B = rng.standard_normal((n, k))
    offs = inputs.uneven_offsets(n, 16, 64, rng)
    blocks = O.partition(A, B, offs)
    QR = [O.block_qr(Ai) for Ai, _ in blocks]
    Qr = [O.round_bf16(q) for q, _ in QR]
    cs = [O.block_coefficients(q, r, bi) for (q, r), (_, bi) in zip(QR, blocks)]
    m = len(Qr)
    mu = np.linalg.eigvalsh(sum(Q @ Q.T for Q in Qr) / m)
    x_fp = np.linalg.solve(sum(Q @ Q.T for Q in Qr), sum(Q @ c for Q, c in zip(Qr, cs)))
    g, e, rho = O.optimal_params(mu[0], min(mu[-1], 1.0))
    alpha, beta, rho_hb = O.hb_optimal_params(m * mu[0], m * mu[-1])
    bt = apc.apc_batch_setup([torch.tensor(A, device=dev)], [torch.tensor(B, device=dev)], [offs])
    chunk = max(1, int(0.5 / -np.log(rho_hb)))
    observed = {}
    for method in ("hb", "apc"):
        if method == "hb":
            bt.set_hb_params([alpha], [beta])
        else:
            bt.set_params([g], [e])
        bt.reset()
        ts, errs = [], []
        for t in range(chunk, 400 * chunk, chunk):
            bt.iterate(chunk)
            ts.append(t)
            errs.append(np.linalg.norm(bt.xbar(0).cpu().numpy() - x_fp) / np.linalg.norm(x_fp))
            if errs[-1] < 1e-5:
                break
        observed[method] = _tail_rate(ts, errs, 1e-4)
    assert 0.8 <= np.log(observed["hb"]) / np.log(rho_hb) <= 1.1, (observed, rho_hb)
    assert 0.8 <= np.log(observed["apc"]) / np.log(rho_hb) <= 1.1, (observed, rho_hb)
