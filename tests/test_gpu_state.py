"""Checkpoint/resume of the iteration state (apc_export_state /
apc_import_state) and the deterministic reduction mode (apc_set_deterministic),
through the C ABI.  In deterministic mode the clusters' partial sums are added
in a fixed order, so "T iterations, export, import into a fresh context, T
more" equals "2T iterations" bit for bit; the mode computes Eq. (cons) like
the default one (parity against the oracle on the stored bases)."""
import numpy as np
import pytest

from oracle import apc_oracle as O
from paper_1708_01413_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _env():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1708_01413_gb300 import apc, build
    build.build()
    return apc, torch.device("cuda:0")


def _system(n, m, seed):
    A, _, b = inputs.gaussian_system(n, seed)
    offs = inputs.even_offsets(n, m)
    bl = O.partition(A, b, offs)
    QR = [O.block_qr(Ai) for Ai, _ in bl]
    g, e, _ = O.optimal_params(*O.mu_bounds([q for q, _ in QR]))
    return A, b, offs, bl, QR, g, e


@pytest.mark.parametrize("prec", ["bf16", "f32", "f64"])
def test_deterministic_mode_is_reproducible_and_matches_oracle(prec):
    apc, dev = _env()
    n, m, T = 2048, 16, 40
    A, b, offs, bl, QR, g, e = _system(n, m, 91)
    ctx = apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(b, device=dev), offs, precision=prec)
    assert ctx.info()["clusters"] > 1
    ctx.set_deterministic(True)
    runs = []
    for _ in range(2):
        ctx.reset()
        ctx.iterate(g, e, T)
        runs.append((ctx.xbar().clone(), ctx.x().clone()))
    assert torch.equal(runs[0][0], runs[1][0]) and torch.equal(runs[0][1], runs[1][1])
    rnd = {"bf16": O.round_bf16, "f32": lambda q: q.astype(np.float32).astype(np.float64), "f64": lambda q: q}[prec]
    Qr = [rnd(Q) for Q, _ in QR]
    xs0 = [Qt @ O.block_coefficients(Q, R, bi) for Qt, (Q, R), (_, bi) in zip(Qr, QR, bl)]
    ref = O.apc_run(A, b, offs, g, e, max_iters=T, Qs=Qr, xs0=xs0)
    xb = runs[0][0].cpu().numpy()
    tol = 1e-10 if prec == "f64" else max(1e-5, abs(e) * T * 2.0 ** -24)
    assert np.linalg.norm(xb - ref.xbar) <= tol * np.linalg.norm(ref.xbar)


@pytest.mark.parametrize("prec", ["bf16", "f64"])
def test_export_import_resumes_bit_for_bit(prec):
    apc, dev = _env()
    n, m, T = 1536, 12, 30
    A, b, offs, bl, QR, g, e = _system(n, m, 92)
    At, bt = torch.tensor(A, device=dev), torch.tensor(b, device=dev)
    c1 = apc.apc_setup(At, bt, offs, precision=prec)
    c1.set_deterministic(True)
    c1.reset()
    c1.iterate(g, e, T)
    state = c1.export_state()
    mon = c1.monitor()
    c1.iterate(g, e, T)
    want_xbar, want_x = c1.xbar().clone(), c1.x().clone()
    c2 = apc.apc_setup(At, bt, offs, precision=prec)
    c2.set_deterministic(True)
    c2.import_state(state)
    assert c2.monitor() == pytest.approx(mon, rel=1e-12)  # its block sums are added by atomics
    c2.iterate(g, e, T)
    assert torch.equal(c2.xbar(), want_xbar)
    assert torch.equal(c2.x(), want_x)
    # the exporting context itself can go back to the checkpoint
    c1.import_state(state)
    c1.iterate(g, e, T)
    assert torch.equal(c1.xbar(), want_xbar)


def test_import_rejects_a_state_of_another_shape():
    apc, dev = _env()
    A, b, offs, bl, QR, g, e = _system(512, 8, 93)
    At, bt = torch.tensor(A, device=dev), torch.tensor(b, device=dev)
    c1 = apc.apc_setup(At, bt, offs, precision="f32")
    c1.reset()
    state = c1.export_state()
    c2 = apc.apc_setup(At, bt, inputs.even_offsets(512, 4), precision="f32")
    with pytest.raises(apc.ApcError) as ei:
        c2.import_state(state)
    assert ei.value.name == "INVALID_ARG"
    c3 = apc.apc_setup(At, bt, offs, precision="bf16")
    with pytest.raises(apc.ApcError) as ei:
        c3.import_state(state)
    assert ei.value.name == "INVALID_ARG"
    with pytest.raises(apc.ApcError) as ei:
        c1.import_state(state[: len(state) // 2])
    assert ei.value.name == "INVALID_ARG"
