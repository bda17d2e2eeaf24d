"""The allocation-free residual entry point (apc_residual_noalloc) against the
context-based apc_residual, through the C ABI, on two calls in a row.

apc_residual_noalloc serves callers that cannot allocate device memory when
they need the check; its working memory is a fixed array inside the library,
shared by all calls.  This file is collected last so that a failure here does
not stop a `-x` run before the other tests."""
import numpy as np
import pytest

from paper_1708_01413_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _env():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1708_01413_gb300 import apc, build
    build.build()
    return apc, torch.device("cuda:0")


def test_noalloc_residual_matches_context_residual_twice():
    apc, dev = _env()
    N, n, m = 2500, 2200, 10  # tall; several hundred row blocks of the residual kernel, ragged tail
    A, _, b = inputs.gaussian_system(n, 21, N=N)
    offs = inputs.even_offsets(N, m)
    At, bt = torch.tensor(A, device=dev), torch.tensor(b, device=dev)
    ctx = apc.apc_setup(At, bt, offs, precision="f64")
    rng = np.random.default_rng(5)
    for call in range(2):
        x = torch.tensor(rng.standard_normal(n), device=dev)
        ref_vec = torch.empty(N, dtype=torch.float64, device=dev)
        ref_rel = ctx.residual(x, resid_out=ref_vec)
        out = torch.full((N,), float("nan"), dtype=torch.float64, device=dev)
        rel = apc.apc_residual_noalloc(At, x, bt, resid_out=out)
        assert rel == pytest.approx(ref_rel, rel=1e-12), call
        diff = (out - ref_vec).abs().max().item()
        assert diff <= 1e-12 * ref_vec.abs().max().item(), call
        # against the plain definition as well
        assert rel == pytest.approx(np.linalg.norm(b - A @ x.cpu().numpy()) / np.linalg.norm(b), rel=1e-12)


def test_noalloc_residual_rejects_sizes_beyond_its_array():
    apc, dev = _env()
    import ctypes as C
    L = apc.lib()
    rel = C.c_double()
    dummy = C.c_void_p(16)  # never dereferenced: the size check comes first
    rc = L.apc_residual_noalloc(dummy, 8, 1 << 21, 8, dummy, dummy, None, C.byref(rel), None)
    assert apc.ERRORS[rc] == "UNSUPPORTED"
    assert b"static scratch limit" in L.apc_last_error(None)


@pytest.mark.parametrize("n", [2048, 4096])
def test_noalloc_residual_chunk_boundaries_strided_rows_and_no_vector(n):
    # n a whole number of the kernel's 2048-column chunks (no ragged last
    # chunk), A read as the left n columns of a wider matrix (lda > n), and no
    # residual vector requested; checked against the context-based residual
    # and against the plain definition, on two calls in a row
    apc, dev = _env()
    N, extra = n + 40, 24
    m = (N + 199) // 200  # blocks of at most 200 rows
    A, _, b = inputs.gaussian_system(n, 22, N=N)
    wide = np.concatenate([A, np.random.default_rng(1).standard_normal((N, extra))], axis=1)
    Aw = torch.tensor(wide, device=dev)[:, :n]
    assert Aw.stride(0) == n + extra
    At, bt = torch.tensor(A, device=dev), torch.tensor(b, device=dev)
    ctx = apc.apc_setup(At, bt, inputs.even_offsets(N, m), precision="f64")
    rng = np.random.default_rng(6)
    for call in range(2):
        x = torch.tensor(rng.standard_normal(n), device=dev)
        ref_rel = ctx.residual(x)
        rel = apc.apc_residual_noalloc(Aw, x, bt)
        assert rel == pytest.approx(ref_rel, rel=1e-12), call
        assert rel == pytest.approx(np.linalg.norm(b - A @ x.cpu().numpy()) / np.linalg.norm(b), rel=1e-12)
        out = torch.full((N,), float("nan"), dtype=torch.float64, device=dev)
        rel2 = apc.apc_residual_noalloc(Aw, x, bt, resid_out=out)
        assert rel2 == rel
        assert np.allclose(out.cpu().numpy(), b - A @ x.cpu().numpy(), rtol=0, atol=1e-12 * np.abs(b).max() * n)


def test_noalloc_wrapper_rejects_mismatched_lengths_before_launch():
    # the kernel trusts N, n and the vectors' lengths, so the binding checks
    # them on the host; nothing is launched and the vectors stay untouched
    apc, dev = _env()
    N, n = 300, 200
    A = torch.randn((N, n), dtype=torch.float64, device=dev)
    x = torch.randn(n, dtype=torch.float64, device=dev)
    rhs = torch.randn(N, dtype=torch.float64, device=dev)
    out = torch.zeros(N, dtype=torch.float64, device=dev)
    for bad in (dict(x=x[:-1]), dict(rhs=rhs[:-1]), dict(resid_out=out[:-1]), dict(resid_out=torch.zeros(2 * N, dtype=torch.float64, device=dev)[::2]),
                dict(x=torch.randn(n + 1, dtype=torch.float64, device=dev))):
        args = dict(x=x, rhs=rhs, resid_out=out)
        args.update(bad)
        with pytest.raises(ValueError):
            apc.apc_residual_noalloc(A, args["x"], args["rhs"], resid_out=args["resid_out"])
    assert float(out.abs().max()) == 0.0
