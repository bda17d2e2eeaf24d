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
