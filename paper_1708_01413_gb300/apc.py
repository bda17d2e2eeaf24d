"""Thin ctypes binding of the C ABI in ``include/apc.h`` and ``include/apc_batch.h``.

Argument marshalling only: every step of the solver runs in the CUDA library
``_build/libapc.so``.  PyTorch supplies device memory (tensors are passed by
``data_ptr()``) and the current CUDA stream.  There is no CPU fallback: if the
library is missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libapc.so")

APC_F64, APC_F32, APC_BF16 = 0, 1, 2
PRECISIONS = {"f64": APC_F64, "f32": APC_F32, "bf16": APC_BF16}

ERRORS = {
    0: "OK", -1: "INVALID_ARG", -2: "SINGULAR_BLOCK", -3: "NONFINITE", -4: "PARAMS",
    -5: "NOT_CONVERGED", -6: "DIVERGED", -7: "LAUNCH", -8: "TIMEOUT", -9: "CUDA",
    -10: "UNSUPPORTED", -11: "NOMEM",
}

# Every function the header declares; tests check the library exports them.
EXPORTED = (
    "apc_setup", "apc_optimal_params", "apc_reset", "apc_iterate", "apc_get_xbar", "apc_get_x",
    "apc_get_basis", "apc_residual", "apc_solve", "apc_backward", "apc_backward_params", "apc_set_test_hooks", "apc_context_info", "apc_last_error", "apc_destroy",
    "apc_spectral_bounds", "apc_setup_rows", "apc_hb_optimal_params", "apc_batch_set_hb_params",
    "apc_batch_setup", "apc_batch_set_params", "apc_batch_reset", "apc_batch_iterate", "apc_batch_get_xbar",
    "apc_batch_get_x", "apc_batch_set_test_hooks", "apc_batch_info", "apc_batch_last_error", "apc_batch_destroy",
    "apc_residual_noalloc", "apc_forward_rhs", "apc_backward_rhs", "apc_batch_forward", "apc_batch_backward",
    "apc_monitor", "apc_set_deterministic", "apc_state_bytes", "apc_export_state", "apc_import_state",
    "apc_batch_set_tiles", "apc_batch_get_tiles", "apc_batch_autotune", "apc_solve_rhs", "apc_setup_report",
)


class ApcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"APC_ERR_{ERRORS.get(code, code)} ({code}): {msg}")
        self.code = code
        self.name = ERRORS.get(code, str(code))


class apc_options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("cluster_size", C.c_int32), ("workers_per_warp", C.c_int32),
                ("timeout_s", C.c_double), ("rows_per_group", C.c_int32)]


class apc_stats(C.Structure):
    _fields_ = [("iterations", C.c_int64), ("sweeps", C.c_int32), ("rel_residual", C.c_double),
                ("seconds", C.c_double), ("residual_checks", C.c_int64), ("monitor_checks", C.c_int64)]


_lib = None


def lib() -> C.CDLL:
    """Load libapc.so (built by ``build.build()``); raise if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
    L = C.CDLL(LIB_PATH)
    vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int32, C.c_double
    L.apc_setup.argtypes = [C.POINTER(vp), vp, i64, i64, i64, vp, C.POINTER(i64), i32,
                            C.POINTER(apc_options), vp]
    L.apc_setup_rows.argtypes = [C.POINTER(vp), vp, i64, i64, i64, vp, C.POINTER(i64), C.POINTER(i64), i32,
                                 C.POINTER(apc_options), vp]
    L.apc_optimal_params.argtypes = [dbl, dbl, C.POINTER(dbl), C.POINTER(dbl), C.POINTER(dbl)]
    L.apc_reset.argtypes = [vp, vp, vp]
    L.apc_iterate.argtypes = [vp, dbl, dbl, i64, vp]
    L.apc_get_xbar.argtypes = [vp, vp, vp]
    L.apc_get_x.argtypes = [vp, vp, i64, vp]
    L.apc_get_basis.argtypes = [vp, i32, vp, i64, vp]
    L.apc_residual.argtypes = [vp, vp, vp, vp, C.POINTER(dbl), vp]
    L.apc_solve.argtypes = [vp, dbl, dbl, dbl, i64, i64, i32, vp, C.POINTER(apc_stats), vp]
    L.apc_context_info.argtypes = [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i32), C.POINTER(i32),
                                   C.POINTER(i32), C.POINTER(i32), C.POINTER(i64), C.POINTER(i32)]
    L.apc_backward.argtypes = [vp, vp, i64, dbl, dbl, vp, vp]
    L.apc_backward_params.argtypes = [vp, vp, vp, i64, dbl, dbl, i32, vp, C.POINTER(dbl), C.POINTER(dbl), vp]
    L.apc_set_test_hooks.argtypes = [vp, i32, dbl]
    L.apc_spectral_bounds.argtypes = [vp, i32, C.c_uint64, C.POINTER(dbl), C.POINTER(dbl), vp]
    L.apc_residual_noalloc.argtypes = [vp, i64, i64, i64, vp, vp, vp, C.POINTER(dbl), vp]
    L.apc_forward_rhs.argtypes = [vp, vp, i64, i64, i64, dbl, dbl, vp, i64, vp]
    L.apc_monitor.argtypes = [vp, C.POINTER(dbl), vp]
    L.apc_setup_report.argtypes = [vp, C.POINTER(i32), C.POINTER(dbl)]
    L.apc_solve_rhs.argtypes = [vp, vp, i64, i64, dbl, dbl, dbl, i64, i64, i32, vp, i64, C.POINTER(apc_stats), vp]
    L.apc_set_deterministic.argtypes = [vp, i32]
    L.apc_state_bytes.argtypes = [vp, C.POINTER(C.c_size_t)]
    L.apc_export_state.argtypes = [vp, vp, C.c_size_t, vp]
    L.apc_import_state.argtypes = [vp, vp, C.c_size_t, vp]
    L.apc_backward_rhs.argtypes = [vp, vp, i64, i64, i64, dbl, dbl, vp, i64, vp]
    L.apc_batch_forward.argtypes = [vp, C.POINTER(vp), i64, C.POINTER(vp), vp]
    L.apc_batch_set_tiles.argtypes = [vp, i32, i32, i32, i32, i32, i32]
    L.apc_batch_get_tiles.argtypes = [vp] + [C.POINTER(i32)] * 6
    L.apc_batch_autotune.argtypes = [vp, i64, i32, C.POINTER(i32), C.POINTER(dbl), C.POINTER(dbl), vp]
    L.apc_batch_backward.argtypes = [vp, C.POINTER(vp), i64, C.POINTER(vp), vp]
    L.apc_last_error.argtypes = [vp]
    L.apc_last_error.restype = C.c_char_p
    L.apc_destroy.argtypes = [vp]
    L.apc_destroy.restype = None
    L.apc_batch_setup.argtypes = [C.POINTER(vp), i32, C.POINTER(i64), C.POINTER(i32), C.POINTER(i64),
                                  C.POINTER(vp), C.POINTER(vp), i32, C.POINTER(apc_options), vp]
    L.apc_batch_set_params.argtypes = [vp, C.POINTER(dbl), C.POINTER(dbl)]
    L.apc_batch_set_hb_params.argtypes = [vp, C.POINTER(dbl), C.POINTER(dbl)]
    L.apc_hb_optimal_params.argtypes = [dbl, dbl, i32, C.POINTER(dbl), C.POINTER(dbl), C.POINTER(dbl)]
    L.apc_batch_reset.argtypes = [vp, vp, vp]
    L.apc_batch_iterate.argtypes = [vp, i64, vp]
    L.apc_batch_get_xbar.argtypes = [vp, i32, vp, i64, vp]
    L.apc_batch_get_x.argtypes = [vp, i32, i32, vp, i64, vp]
    L.apc_batch_set_test_hooks.argtypes = [vp, i32, dbl]
    L.apc_batch_info.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i64), C.POINTER(i64),
                                 C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]
    L.apc_batch_last_error.argtypes = [vp]
    L.apc_batch_last_error.restype = C.c_char_p
    L.apc_batch_destroy.argtypes = [vp]
    L.apc_batch_destroy.restype = None
    for name in EXPORTED:
        if name not in ("apc_last_error", "apc_destroy", "apc_batch_last_error", "apc_batch_destroy"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return C.c_void_p(0 if t is None else t.data_ptr())


def _check(rc: int, ctx=None):
    if rc != 0:
        msg = lib().apc_last_error(ctx).decode(errors="replace")
        raise ApcError(rc, msg)


def apc_hb_optimal_params(mu_min: float, mu_max: float, m: int):
    """(alpha, beta, rho) of heavy ball on the Sec. 6 preconditioned system."""
    a, b, r = C.c_double(), C.c_double(), C.c_double()
    _check(lib().apc_hb_optimal_params(mu_min, mu_max, int(m), C.byref(a), C.byref(b), C.byref(r)))
    return a.value, b.value, r.value


def apc_optimal_params(mu_min: float, mu_max: float):
    """Theorem 1's (gamma*, eta*, rho) from the extreme eigenvalues of X."""
    g, e, r = C.c_double(), C.c_double(), C.c_double()
    _check(lib().apc_optimal_params(mu_min, mu_max, C.byref(g), C.byref(e), C.byref(r)))
    return g.value, e.value, r.value


class Context:
    """Owns an ``apc_ctx``; methods mirror the C entry points."""

    def __init__(self, handle: C.c_void_p, device, offsets=None):
        self.handle = handle
        self.device = device
        self._offs = offsets

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def close(self):
        if self.handle:
            lib().apc_destroy(self.handle)
            self.handle = None

    def info(self) -> dict:
        n, N, cb = C.c_int64(), C.c_int64(), C.c_int64()
        m, w, cs, cl, rg = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        _check(lib().apc_context_info(self.handle, C.byref(n), C.byref(N), C.byref(m), C.byref(w),
                                      C.byref(cs), C.byref(cl), C.byref(cb), C.byref(rg)), self.handle)
        return dict(n=n.value, N=N.value, m=m.value, width=w.value, cluster_size=cs.value,
                    clusters=cl.value, q_bytes=cb.value, rows_per_group=rg.value)

    def setup_report(self) -> dict:
        """Cholesky-QR passes taken at set-up and the first pass's probed
        departure from orthogonality (apc_setup_report)."""
        n, e = C.c_int32(), C.c_double()
        _check(lib().apc_setup_report(self.handle, C.byref(n), C.byref(e)), self.handle)
        return {"qr_passes": n.value, "orth_probe": e.value}

    def reset(self, rhs=None, stream=None):
        _check(lib().apc_reset(self.handle, _ptr(rhs), _stream(stream)), self.handle)

    def iterate(self, gamma: float, eta: float, iters: int, stream=None):
        _check(lib().apc_iterate(self.handle, gamma, eta, int(iters), _stream(stream)), self.handle)

    def xbar(self, out=None, stream=None):
        import torch
        info_n = self.info()["n"]
        out = torch.empty(info_n, dtype=torch.float64, device=self.device) if out is None else out
        _check(lib().apc_get_xbar(self.handle, _ptr(out), _stream(stream)), self.handle)
        return out

    def x(self, stream=None):
        import torch
        inf = self.info()
        out = torch.empty((inf["m"], inf["n"]), dtype=torch.float64, device=self.device)
        _check(lib().apc_get_x(self.handle, _ptr(out), inf["n"], _stream(stream)), self.handle)
        return out

    def basis(self, block: int, stream=None):
        """Q_i of block ``block`` as an n x p_i FP64 tensor."""
        import torch
        inf = self.info()
        p = int(self._offs[block + 1] - self._offs[block])
        out = torch.empty((inf["n"], p), dtype=torch.float64, device=self.device)
        _check(lib().apc_get_basis(self.handle, int(block), _ptr(out), p, _stream(stream)), self.handle)
        return out

    def residual(self, x, rhs=None, resid_out=None, stream=None) -> float:
        rel = C.c_double()
        _check(lib().apc_residual(self.handle, _ptr(x), _ptr(rhs), _ptr(resid_out), C.byref(rel),
                                  _stream(stream)), self.handle)
        return rel.value

    def set_deterministic(self, on: bool = True):
        """Fixed-order reduction of the clusters' partial sums (bit-for-bit
        reproducible trajectories; apc_set_deterministic)."""
        _check(lib().apc_set_deterministic(self.handle, int(bool(on))), self.handle)

    def export_state(self, stream=None) -> bytes:
        """The iteration state (x_i, xbar, z buffers, pass counter) as bytes."""
        size = C.c_size_t()
        _check(lib().apc_state_bytes(self.handle, C.byref(size)), self.handle)
        buf = C.create_string_buffer(size.value)
        _check(lib().apc_export_state(self.handle, buf, size.value, _stream(stream)), self.handle)
        return buf.raw

    def import_state(self, state: bytes, stream=None):
        """Load a state from export_state of a context of the same shape."""
        buf = C.create_string_buffer(bytes(state), len(state))
        _check(lib().apc_import_state(self.handle, buf, len(state), _stream(stream)), self.handle)

    def monitor(self, stream=None) -> float:
        """The free residual monitor ||r - A xbar|| / ||r|| of the current
        state (apc_monitor), without reading A."""
        rel = C.c_double()
        _check(lib().apc_monitor(self.handle, C.byref(rel), _stream(stream)), self.handle)
        return rel.value

    def spectral_bounds(self, steps: int = 100, seed: int = 1, stream=None):
        """Lanczos estimates (mu_min, mu_max) of the extreme eigenvalues of X
        (Ritz values: inside the spectrum)."""
        lo, hi = C.c_double(), C.c_double()
        _check(lib().apc_spectral_bounds(self.handle, int(steps), C.c_uint64(seed), C.byref(lo), C.byref(hi),
                                         _stream(stream)), self.handle)
        return lo.value, hi.value

    def set_test_hooks(self, grid_barrier_skew: int = 0, timeout_s: float = 2.0):
        """Failure injection for tests (see apc_set_test_hooks in the header)."""
        _check(lib().apc_set_test_hooks(self.handle, int(grid_barrier_skew), float(timeout_s)), self.handle)

    def backward(self, g, T: int, gamma: float, eta: float, out=None, stream=None):
        """dL/db for L depending on xbar(T) through T iterations from the
        least-norm initialisation; g = dL/dxbar(T) (FP64, n)."""
        import torch
        N = self.info()["N"]
        out = torch.empty(N, dtype=torch.float64, device=self.device) if out is None else out
        _check(lib().apc_backward(self.handle, _ptr(g.contiguous()), int(T), gamma, eta, _ptr(out),
                                  _stream(stream)), self.handle)
        return out

    def backward_params(self, g, T: int, gamma: float, eta: float, b=None, ckpt_every: int = 20, out=None,
                        stream=None):
        """(dL/db, dL/dgamma, dL/deta) through T iterations from the least-norm
        start for right-hand side b (None: the b of set-up); the forward states
        are recomputed from checkpoints every ``ckpt_every`` iterations."""
        import torch
        N = self.info()["N"]
        out = torch.empty(N, dtype=torch.float64, device=self.device) if out is None else out
        dg, de = C.c_double(), C.c_double()
        _check(lib().apc_backward_params(self.handle, _ptr(g.contiguous()), _ptr(b.contiguous() if b is not None else None),
                                         int(T), gamma, eta, int(ckpt_every), _ptr(out), C.byref(dg), C.byref(de),
                                         _stream(stream)), self.handle)
        return out, dg.value, de.value

    def _rhs_matrix(self, B, rows):
        import torch
        if not B.is_cuda or B.dtype != torch.float64:
            raise TypeError("float64 CUDA tensors expected")
        B = B.unsqueeze(1) if B.dim() == 1 else B
        if B.dim() != 2 or B.shape[0] != rows or B.stride(1) != 1:
            raise ValueError(f"expected a row-major ({rows}, k) tensor, got {tuple(B.shape)}")
        return B

    def forward_rhs(self, B, T: int, gamma: float, eta: float, out=None, stream=None):
        """xbar(T) for every column of B (N x k) from the least-norm start, in
        one call (apc_forward_rhs); returns an n x k FP64 tensor."""
        import torch
        inf = self.info()
        B = self._rhs_matrix(B, inf["N"])
        k = B.shape[1]
        out = torch.empty((inf["n"], k), dtype=torch.float64, device=self.device) if out is None else out
        with torch.cuda.device(self.device):
            _check(lib().apc_forward_rhs(self.handle, _ptr(B), k, B.stride(0), int(T), float(gamma), float(eta),
                                         _ptr(out), out.stride(0), _stream(stream)), self.handle)
        return out

    def backward_rhs(self, G, T: int, gamma: float, eta: float, out=None, stream=None):
        """dL/dB (N x k) from G = dL/dxbar(T) (n x k) through the map of
        forward_rhs, in one call (apc_backward_rhs)."""
        import torch
        inf = self.info()
        G = self._rhs_matrix(G, inf["n"])
        k = G.shape[1]
        out = torch.empty((inf["N"], k), dtype=torch.float64, device=self.device) if out is None else out
        with torch.cuda.device(self.device):
            _check(lib().apc_backward_rhs(self.handle, _ptr(G), k, G.stride(0), int(T), float(gamma), float(eta),
                                          _ptr(out), out.stride(0), _stream(stream)), self.handle)
        return out

    def solve_rhs(self, B, gamma, eta, tol=1e-10, max_iters=10**6, check_every=100, refine=False, stream=None,
                  raise_on_error=True):
        """apc_solve for every column of B (N x k) in one call (apc_solve_rhs);
        returns (X n x k, stats summed over the columns)."""
        import torch
        inf = self.info()
        B = self._rhs_matrix(B, inf["N"])
        k = B.shape[1]
        out = torch.empty((inf["n"], k), dtype=torch.float64, device=self.device)
        st = apc_stats()
        with torch.cuda.device(self.device):
            rc = lib().apc_solve_rhs(self.handle, _ptr(B), k, B.stride(0), float(gamma), float(eta), float(tol),
                                     int(max_iters), int(check_every), int(bool(refine)), _ptr(out), out.stride(0),
                                     C.byref(st), _stream(stream))
        stats = dict(iterations=st.iterations, sweeps=st.sweeps, rel_residual=st.rel_residual, seconds=st.seconds,
                     residual_checks=st.residual_checks, monitor_checks=st.monitor_checks, rc=rc)
        if rc != 0 and raise_on_error:
            _check(rc, self.handle)
        return out, stats

    def solve(self, gamma, eta, tol=1e-10, max_iters=10**6, check_every=100, refine=False,
              out=None, stream=None, raise_on_error=True):
        import torch
        n = self.info()["n"]
        out = torch.empty(n, dtype=torch.float64, device=self.device) if out is None else out
        st = apc_stats()
        rc = lib().apc_solve(self.handle, gamma, eta, tol, int(max_iters), int(check_every), int(bool(refine)),
                             _ptr(out), C.byref(st), _stream(stream))
        stats = dict(iterations=st.iterations, sweeps=st.sweeps, rel_residual=st.rel_residual,
                     seconds=st.seconds, residual_checks=st.residual_checks, monitor_checks=st.monitor_checks, rc=rc)
        if rc != 0 and raise_on_error:
            _check(rc, self.handle)
        return out, stats


class APCSolveFn:
    """Differentiable T-iteration APC solve, xbar(T) = F(b, gamma, eta), for torch.autograd.

    ``APCSolveFn.apply(b, ctx, gamma, eta, T, ckpt_every=20)``: b is an FP64
    CUDA tensor of shape (N,) or (N, k); gamma and eta are numbers or 0-d
    tensors.  With only b differentiated, each direction is one call into the
    library for all k columns: ``Context.forward_rhs`` and
    ``Context.backward_rhs`` (on a BF16 context of a square system with
    2 <= k <= 32 the columns run together on the tensor cores in the form of
    App. A; otherwise column after column inside the call).  When gamma or eta
    is a tensor that requires grad, the columns go one after another through
    the single-system iteration, and dL/dgamma, dL/deta (summed over the
    columns) come from ``Context.backward_params`` with forward checkpoints
    every ``ckpt_every`` iterations."""

    _fn = None

    @classmethod
    def apply(cls, b, ctx, gamma, eta, T, ckpt_every=20):
        if cls._fn is None:
            import torch

            class _F(torch.autograd.Function):
                @staticmethod
                def forward(fctx, b, solver, gamma, eta, T, ckpt_every):
                    g, e = float(gamma), float(eta)
                    params = any(torch.is_tensor(p) and p.requires_grad for p in (gamma, eta))
                    cols = b.unsqueeze(1) if b.dim() == 1 else b
                    if params:
                        outs = []
                        for j in range(cols.shape[1]):
                            solver.reset(cols[:, j].contiguous())
                            solver.iterate(g, e, T)
                            outs.append(solver.xbar())
                        x = torch.stack(outs, dim=1)
                    else:
                        x = solver.forward_rhs(cols.contiguous(), T, g, e)
                    fctx.save_for_backward(b)
                    fctx.solver, fctx.g, fctx.e, fctx.T, fctx.ck = solver, g, e, T, ckpt_every
                    fctx.vec, fctx.params = b.dim() == 1, params
                    fctx.like = (gamma if torch.is_tensor(gamma) else None, eta if torch.is_tensor(eta) else None)
                    return x[:, 0] if b.dim() == 1 else x

                @staticmethod
                def backward(fctx, gx):
                    (b,) = fctx.saved_tensors
                    gcols = gx.unsqueeze(1) if fctx.vec else gx
                    bcols = b.unsqueeze(1) if fctx.vec else b
                    dg = de = 0.0
                    if fctx.params:
                        dbs = []
                        for j in range(gcols.shape[1]):
                            db, dgj, dej = fctx.solver.backward_params(gcols[:, j].contiguous(), fctx.T, fctx.g,
                                                                       fctx.e, b=bcols[:, j].contiguous(),
                                                                       ckpt_every=fctx.ck)
                            dg, de = dg + dgj, de + dej
                            dbs.append(db)
                        db = torch.stack(dbs, dim=1)
                    else:
                        db = fctx.solver.backward_rhs(gcols.contiguous(), fctx.T, fctx.g, fctx.e)
                    grads = []
                    for k, val in ((2, dg), (3, de)):
                        ref = fctx.like[k - 2]
                        grads.append(torch.tensor(val, dtype=ref.dtype, device=ref.device)
                                     if fctx.needs_input_grad[k] and ref is not None else None)
                    return (db[:, 0] if fctx.vec else db), None, grads[0], grads[1], None, None

            cls._fn = _F
        return cls._fn.apply(b, ctx, gamma, eta, T, ckpt_every)


def apc_residual_noalloc(A, x, rhs, resid_out=None, stream=None) -> float:
    """||rhs - A x|| / ||rhs|| in FP64 without any device allocation (see the
    header): A is an N x n row-major FP64 CUDA tensor (rows may be strided, so
    a column slice of a wider matrix is accepted), x an n-vector and rhs an
    N-vector (FP64, contiguous), resid_out an optional contiguous N-vector
    receiving rhs - A x.  Every tensor must be on one device; the call runs
    with that device current.  Lengths are checked here, before anything is
    launched, because the kernel trusts them."""
    import torch
    ts = (A, x, rhs) + ((resid_out,) if resid_out is not None else ())
    for t in ts:
        if not t.is_cuda or t.dtype != torch.float64:
            raise TypeError("float64 CUDA tensors expected")
    if any(t.device != A.device for t in ts):
        raise ValueError("A, x, rhs and resid_out must be on one device")
    if A.dim() != 2 or A.stride(1) != 1 or A.shape[0] < 1 or A.shape[1] < 1:
        raise ValueError("A must be a non-empty 2-D tensor with unit column stride")
    N, n = int(A.shape[0]), int(A.shape[1])
    if not x.is_contiguous() or x.numel() != n:
        raise ValueError(f"x must be a contiguous vector of n = {n} values, got {tuple(x.shape)}")
    if not rhs.is_contiguous() or rhs.numel() != N:
        raise ValueError(f"rhs must be a contiguous vector of N = {N} values, got {tuple(rhs.shape)}")
    if resid_out is not None and (not resid_out.is_contiguous() or resid_out.numel() != N):
        raise ValueError(f"resid_out must be a contiguous vector of N = {N} values, got {tuple(resid_out.shape)}")
    rel = C.c_double()
    with torch.cuda.device(A.device):
        _check(lib().apc_residual_noalloc(_ptr(A), A.stride(0), N, n, _ptr(x), _ptr(rhs), _ptr(resid_out),
                                          C.byref(rel), _stream(stream)))
    return rel.value


def apc_setup_rows(A, b, row_sets, precision="f32", cluster_size=0, timeout_s=0.0, stream=None,
                   workers_per_warp=0, rows_per_group=0) -> Context:
    """Factor a partition whose blocks are arbitrary row sets: block i holds
    the rows ``row_sets[i]`` of A (FP64 CUDA tensor, N x n) and b."""
    import numpy as np
    import torch
    if not (A.is_cuda and b.is_cuda) or A.dtype != torch.float64 or b.dtype != torch.float64:
        raise TypeError("A and b must be float64 CUDA tensors")
    if A.dim() != 2 or A.stride(1) != 1:
        raise ValueError("A must be a row-major 2-D tensor")
    b = b.contiguous()
    sets = [np.asarray(r, dtype=np.int64) for r in row_sets]
    index = np.ascontiguousarray(np.concatenate(sets))
    offs = np.ascontiguousarray(np.concatenate([[0], np.cumsum([len(r) for r in sets])]).astype(np.int64))
    opt = apc_options(PRECISIONS[precision] if isinstance(precision, str) else int(precision),
                      int(cluster_size), int(workers_per_warp), float(timeout_s), int(rows_per_group))
    h = C.c_void_p()
    with torch.cuda.device(A.device):
        rc = lib().apc_setup_rows(C.byref(h), _ptr(A), A.shape[0], A.shape[1], A.stride(0), _ptr(b),
                                  index.ctypes.data_as(C.POINTER(C.c_int64)),
                                  offs.ctypes.data_as(C.POINTER(C.c_int64)), len(sets), C.byref(opt),
                                  _stream(stream))
    _check(rc, None)
    return Context(h, A.device, offs)


def apc_setup(A, b, row_offsets, precision="f32", cluster_size=0, timeout_s=0.0, stream=None,
              workers_per_warp=0, rows_per_group=0) -> Context:
    """Factor the row blocks of A (FP64 CUDA tensor, N x n) for right-hand side b."""
    import numpy as np
    import torch
    if not (A.is_cuda and b.is_cuda) or A.dtype != torch.float64 or b.dtype != torch.float64:
        raise TypeError("A and b must be float64 CUDA tensors")
    if A.dim() != 2 or A.stride(1) != 1:
        raise ValueError("A must be a row-major 2-D tensor")
    b = b.contiguous()
    offs = np.ascontiguousarray(np.asarray(row_offsets, dtype=np.int64))
    m = len(offs) - 1
    opt = apc_options(PRECISIONS[precision] if isinstance(precision, str) else int(precision),
                      int(cluster_size), int(workers_per_warp), float(timeout_s), int(rows_per_group))
    h = C.c_void_p()
    with torch.cuda.device(A.device):
        rc = lib().apc_setup(C.byref(h), _ptr(A), A.shape[0], A.shape[1], A.stride(0), _ptr(b),
                             offs.ctypes.data_as(C.POINTER(C.c_int64)), m, C.byref(opt), _stream(stream))
    _check(rc, None)
    return Context(h, A.device, offs)


def _check_batch(rc: int, handle=None):
    if rc != 0:
        msg = lib().apc_batch_last_error(handle).decode(errors="replace")
        raise ApcError(rc, msg)


class Batch:
    """Owns an ``apc_batch``: independent square systems advanced together."""

    def __init__(self, handle: C.c_void_p, device, n, k, B, key=None):
        self.handle = handle
        self.device = device
        self.n = list(n)
        self.k = k
        self._B = B  # the caller's right-hand sides (kept alive for reset)
        self.key = key  # tile-cache key (tile_cache_key)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def close(self):
        if self.handle:
            lib().apc_batch_destroy(self.handle)
            self.handle = None

    def info(self) -> dict:
        ns, k, grid, ua, ub = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        qb, sb = C.c_int64(), C.c_int64()
        _check_batch(lib().apc_batch_info(self.handle, C.byref(ns), C.byref(k), C.byref(qb), C.byref(sb),
                                          C.byref(grid), C.byref(ua), C.byref(ub)), self.handle)
        return {"nsys": ns.value, "k": k.value, "q_bytes": qb.value, "state_bytes": sb.value,
                "grid": grid.value, "units_a": ua.value, "units_b": ub.value}

    def set_params(self, gammas, etas):
        import numpy as np
        g = np.ascontiguousarray(np.asarray(gammas, dtype=np.float64))
        e = np.ascontiguousarray(np.asarray(etas, dtype=np.float64))
        if g.shape != (len(self.n),) or e.shape != (len(self.n),):
            raise ValueError("one gamma and one eta per system")
        _check_batch(lib().apc_batch_set_params(self.handle, g.ctypes.data_as(C.POINTER(C.c_double)),
                                                e.ctypes.data_as(C.POINTER(C.c_double))), self.handle)

    def set_hb_params(self, alphas, betas):
        """Switch to the preconditioned heavy-ball method (Sec. 4.3 / Sec. 6)."""
        import numpy as np
        a = np.ascontiguousarray(np.asarray(alphas, dtype=np.float64))
        b_ = np.ascontiguousarray(np.asarray(betas, dtype=np.float64))
        if a.shape != (len(self.n),) or b_.shape != (len(self.n),):
            raise ValueError("one alpha and one beta per system")
        _check_batch(lib().apc_batch_set_hb_params(self.handle, a.ctypes.data_as(C.POINTER(C.c_double)),
                                                   b_.ctypes.data_as(C.POINTER(C.c_double))), self.handle)

    def reset(self, B=None, stream=None):
        arr = None
        if B is not None:
            B = [_batch_rhs(b_, n_, self.k) for b_, n_ in zip(B, self.n)]
            arr = (C.c_void_p * len(B))(*[b_.data_ptr() for b_ in B])
            self._B = B
        with _device(self.device):
            _check_batch(lib().apc_batch_reset(self.handle, arr, _stream(stream)), self.handle)

    def iterate(self, iters: int, stream=None):
        with _device(self.device):
            _check_batch(lib().apc_batch_iterate(self.handle, int(iters), _stream(stream)), self.handle)

    def xbar(self, s: int, stream=None):
        import torch
        out = torch.empty((self.n[s], self.k), dtype=torch.float64, device=self.device)
        with _device(self.device):
            _check_batch(lib().apc_batch_get_xbar(self.handle, s, _ptr(out), self.k, _stream(stream)), self.handle)
        return out

    def x(self, s: int, worker: int, stream=None):
        import torch
        out = torch.empty((self.n[s], self.k), dtype=torch.float64, device=self.device)
        with _device(self.device):
            _check_batch(lib().apc_batch_get_x(self.handle, s, worker, _ptr(out), self.k, _stream(stream)),
                         self.handle)
        return out

    def set_test_hooks(self, grid_barrier_skew: int = 0, timeout_s: float = 0.0):
        _check_batch(lib().apc_batch_set_test_hooks(self.handle, int(grid_barrier_skew), float(timeout_s)),
                     self.handle)

    def set_tiles(self, rows_a: int, cols_b: int, prefetch: int, l2: int = 0, split_a: int = 1, split_b: int = 1):
        """Work-unit shape, prefetch distance, L2 policy and unit splits of the
        persistent kernel (apc_batch_set_tiles)."""
        _check_batch(lib().apc_batch_set_tiles(self.handle, int(rows_a), int(cols_b), int(prefetch), int(l2),
                                               int(split_a), int(split_b)), self.handle)

    def tiles(self):
        v = [C.c_int32() for _ in range(6)]
        _check_batch(lib().apc_batch_get_tiles(self.handle, *[C.byref(x) for x in v]), self.handle)
        return tuple(x.value for x in v)

    def autotune(self, iters: int = 5, reps: int = 3, cache: str | None = None, stream=None):
        """Run the tile tuner (apc_batch_autotune) and store its choice in the
        tile cache under this batch's key; the iteration state must be reset
        afterwards.  Returns (tiles, ms per iteration tuned, ms default)."""
        out = (C.c_int32 * 6)()
        best, dflt = C.c_double(), C.c_double()
        with _device(self.device):
            _check_batch(lib().apc_batch_autotune(self.handle, int(iters), int(reps), out, C.byref(best),
                                                  C.byref(dflt), _stream(stream)), self.handle)
        tiles = tuple(int(x) for x in out)
        store_tiles(self.key, tiles, cache)
        return tiles, best.value, dflt.value

    def forward(self, T: int, B=None, stream=None):
        """Reset (with new right-hand sides B, one n_s x k tensor per system, or
        the stored ones), T iterations and every system's xbar(T), in one call
        (apc_batch_forward)."""
        import torch
        arr = None
        if B is not None:
            B = [_batch_rhs(b_, n_, self.k) for b_, n_ in zip(B, self.n)]
            arr = (C.c_void_p * len(B))(*[b_.data_ptr() for b_ in B])
            self._B = B
        outs = [torch.empty((n_, self.k), dtype=torch.float64, device=self.device) for n_ in self.n]
        oarr = (C.c_void_p * len(outs))(*[o.data_ptr() for o in outs])
        with _device(self.device):
            _check_batch(lib().apc_batch_forward(self.handle, arr, int(T), oarr, _stream(stream)), self.handle)
        return outs

    def backward(self, G, T: int, stream=None):
        """dL/dB_s for every system from G_s = dL/dxbar_s(T) (n_s x k each)
        through T iterations (apc_batch_backward)."""
        import torch
        G = [_batch_rhs(g_, n_, self.k) for g_, n_ in zip(G, self.n)]
        garr = (C.c_void_p * len(G))(*[g_.data_ptr() for g_ in G])
        outs = [torch.empty((n_, self.k), dtype=torch.float64, device=self.device) for n_ in self.n]
        oarr = (C.c_void_p * len(outs))(*[o.data_ptr() for o in outs])
        with _device(self.device):
            _check_batch(lib().apc_batch_backward(self.handle, garr, int(T), oarr, _stream(stream)), self.handle)
        return outs


def _device(dev):
    import torch
    return torch.cuda.device(dev)



def _batch_rhs(B, n, k):
    import torch
    if not B.is_cuda or B.dtype != torch.float64:
        raise TypeError("float64 CUDA tensors expected")
    B = B.reshape(n, k) if B.dim() == 1 else B
    if tuple(B.shape) != (n, k):
        raise ValueError(f"right-hand side of shape {tuple(B.shape)}, expected {(n, k)}")
    return B.contiguous()


TILE_CACHE = os.environ.get("APC_TILE_CACHE", os.path.join(HERE, "_build", "tile_cache.json"))


def tile_cache_key(ns, block_sizes, k, sms) -> str:
    """Key of the tile cache: histograms of the systems' sizes n and of the
    block sizes p (power-of-two buckets), the right-hand sides and the SM count."""
    import collections
    hn = collections.Counter(int(n).bit_length() for n in ns)
    hp = collections.Counter(int(p).bit_length() for p in block_sizes)
    fmt = lambda h: ",".join(f"{b}:{h[b]}" for b in sorted(h))  # noqa: E731
    return f"n[{fmt(hn)}]|p[{fmt(hp)}]|k{int(k)}|sm{int(sms)}"


def load_tiles(key, cache=None):
    import json
    path = cache or TILE_CACHE
    try:
        with open(path) as fh:
            v = json.load(fh).get(key)
        return tuple(int(x) for x in v) if v else None
    except (OSError, ValueError):
        return None


def store_tiles(key, tiles, cache=None):
    import json
    path = cache or TILE_CACHE
    try:
        with open(path) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        d = {}
    d[key] = [int(x) for x in tiles]
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(d, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def apc_batch_setup(As, Bs, row_offsets, timeout_s=0.0, stream=None, tiles="cache", cache=None) -> Batch:
    """Factor every system: As[s] an n_s x n_s FP64 CUDA tensor, Bs[s] its
    n_s x k right-hand sides (k equal for all systems, <= 32), row_offsets[s]
    its m_s + 1 block offsets.  ``tiles``: "cache" (the tuner's stored choice
    for this batch's key, else the default shape), "default", or a tuple
    (rows_a, cols_b, prefetch)."""
    import numpy as np
    import torch
    nsys = len(As)
    if nsys < 1 or len(Bs) != nsys or len(row_offsets) != nsys:
        raise ValueError("one A, one B and one offset list per system")
    ns = [int(A.shape[0]) for A in As]
    k = int(Bs[0].shape[1]) if Bs[0].dim() == 2 else 1
    for A in As:
        if not A.is_cuda or A.dtype != torch.float64 or A.dim() != 2 or A.shape[0] != A.shape[1]:
            raise TypeError("square float64 CUDA matrices expected")
    As = [A.contiguous() for A in As]
    Bs = [_batch_rhs(B, n_, k) for B, n_ in zip(Bs, ns)]
    offs = [np.asarray(o, dtype=np.int64) for o in row_offsets]
    n_arr = np.ascontiguousarray(np.asarray(ns, dtype=np.int64))
    m_arr = np.ascontiguousarray(np.asarray([len(o) - 1 for o in offs], dtype=np.int32))
    o_arr = np.ascontiguousarray(np.concatenate(offs))
    a_arr = (C.c_void_p * nsys)(*[A.data_ptr() for A in As])
    b_arr = (C.c_void_p * nsys)(*[B.data_ptr() for B in Bs])
    opt = apc_options(APC_BF16, 0, 0, float(timeout_s))
    h = C.c_void_p()
    with torch.cuda.device(As[0].device):
        rc = lib().apc_batch_setup(C.byref(h), nsys, n_arr.ctypes.data_as(C.POINTER(C.c_int64)),
                                   m_arr.ctypes.data_as(C.POINTER(C.c_int32)),
                                   o_arr.ctypes.data_as(C.POINTER(C.c_int64)), a_arr, b_arr, k, C.byref(opt),
                                   _stream(stream))
    _check_batch(rc, None)
    sms = torch.cuda.get_device_properties(As[0].device).multi_processor_count
    key = tile_cache_key(ns, [int(o[i + 1] - o[i]) for o in offs for i in range(len(o) - 1)], k, sms)
    bt = Batch(h, As[0].device, ns, k, Bs, key)
    chosen = load_tiles(key, cache) if tiles == "cache" else (None if tiles == "default" else tuple(tiles))
    if chosen:
        bt.set_tiles(*chosen)
    return bt
