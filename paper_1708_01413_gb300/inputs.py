"""Seeded synthetic inputs for the APC solver (test and benchmark workloads).

This module only draws random numbers and lays them out; it holds none of the
method's arithmetic.  Both the CPU oracle's tests and the GPU path consume the
arrays it returns.

Workload recipes (shapes and distributions of the paper's experiments, Sec. 5,
"Standard Gaussian" rows of Table 2, and the scaled / batched / differentiated
variants exercised by the solver):

* ``gaussian_system``  A n x n with i.i.d. N(0,1) entries, x_true ~ N(0,1),
  b = A x_true.
* ``scaled_system``    A = D_r G D_c, G i.i.d. N(0,1), D_r and D_c diagonal with
  entries log-uniform in [10^-lo, 10^hi]; optionally tall (N > n rows) and with
  D_c narrowed to [10^-c, 10^c] (row scaling leaves every block's row space,
  hence X, unchanged; column scaling sets kappa(X)).
* ``batch_systems``    independent systems with n ~ U{n_lo..n_hi},
  A = G + 0.5 sqrt(n) I, uneven row blocks p_i ~ U{p_lo..p_hi} (the last block
  truncated), k right-hand sides b ~ N(0,1).
* ``even_offsets``     m contiguous row blocks of N/m rows.
"""
from __future__ import annotations

import numpy as np

__all__ = ["gaussian_system", "scaled_system", "batch_systems", "even_offsets",
           "uneven_offsets", "target_vector", "gaussian_system_torch", "scaled_system_torch",
           "batch_specs", "batch_systems_torch"]


def even_offsets(N: int, m: int) -> np.ndarray:
    """Row offsets of m contiguous blocks; the first N % m blocks get one extra row."""
    base, extra = divmod(N, m)
    sizes = [base + (1 if i < extra else 0) for i in range(m)]
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


def uneven_offsets(N: int, p_lo: int, p_hi: int, rng: np.random.Generator) -> np.ndarray:
    """Row offsets with block sizes drawn uniformly from {p_lo..p_hi}; the
    last block is truncated at N."""
    offs = [0]
    while offs[-1] < N:
        offs.append(min(N, offs[-1] + int(rng.integers(p_lo, p_hi + 1))))
    return np.asarray(offs, dtype=np.int64)


def gaussian_system(n: int, seed: int, N: int | None = None, k: int = 1, mean: float = 0.0):
    """(A, x_true, b): A N x n i.i.d. N(mean, 1), x_true n (x k) ~ N(0,1), b = A x_true."""
    rng = np.random.default_rng(seed)
    N = n if N is None else N
    A = rng.standard_normal((N, n)) + mean
    x_true = rng.standard_normal((n,) if k == 1 else (n, k))
    return A, x_true, A @ x_true


def scaled_system(n: int, seed: int, lo: float = 2.0, hi: float = 2.0, N: int | None = None,
                  col_decades: float | None = None):
    """(A, x_true, b) with A = D_r G D_c (N x n, N = n by default), D entries
    log-uniform in [10^-lo, 10^hi]; ``col_decades`` = c narrows D_c to
    [10^-c, 10^c] (D_r keeps the full range)."""
    rng = np.random.default_rng(seed)
    N = n if N is None else N
    G = rng.standard_normal((N, n))
    d_r = 10.0 ** rng.uniform(-lo, hi, size=N)
    c_lo, c_hi = (lo, hi) if col_decades is None else (col_decades, col_decades)
    d_c = 10.0 ** rng.uniform(-c_lo, c_hi, size=n)
    A = (d_r[:, None] * G) * d_c[None, :]
    x_true = rng.standard_normal(n)
    return A, x_true, A @ x_true


def batch_systems(nsys: int, seed: int, n_lo: int = 256, n_hi: int = 4096,
                  p_lo: int = 16, p_hi: int = 128, k: int = 32):
    """List of (A, B, row_offsets) for ``nsys`` independent systems."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(nsys):
        n = int(rng.integers(n_lo, n_hi + 1))
        A = rng.standard_normal((n, n)) + 0.5 * np.sqrt(n) * np.eye(n)
        offs = uneven_offsets(n, p_lo, p_hi, rng)
        B = rng.standard_normal((n, k))
        out.append((A, B, offs))
    return out


def target_vector(n: int, seed: int, k: int = 1) -> np.ndarray:
    """x_target ~ N(0,1) for the differentiated loss 0.5 ||xbar_T - x_target||^2."""
    rng = np.random.default_rng(seed + 7919)
    return rng.standard_normal((n,) if k == 1 else (n, k))


# Device-side generators for the full-size workloads (a host draw of 10^9
# normals takes tens of seconds).  These use torch's own seeded generator on
# the given device; results differ from the NumPy streams above, so a test
# that compares against the oracle copies the device arrays back to the host.

def gaussian_system_torch(n: int, seed: int, device, dtype=None, N: int | None = None):
    """(A, x_true, b) on the device: A N x n (N = n by default) i.i.d. N(0,1),
    x_true ~ N(0,1), b = A x_true."""
    import torch
    dtype = torch.float64 if dtype is None else dtype
    N = n if N is None else N
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    A = torch.randn((N, n), generator=g, device=device, dtype=dtype)
    x_true = torch.randn((n,), generator=g, device=device, dtype=dtype)
    return A, x_true, A @ x_true


def scaled_system_torch(n: int, seed: int, device, lo: float = 2.0, hi: float = 2.0, N: int | None = None,
                        col_decades: float | None = None):
    """Device draw of ``scaled_system``'s family (same arguments; a different stream)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    N = n if N is None else N
    A = torch.randn((N, n), generator=g, device=device, dtype=torch.float64)
    d_r = 10.0 ** (torch.rand((N,), generator=g, device=device, dtype=torch.float64) * (lo + hi) - lo)
    c_lo, c_hi = (lo, hi) if col_decades is None else (col_decades, col_decades)
    d_c = 10.0 ** (torch.rand((n,), generator=g, device=device, dtype=torch.float64) * (c_lo + c_hi) - c_lo)
    A.mul_(d_r[:, None]).mul_(d_c[None, :])
    x_true = torch.randn((n,), generator=g, device=device, dtype=torch.float64)
    return A, x_true, A @ x_true


def batch_specs(nsys: int, seed: int, n_lo: int = 256, n_hi: int = 4096, p_lo: int = 16, p_hi: int = 128):
    """Sizes and row partitions of ``nsys`` independent systems: n ~ U{n_lo..n_hi},
    block sizes p_i ~ U{p_lo..p_hi} (the last block truncated).  Host-side draw,
    cheap at any size; the matrices come from ``batch_systems_torch``."""
    rng = np.random.default_rng(seed)
    specs = []
    for _ in range(nsys):
        n = int(rng.integers(n_lo, n_hi + 1))
        specs.append((n, uneven_offsets(n, p_lo, p_hi, rng)))
    return specs


def batch_systems_torch(specs, seed: int, device, k: int = 32):
    """(As, Bs, offsets) on the device for ``batch_specs``: A = G + 0.5 sqrt(n) I
    with G i.i.d. N(0,1), B n x k i.i.d. N(0,1), FP64."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    As, Bs, offs = [], [], []
    for n, o in specs:
        A = torch.randn((n, n), generator=g, device=device, dtype=torch.float64)
        A.diagonal().add_(0.5 * float(np.sqrt(n)))
        As.append(A)
        Bs.append(torch.randn((n, k), generator=g, device=device, dtype=torch.float64))
        offs.append(o)
    return As, Bs, offs
