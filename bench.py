"""Benchmark of the APC hot loop on one GB300.

Workload (headline metric): A = D_r G D_c, 32768 x 32768, G i.i.d. N(0,1),
D_r, D_c diagonal log-uniform in [1e-2, 1e2]; m = 128 contiguous row blocks of
256 rows; Q_i stored in BF16 (2 GiB), FP32 accumulation, FP64 setup.  One step
= `--iters-per-step` APC iterations of Eq. (cons) in one persistent launch.
`value` = APC iterations per second with everything resident in HBM.  Q
(2 GiB) is far larger than L2 (129 MB), so no flush is needed between steps.

Also on the same JSON line:
  e2e          the same metric through the C ABI with host buffers: per step an
               H2D copy of the right-hand side, the least-norm reset, the
               iterations and a D2H copy of xbar;
  roofline     of the iteration kernel (algorithmic bytes / launch time);
  fp32         the FP32 path on the same matrix;
  tts          time to relative residual 1e-10, BF16 + FP64 refinement against
               FP32 + FP64 refinement (and the floor of plain FP32), on a tall
               Gaussian system (2304 x 2048, 9 blocks of 256, kappa(X) ~ 1e3): the
               32768 scaled matrix has kappa(X) ~ 1e12 and needs far more
               iterations than a benchmark can run;
  small_f64    the paper-sized FP64 case (Gaussian 500 x 500, m = 10): microseconds per
               iteration (latency-bound: Q fits in L2) and the solve to 1e-10;
  tts_n32768   the same comparison at the headline size on a tall Gaussian
               system (36864 x 32768, 144 blocks of 256, kappa(X) ~ 1e3), with
               the spectrum estimated on the GPU (Lanczos);
  tts_dc<c>    the same on the headline's matrix family made tall (36864 x
               32768, D_r over 4 decades, D_c narrowed to 10^-c..10^c): the
               square matrix has kappa(X) >= 1e6 even at D_c = I;
  batch        the batched solver on 256 independent systems (n ~ U{256..4096},
               A = G + 0.5 sqrt(n) I, blocks p_i ~ U{16..128}, k = 32
               right-hand sides, BF16 bases): iterations per second of the
               whole batch and its roofline (HBM bytes and tensor-pipe work),
               and the preconditioned heavy-ball method (Sec. 6) on the same
               kernel;
  cpu_baseline the FP64 oracle timed on a bounded sample (8 of the 128 blocks).

`--impl reference` times the FP64 CPU oracle alone on the same workload (the
paper has no code; the oracle is the reference implementation of the method).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_FULL, M_FULL = 32768, 128
METRIC = "time to 1e-10 rel. residual & APC iter/s at n=32768: BF16+IR vs FP32, HBM %"
KERNEL_SOURCES = ("apc_iter_impl.cuh", "apc_iter.cu", "apc_iter_bf16.cu", "apc_iter_f32.cu", "apc_iter_f64.cu",
                  "apc_ptx.cuh", "apc_internal.h")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "apc_iter_kernel_traffic.md")
SAMPLE_BLOCKS = 8


def kernel_source_hash():
    """Hash of the iteration kernel's sources: a DRAM traffic figure measured
    with ncu is reported only while the kernel is unchanged."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1708_01413_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(workload_key):
    """DRAM bytes per iteration of the iteration kernel for `workload_key`, from
    the committed ncu summary; None if absent or taken on other sources."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    src, val = None, None
    for line in open(TRAFFIC_FILE):
        line = line.strip().strip("`")
        if line.startswith("source_hash:"):
            src = line.split(":", 1)[1].strip()
        if line.startswith(f"traffic_bytes_per_iteration[{workload_key}]:"):
            val = float(line.split(":", 1)[1].strip())
    return val if src == kernel_source_hash() else None


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            for k in ("hbm_gbs", "hbm_GBs", "hbm"):
                if k in d:
                    return float(d[k]), "measured"
        except Exception:
            pass
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except Exception:
                self.proc.kill()

    def summary(self):
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        rows = [r for r in self.rows if len(r) >= 9]
        sm = [v for v in (num(r[1]) for r in rows) if v is not None]
        mx = [v for v in (num(r[2]) for r in rows) if v is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({nm for r in rows for nm, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _dist():
    return int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0"))


def max_over_ranks(x, device=None):
    """The largest x over the ranks of the default process group, after a
    barrier (x itself without one): the job's time is its slowest rank's."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.barrier()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, max_ms):
    """Whole-job throughput of `world` replicas that each processed
    `units_per_rank` units, timed by the slowest rank (weak scaling)."""
    return units_per_rank * world / (max_ms / 1e3)


def _threads():
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS"):
        if os.environ.get(k):
            return int(os.environ[k])
    return os.cpu_count() or 1


# ---------------------------------------------------------------------------
# FP64 oracle on a bounded sample (cpu_baseline leg and --impl reference)
# ---------------------------------------------------------------------------

class OracleSample:
    """The FP64 oracle's iteration on SAMPLE_BLOCKS of the workload's row
    blocks; one step's time is scaled by m_total / SAMPLE_BLOCKS (the
    iteration's cost is linear in the number of blocks), so the figure is an
    extrapolation to the whole workload."""

    def __init__(self, A_rows, p, m_total):
        import numpy as np
        from oracle import apc_oracle as O
        self.O = O
        rows = A_rows.shape[0]
        offs = np.arange(0, rows + 1, p)
        blocks = O.partition(A_rows, np.zeros(rows), offs)
        self.Qs = [O.block_qr(Ai)[0] for Ai, _ in blocks]
        rng = np.random.default_rng(0)
        n = A_rows.shape[1]
        self.xs = [rng.standard_normal(n) for _ in self.Qs]
        self.xbar = sum(self.xs) / len(self.xs)
        self.scale = m_total / len(self.Qs)

    def step_seconds(self):
        t0 = time.perf_counter()
        self.xs, self.xbar = self.O.apc_step(self.xs, self.xbar, self.Qs, 1.0, 1.5)
        return (time.perf_counter() - t0) * self.scale

    def timed(self, steps, warmup=1):
        """Median extrapolated seconds per iteration over `steps` timed steps."""
        for _ in range(warmup):
            self.step_seconds()
        return statistics.median(self.step_seconds() for _ in range(steps))

    def describe(self, n, p, m):
        return (f"{len(self.Qs)} of {m} row blocks ({len(self.Qs) * p} x {n} FP64) of the workload, one Eq. (cons) "
                f"iteration per step, step time scaled x{self.scale:g} to all blocks (extrapolated)")


CPU_STEPS = 10


def single_core_rate(n, p, m):
    """The same oracle sample timed in a child process limited to one thread
    (BLAS and OpenMP), in iterations per second of the whole workload."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample-worker", "--n", str(n), "--m", str(m)],
                       capture_output=True, text=True, env=env, timeout=600)
    if r.returncode != 0:
        return None
    return float(r.stdout.strip().splitlines()[-1])


def cpu_baseline(A_rows, n, p, m):
    """cpu_baseline of the JSON line: the oracle on the bounded sample with all
    host cores and with one core."""
    sample = OracleSample(A_rows, p, m)
    sec = sample.timed(CPU_STEPS)
    try:
        single = single_core_rate(n, p, m)
    except Exception:
        single = None
    return {"value": 1.0 / sec, "unit": "iter/s", "cores": _threads(), "nproc": os.cpu_count(), "kind": "oracle",
            "single_core_value": single, "extrapolated": True, "steps": CPU_STEPS,
            "sample": sample.describe(n, p, m)}


def _sample_rows(n, p, seed):
    """The first SAMPLE_BLOCKS row blocks of the scaled system (host draw)."""
    import numpy as np
    rows = SAMPLE_BLOCKS * p
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((rows, n))
    d_r = 10.0 ** rng.uniform(-2, 2, size=rows)
    d_c = 10.0 ** rng.uniform(-2, 2, size=n)
    return (d_r[:, None] * G) * d_c[None, :]


def run_reference(args):
    world, rank = _dist()
    if rank != 0:
        return
    p = args.n // args.m
    sample = OracleSample(_sample_rows(args.n, p, 0), p, args.m)
    times = []
    for s in range(args.warmup + args.steps):
        t = sample.step_seconds()
        if s >= args.warmup:
            times.append(t)
    sec = statistics.mean(times)
    value = 1.0 / sec
    try:
        single = single_core_rate(args.n, p, args.m)
    except Exception:
        single = None
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "iter/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"APC n={args.n} A=D_r G D_c (log-uniform 1e-2..1e2), m={args.m} blocks of {p}"},
        "cpu_baseline": {"value": value, "unit": "iter/s", "cores": _threads(), "nproc": os.cpu_count(),
                         "kind": "oracle", "single_core_value": single, "extrapolated": True,
                         "sample": sample.describe(args.n, p, args.m)},
        "e2e": {"value": value, "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_cpu_sample_worker(args):
    """Child process of single_core_rate: print the sample's iterations/s."""
    p = args.n // args.m
    sample = OracleSample(_sample_rows(args.n, p, 0), p, args.m)
    print(1.0 / sample.timed(CPU_STEPS), flush=True)


# ---------------------------------------------------------------------------
# the CUDA path
# ---------------------------------------------------------------------------

def _ev():
    import torch
    return torch.cuda.Event(enable_timing=True)


def time_to_tolerance(dev, tol=1e-10):
    """Time to relative residual `tol`: BF16 + FP64 refinement against FP32 +
    FP64 refinement (and the floor of plain FP32), on a tall Gaussian system
    (N = 2304 equations, n = 2048 unknowns, 9 blocks of 256; kappa(X) ~ 1e3).
    (gamma*, eta*) from Theorem 1 with the extreme eigenvalues of
    X = (1/m) sum_i Q_i Q_i^T, from a host eigensolve of the GPU's FP64 bases."""
    import numpy as np
    import torch
    from paper_1708_01413_gb300 import apc, inputs
    n, N, m = 2048, 2304, 9
    A, x_true, b = inputs.gaussian_system(n, 11, N=N)
    offs = inputs.even_offsets(N, m)
    At, bt = torch.tensor(A, device=dev), torch.tensor(b, device=dev)
    ctx64 = apc.apc_setup(At, bt, offs, precision="f64")
    X = sum(q @ q.T for q in (ctx64.basis(i).cpu().numpy() for i in range(m))) / m
    ctx64.close()
    mu = np.linalg.eigvalsh(X)
    g, e, rho = apc.apc_optimal_params(float(mu[0]), float(mu[-1]))
    out = {"workload": f"tall Gaussian N={N}, n={n}, m={m} blocks of {N // m}", "kappa_X": float(mu[-1] / mu[0]),
           "gamma": g, "eta": e, "rho": rho, "tol": tol}
    runs = (("bf16_ir", "bf16", True), ("f32_ir", "f32", True), ("f32_plain", "f32", False))
    for key, prec, refine in runs:
        ctx = apc.apc_setup(At, bt, offs, precision=prec)
        ctx.solve(g, e, tol=tol, max_iters=200, check_every=50, refine=refine, raise_on_error=False)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x, st = ctx.solve(g, e, tol=tol, max_iters=20000, check_every=50, refine=refine, raise_on_error=False)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        xh = x.cpu().numpy()
        out[key] = {"seconds": dt, "iterations": st["iterations"], "sweeps": st["sweeps"],
                    "rel_residual": st["rel_residual"],
                    "rel_error": float(np.linalg.norm(xh - x_true) / np.linalg.norm(x_true)),
                    "converged": st["rc"] == 0}
        ctx.close()
    return out


def time_to_tolerance_large(dev, tol=1e-10, n=32768, N=36864, p=256, col_decades=None, max_iters=5000,
                            plain=True, lanczos_steps=150, lo_margin=0.98):
    """Time to relative residual `tol` at the headline size: a tall Gaussian
    system (N = 36864 equations, n = 32768 unknowns, 144 blocks of 256; kappa(X)
    stays ~1e3 at any size for this aspect ratio), BF16 + FP64 refinement
    against FP32 + FP64 refinement, plus the residual plain FP32 reaches in a
    bounded run.  With `col_decades` = c the matrix is the headline's family
    instead, tall: A = D_r G D_c, D_r log-uniform in [1e-2, 1e2], D_c narrowed to
    [10^-c, 10^c] (the square matrix has kappa(X) >= 1e6 even at D_c = I).
    Each context estimates the extreme eigenvalues of its own X with the GPU
    Lanczos (apc_spectral_bounds), margins 0.98 / 1.01, then Theorem 1's
    (gamma, eta).  `seconds` covers the solve alone; set-up and Lanczos are
    reported beside it, and `total_s` is the user-visible time to the
    tolerance: set-up + Lanczos + solve.  FP32 checks its inner solves with the
    free residual monitor, BF16 with FP64 residuals (counts beside)."""
    import torch
    from paper_1708_01413_gb300 import apc, inputs
    m = N // p
    if col_decades is None:
        A, x_true, b = inputs.gaussian_system_torch(n, 13, dev, N=N)
        workload = f"tall Gaussian N={N}, n={n}, m={m} blocks of {p}"
    else:
        A, x_true, b = inputs.scaled_system_torch(n, 17, dev, N=N, col_decades=col_decades)
        workload = (f"tall A=D_r G D_c N={N}, n={n}, D_r log-uniform 1e-2..1e2, D_c log-uniform "
                    f"1e-{col_decades:g}..1e{col_decades:g}, m={m} blocks of {p}")
    offs = inputs.even_offsets(N, m)
    out = {"workload": workload, "tol": tol}
    runs = [("bf16_ir", "bf16", True, max_iters), ("f32_ir", "f32", True, max_iters)]
    if plain:
        runs.append(("f32_plain", "f32", False, 2000))
    for key, prec, refine, max_iters in runs:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx = apc.apc_setup(A, b, offs, precision=prec)
        torch.cuda.synchronize()
        t_setup = time.perf_counter() - t0
        try:
            t0 = time.perf_counter()
            lo, hi = ctx.spectral_bounds(steps=lanczos_steps)
            t_lanczos = time.perf_counter() - t0
            g, e, rho = apc.apc_optimal_params(lo_margin * lo, min(1.0, 1.01 * hi))
            ctx.solve(g, e, tol=tol, max_iters=100, check_every=50, refine=refine, raise_on_error=False)  # warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            x, st = ctx.solve(g, e, tol=tol, max_iters=max_iters, check_every=50, refine=refine,
                              raise_on_error=False)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            out[key] = {"seconds": dt, "iterations": st["iterations"], "sweeps": st["sweeps"],
                        "rel_residual": st["rel_residual"],
                        "rel_error": float(torch.linalg.norm(x - x_true) / torch.linalg.norm(x_true)),
                        "converged": st["rc"] == 0, "mu_bounds": [lo, hi], "kappa_X": hi / lo, "rho": rho,
                        "setup_s": round(t_setup, 3), "lanczos_s": round(t_lanczos, 3),
                        "total_s": round(t_setup + t_lanczos + dt, 3),
                        "residual_checks": st["residual_checks"], "monitor_checks": st["monitor_checks"]}
        finally:
            ctx.close()
    del A, b
    torch.cuda.empty_cache()
    return out


def time_small_f64(dev, tol=1e-10):
    """The paper-sized FP64 case: Gaussian 500 x 500, m = 10 blocks of 50, (gamma*, eta*) from
    Theorem 1 with the host eigenvalues of X; Q (2 MB) sits in L2, so an iteration is bound by
    the grid barrier and the pipeline's latency, not by HBM.  Microseconds per iteration (CUDA
    events over 5000 iterations in one launch) and the solve to relative residual `tol`."""
    import numpy as np
    import torch
    from paper_1708_01413_gb300 import apc, inputs
    n, m = 500, 10
    A, x_true, b = inputs.gaussian_system(n, 0)
    offs = inputs.even_offsets(n, m)
    ctx = apc.apc_setup(torch.tensor(A, device=dev), torch.tensor(b, device=dev), offs, precision="f64")
    try:
        X = sum(q @ q.T for q in (ctx.basis(i).cpu().numpy() for i in range(m))) / m
        mu = np.linalg.eigvalsh(X)
        g, e, rho = apc.apc_optimal_params(float(mu[0]), float(mu[-1]))
        ctx.reset()
        ctx.iterate(g, e, 200)
        torch.cuda.synchronize()
        e0, e1 = _ev(), _ev()
        T = 5000
        e0.record()
        ctx.iterate(g, e, T)
        e1.record()
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) * 1e3 / T
        ctx.solve(g, e, tol=tol, max_iters=1000, check_every=1000, raise_on_error=False)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x, st = ctx.solve(g, e, tol=tol, max_iters=500000, check_every=2000, raise_on_error=False)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        info = ctx.info()
        return {"workload": f"Gaussian {n} x {n}, m = {m} blocks of {n // m}, FP64", "kappa_X": float(mu[-1] / mu[0]),
                "gamma": g, "eta": e, "rho": rho, "us_per_iter": us, "clusters": info["clusters"],
                "solve": {"tol": tol, "seconds": dt, "iterations": st["iterations"],
                          "rel_residual": st["rel_residual"],
                          "rel_error": float(np.linalg.norm(x.cpu().numpy() - x_true) / np.linalg.norm(x_true)),
                          "converged": st["rc"] == 0}}
    finally:
        ctx.close()


def time_fp32(A, b, offs, gamma, eta, T, peak, stream):
    """The FP32 path (Q in FP32) on the same matrix: iterations/s and HBM GB/s."""
    import torch
    from paper_1708_01413_gb300 import apc
    n, m = A.shape[1], len(offs) - 1
    c32 = apc.apc_setup(A, b, offs, precision="f32")
    try:
        c32.reset()
        c32.iterate(gamma, eta, T)
        torch.cuda.synchronize()
        a0, a1 = _ev(), _ev()
        a0.record(stream)
        for _ in range(3):
            c32.iterate(gamma, eta, T)
        a1.record(stream)
        torch.cuda.synchronize()
        s32 = a0.elapsed_time(a1) / 1e3
        b32 = c32.info()["q_bytes"] + 2 * m * n * 4 + 2 * n * 8
        gbs = b32 * 3 * T / s32 / 1e9
        info = c32.info()
        tpi = measured_traffic(f"n={n},m={m},f32")
        return {"iter_per_s": 3 * T / s32, "hbm_gbs": gbs, "frac": gbs / peak,
                "cluster_size": info["cluster_size"], "rows_per_group": info["rows_per_group"],
                "algorithmic_bytes_per_iter": b32, "traffic_bytes_per_iter": tpi}
    finally:
        c32.close()


def time_batch(dev, peak, stream, iters=50, reps=3, nsys=256, k=32, clocks=None, tiles="tune"):
    """The batched solver (one persistent launch of `iters` iterations per
    step) on the 256-system workload.  Algorithmic bytes per iteration: the
    packed BF16 bases read twice (one product each), the machines' iterates
    and the master's estimate read and written once (heavy ball: estimate and
    momentum, no machines' iterates)."""
    import numpy as np
    import torch
    from paper_1708_01413_gb300 import apc, inputs
    specs = inputs.batch_specs(nsys, seed=2024)
    As, Bs, offs = inputs.batch_systems_torch(specs, seed=2024, device=dev, k=k)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    bt = apc.apc_batch_setup(As, Bs, offs)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    del As, Bs
    torch.cuda.empty_cache()
    info = bt.info()
    bt.set_params([1.0] * nsys, [1.0] * nsys)  # in S for every system; the cost does not depend on them
    bt.reset()
    if tiles == "tune":
        tiles, ms_tuned, ms_default = bt.autotune(iters=5, reps=2)  # the project's tile tuner (cached per key)
    else:  # given tiles (profiling): rows_a,cols_b,prefetch,l2,split_a,split_b
        tiles = tuple(int(v) for v in tiles.split(","))
        bt.set_tiles(*tiles)
        ms_tuned = ms_default = None
    bt.reset()
    bt.iterate(iters)
    torch.cuda.synchronize()
    ev = [(_ev(), _ev()) for _ in range(reps)]
    with (clocks if clocks is not None else ClockSampler(torch.cuda.current_device())) as clk:
        for a, b_ in ev:
            a.record(stream)
            bt.iterate(iters)
            b_.record(stream)
        torch.cuda.synchronize()
    sec = statistics.mean(a.elapsed_time(b_) for a, b_ in ev) / 1e3 / iters
    # the preconditioned heavy-ball method (Sec. 6) on the same kernel: no
    # machines' iterates, so its bytes per iteration are the two reads of Q
    bt.set_hb_params([0.5] * nsys, [0.5] * nsys)
    bt.reset()
    bt.iterate(iters)
    torch.cuda.synchronize()
    hb0, hb1 = _ev(), _ev()
    hb0.record(stream)
    for _ in range(reps):
        bt.iterate(iters)
    hb1.record(stream)
    torch.cuda.synchronize()
    sec_hb = hb0.elapsed_time(hb1) / 1e3 / (reps * iters)
    # algorithmic bytes without the kernel's padding (rows to 32, each block's
    # columns to 16, right-hand sides to kp): Q_s is n_s x n_s BF16 (the blocks
    # of a square system hold n_s rows in all), x_i is n_s x k FP32 per machine,
    # the master's estimate n_s x k double-float (8 bytes); each read and
    # written once per iteration (heavy ball: estimate and momentum, no x_i)
    ns = np.array([n for n, _ in specs], dtype=np.float64)
    ms = np.array([len(o) - 1 for _, o in specs], dtype=np.float64)
    q_alg = float((ns ** 2).sum()) * 2
    x_alg = float((ms * ns).sum()) * k * 4
    xb_alg = float(ns.sum()) * k * 8
    alg = 2 * q_alg + 2 * x_alg + 2 * xb_alg
    alg_hb = 2 * q_alg + 4 * xb_alg
    padded = 2 * info["q_bytes"] + 2 * info["state_bytes"]
    kp = 16 if k <= 16 else 32
    cq = info["q_bytes"] / 2.0  # sum over systems of npad * Cq
    mma_flops = 2.0 * cq * kp * (2 + 3)  # both products, operands in 2 + 3 BF16 planes
    bt.close()
    achieved = alg / sec / 1e9
    return {"workload": f"{nsys} systems, n ~ U{{256..4096}} (sum n^2 = {float((ns ** 2).sum()):.3g}), "
                        f"A = G + 0.5 sqrt(n) I, blocks p_i ~ U{{16..128}}, k = {k}, BF16 bases",
            "iter_per_s": 1.0 / sec, "ms_per_iter": sec * 1e3, "rhs_iter_per_s": nsys * k / sec,
            "iters_per_launch": iters, "launches": reps, "setup_s": round(setup_s, 3), "grid": info["grid"],
            "tiles": {"rows_a": tiles[0], "cols_b": tiles[1], "prefetch": tiles[2], "l2_policy": tiles[3],
                      "split_a": tiles[4], "split_b": tiles[5],
                      "tuner_ms_per_iter": ms_tuned, "default_ms_per_iter": ms_default},
            "clocks": clk.summary(),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "algorithmic_bytes_per_iter": alg, "traffic_model_padded_bytes_per_iter": padded,
                         "kernel": "apc_batch_kernel", "tensor_tflops": mma_flops / sec / 1e12},
            "heavy_ball": {"ms_per_iter": sec_hb * 1e3, "iter_per_s": 1.0 / sec_hb,
                           "achieved_gbs": alg_hb / sec_hb / 1e9,
                           "frac": alg_hb / sec_hb / 1e9 / peak,
                           "algorithmic_bytes_per_iter": alg_hb}}


def time_rhs(dev, peak, stream, n=8192, m=32, k=16, T=200, reps=3, tune=True):
    """The differentiation workload: A n x n Gaussian, m blocks, k right-hand
    sides, T iterations forward (xbar(T) for all k columns) and the reverse
    sweep back to dL/dB, each one call (apc_forward_rhs / apc_backward_rhs).
    BF16 context: the k columns together on the tensor cores (App. A form);
    FP32 context: column after column through the iteration kernel.
    Algorithmic bytes per tensor-core iteration: the packed BF16 basis read
    twice (one product each, n x n x 2 bytes unpadded) plus the machines'
    iterates read and written (forward only: m n k x 4 bytes twice) and the
    master's estimate read and written (double-float, 16 n k bytes); the
    reverse sweep has no per-machine state (every machine's adjoint is one
    shared vector), only its n x k row state (double-float ell and lbar, read
    and written: 32 n k bytes)."""
    import torch
    from paper_1708_01413_gb300 import apc, inputs
    A, _, _ = inputs.gaussian_system_torch(n, 77, dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(78)
    B = torch.randn((n, k), generator=gen, device=dev, dtype=torch.float64)
    G = torch.randn((n, k), generator=gen, device=dev, dtype=torch.float64)
    offs = inputs.even_offsets(n, m)
    gam, eta = 1.0, 1.5
    out = {"workload": f"Gaussian {n} x {n}, m = {m} blocks of {n // m}, k = {k}, T = {T}"}
    if tune:
        # the tile tuner on the same single system (one-system batch, k columns)
        bt = apc.apc_batch_setup([A], [B], [offs])
        bt.set_params([gam], [eta])
        bt.reset()
        tiles, ms_tuned, ms_default = bt.autotune(iters=20, reps=2)
        out["tuner"] = {"tiles": list(tiles), "ms_per_iter": ms_tuned, "default_256_512_ms_per_iter": ms_default}
        bt.close()
    for prec in ("bf16", "f32"):
        ctx = apc.apc_setup(A, B[:, 0].contiguous(), offs, precision=prec)
        try:
            X = ctx.forward_rhs(B, T, gam, eta)  # warm-up (builds the tensor-core batch on BF16)
            ctx.backward_rhs(G, T, gam, eta)
            torch.cuda.synchronize()
            f0, f1, b1 = _ev(), _ev(), _ev()
            with ClockSampler(torch.cuda.current_device()) as clk:
                f0.record(stream)
                for _ in range(reps):
                    ctx.forward_rhs(B, T, gam, eta, out=X)
                f1.record(stream)
                for _ in range(reps):
                    ctx.backward_rhs(G, T, gam, eta)
                b1.record(stream)
                torch.cuda.synchronize()
            fwd = f0.elapsed_time(f1) / reps / 1e3
            bwd = f1.elapsed_time(b1) / reps / 1e3
            r = {"forward_ms": fwd * 1e3, "backward_ms": bwd * 1e3, "total_ms": (fwd + bwd) * 1e3,
                 "clocks": clk.summary()}
            if prec == "bf16":
                q = 2.0 * n * n
                fb, bb = 2 * q + 2 * m * n * k * 4 + 16 * n * k, 2 * q + 32 * n * k
                r.update({"path": "tensor cores (tcgen05), k columns together",
                          "forward_gbs": fb * T / fwd / 1e9, "forward_frac": fb * T / fwd / 1e9 / peak,
                          "backward_gbs": bb * T / bwd / 1e9, "backward_frac": bb * T / bwd / 1e9 / peak,
                          "bytes_per_iter_forward": fb, "bytes_per_step_backward": bb,
                          "q_reads_per_iter": 2})
            else:
                r.update({"path": "iteration kernel, one column after another",
                          "q_reads_per_iter": k})
            out[prec] = r
        finally:
            ctx.close()
    del A
    torch.cuda.empty_cache()
    return out


def summarize(extra):
    """The headline figures of the comparison legs in a few keys."""
    out = {}

    def get(d, *path):
        for k in path:
            if not isinstance(d, dict) or k not in d:
                return None
            d = d[k]
        return float(f"{d:.4g}") if isinstance(d, float) else d

    if "fp32" in extra:
        out["fp32_iter_per_s"] = get(extra, "fp32", "iter_per_s")
        out["fp32_hbm_frac"] = get(extra, "fp32", "frac")
    t = extra.get("tts_n32768", {})
    for key in ("bf16_ir", "f32_ir"):
        if key in t:
            out[f"tts_n32768_{key}_solve_s"] = get(t, key, "seconds")
            out[f"tts_n32768_{key}_total_s"] = get(t, key, "total_s")
            out[f"tts_n32768_{key}_rel_residual"] = get(t, key, "rel_residual")
    for key in sorted(k for k in extra if k.startswith("tts_dc")):
        for run in ("bf16_ir", "f32_ir"):
            out[f"{key}_{run}_total_s"] = get(extra, key, run, "total_s")
            out[f"{key}_{run}_converged"] = get(extra, key, run, "converged")
    if "batch" in extra:
        out["batch_ms_per_iter"] = get(extra, "batch", "ms_per_iter")
        out["batch_hbm_frac"] = get(extra, "batch", "roofline", "frac")
        out["batch_tiles"] = get(extra, "batch", "tiles")
    if "rhs" in extra:
        out["rhs_bf16_forward_ms"] = get(extra, "rhs", "bf16", "forward_ms")
        out["rhs_bf16_backward_ms"] = get(extra, "rhs", "bf16", "backward_ms")
        out["rhs_bf16_hbm_frac"] = get(extra, "rhs", "bf16", "forward_frac")
        out["rhs_f32_total_ms"] = get(extra, "rhs", "f32", "total_ms")
    if "small_f64" in extra:
        out["small_f64_us_per_iter"] = get(extra, "small_f64", "us_per_iter")
    return out


def run_ours(args):
    import numpy as np
    import torch
    from paper_1708_01413_gb300 import apc, inputs

    world, rank = _dist()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    n, m = args.n, args.m
    p = n // m
    A, x_true, b = inputs.scaled_system_torch(n, 1234 + rank, dev)
    offs = inputs.even_offsets(n, m)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx = apc.apc_setup(A, b, offs, precision=args.precision, cluster_size=args.cluster_size)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    info = ctx.info()
    gamma, eta = 1.0, 1.5  # any (gamma, eta) in S: the time per iteration does not depend on them
    T = args.iters_per_step
    stream = torch.cuda.current_stream()
    ctx.reset()
    for _ in range(args.warmup):
        ctx.iterate(gamma, eta, T)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ev = [(_ev(), _ev()) for _ in range(args.steps)]
    with ClockSampler(torch.cuda.current_device()) as clk:
        torch.cuda.synchronize()
        t_start, t_end = _ev(), _ev()
        t_start.record(stream)
        for s in range(args.steps):
            ev[s][0].record(stream)
            ctx.iterate(gamma, eta, T)
            ev[s][1].record(stream)
        t_end.record(stream)
        torch.cuda.synchronize()
    total_ms = max_over_ranks(t_start.elapsed_time(t_end), dev)
    value = job_rate(args.steps * T, world, total_ms)

    # roofline of the iteration kernel: algorithmic bytes per launch / launch time.
    # Per iteration: Q once, x_i read + written (FP32 or FP64), xbar read + written.
    q_bytes = info["q_bytes"]
    s_bytes = 8 if args.precision == "f64" else 4
    bytes_per_iter = q_bytes + 2 * m * n * s_bytes + 2 * n * 8
    launch_s = statistics.mean(a.elapsed_time(bb) for a, bb in ev) / 1e3
    achieved = bytes_per_iter * T / launch_s / 1e9
    peak, peak_kind = hbm_peak()
    tpi = measured_traffic(f"n={n},m={m},{args.precision}")

    e2e = None
    if args.e2e:
        b_host = b.cpu().pin_memory()
        x_host = torch.empty(n, dtype=torch.float64).pin_memory()
        b_dev = torch.empty_like(b)
        x_dev = torch.empty(n, dtype=torch.float64, device=dev)
        k = max(2, min(args.steps, 5))
        torch.cuda.synchronize()
        e0, e1 = _ev(), _ev()
        e0.record(stream)
        for _ in range(k):
            b_dev.copy_(b_host, non_blocking=True)
            ctx.reset(b_dev)
            ctx.iterate(gamma, eta, T)
            ctx.xbar(out=x_dev)
            x_host.copy_(x_dev, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e = {"value": k * T / (e0.elapsed_time(e1) / 1e3), "unit": "iter/s", "h2d_bytes_per_step": n * 8,
               "d2h_bytes_per_step": n * 8}

    extra = {}
    if args.fp32 and rank == 0 and args.precision != "f32":
        ctx.close()
        try:
            extra["fp32"] = time_fp32(A, b, offs, gamma, eta, T, peak, stream)
        except Exception as exc:  # a failed comparison must not lose the headline number
            extra["fp32"] = {"error": str(exc)}
    if args.batch and rank == 0:
        try:
            extra["batch"] = time_batch(dev, peak, stream)
        except Exception as exc:
            extra["batch"] = {"error": str(exc)}
    if args.rhs and rank == 0:
        try:
            extra["rhs"] = time_rhs(dev, peak, stream)
        except Exception as exc:
            extra["rhs"] = {"error": str(exc)}
    if args.tts and rank == 0:
        try:
            extra["tts"] = time_to_tolerance(dev)
        except Exception as exc:
            extra["tts"] = {"error": str(exc)}
        try:
            extra["tts_n32768"] = time_to_tolerance_large(dev)
        except Exception as exc:
            extra["tts_n32768"] = {"error": str(exc)}
        for c in args.tts_dc:
            key = f"tts_dc{c:g}"
            # With D_c over 10^-1..10^1 the spectrum of X is dense near mu_min
            # (kappa(X) ~ 2.6e5) and 150 Lanczos steps overestimate mu_min
            # tenfold: more steps and a wider margin below the smallest Ritz value.
            steps, margin = (150, 0.98) if c <= 0.5 else (800, 0.5)
            try:
                extra[key] = time_to_tolerance_large(dev, col_decades=c, max_iters=30000, plain=False,
                                                     lanczos_steps=steps, lo_margin=margin)
                extra[key]["lanczos_steps"], extra[key]["lo_margin"] = steps, margin
            except Exception as exc:
                extra[key] = {"error": str(exc)}
        try:
            extra["small_f64"] = time_small_f64(dev)
        except Exception as exc:
            extra["small_f64"] = {"error": str(exc)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        A_s = A[:SAMPLE_BLOCKS * p].cpu().numpy()
        del A
        cpu = cpu_baseline(A_s, n, p, m)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "iter/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": f"APC n={n} A=D_r G D_c (log-uniform 1e-2..1e2), m={m} blocks of {p}, "
                                   f"Q {args.precision}, FP32 accumulation",
                       "iters_per_step": T, "l2": f"Q {q_bytes / 2**30:.2f} GiB > L2 129 MB, no flush",
                       "cluster_size": info["cluster_size"], "clusters": info["clusters"],
                       "setup_s": round(setup_s, 3)},
            "e2e": e2e,
            "gpu_launches": args.steps * ((T + (1 << 20) - 1) >> 20),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": (tpi * T if tpi is not None else None),
                         "peak_kind": peak_kind, "kernel": "apc_iter_kernel (MODE_APC)",
                         "algorithmic_bytes_per_launch": bytes_per_iter * T, "source_hash": kernel_source_hash()},
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
        }
        line.update(extra)
        line["summary"] = summarize(extra)  # last, so that a truncated tail of the line keeps it
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_batch_only(args):
    """`--only batch`: the batched workload alone, one JSON line."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    peak, peak_kind = hbm_peak()
    r = time_batch(dev, peak, torch.cuda.current_stream(), iters=args.batch_iters, reps=args.steps,
                   nsys=args.batch_systems, tiles=args.batch_tiles)
    r["roofline"]["peak_kind"] = peak_kind
    line = {"metric": "APC iterations/s of the whole batch (all systems, all right-hand sides)",
            "value": r["iter_per_s"], "unit": "iter/s", "n_gpus": 1, "steps": args.steps, "warmup": 1,
            "ms_per_step": r["ms_per_iter"] * args.batch_iters, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": r["workload"], "iters_per_step": args.batch_iters,
                       "l2": "bases and iterates >> L2 129 MB, no flush"},
            "gpu_launches": args.steps, "roofline": r["roofline"], "clocks": r["clocks"], "batch": r}
    print(json.dumps(line), flush=True)


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=N_FULL)
    p.add_argument("--m", type=int, default=M_FULL)
    p.add_argument("--precision", default="bf16", choices=["bf16", "f32", "f64"])
    p.add_argument("--iters-per-step", type=int, default=100)
    p.add_argument("--cluster-size", type=int, default=0)
    p.add_argument("--fp32", type=int, default=1, help="also time the FP32 path on the same matrix")
    p.add_argument("--tts", type=int, default=1, help="also measure time to 1e-10 (BF16+IR vs FP32+IR)")
    p.add_argument("--tts-dc", type=lambda v: [float(c) for c in v.split(",") if c], default=[0.5, 1.0],
                   help="D_c ranges (decades, comma-separated) of the tall scaled time-to-tolerance legs")
    p.add_argument("--e2e", type=int, default=1)
    p.add_argument("--batch", type=int, default=1, help="also time the batched solver (256 systems, k = 32)")
    p.add_argument("--rhs", type=int, default=1, help="also time the differentiation workload (k = 16, T = 200)")
    p.add_argument("--only", default="all", choices=["all", "batch", "rhs"],
                   help="batch / rhs: time only the batched workload / the differentiation workload (for profiling)")
    p.add_argument("--rhs-T", type=int, default=200, help="iterations of the differentiation workload")
    p.add_argument("--batch-systems", type=int, default=256)
    p.add_argument("--batch-iters", type=int, default=50)
    p.add_argument("--batch-tiles", default="tune",
                   help="'tune' (the tile tuner) or rows_a,cols_b,prefetch,l2,split_a,split_b (profiling)")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--cpu-sample-worker", action="store_true", help=argparse.SUPPRESS)
    args = p.parse_args()
    if args.cpu_sample_worker:
        run_cpu_sample_worker(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        from paper_1708_01413_gb300 import build
        build.build()
        if args.only == "batch":
            run_batch_only(args)
        elif args.only == "rhs":
            import torch
            dev = torch.device("cuda", torch.cuda.current_device())
            peak, _ = hbm_peak()
            r = time_rhs(dev, peak, torch.cuda.current_stream(), T=args.rhs_T, reps=args.steps, tune=False)
            print(json.dumps({"metric": "differentiation workload: forward + reverse sweep", "rhs": r}), flush=True)
        else:
            run_ours(args)


if __name__ == "__main__":
    main()
