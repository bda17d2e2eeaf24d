"""Benchmark of the APC hot loop on one GB300.

Workload: the precision configuration of the solver's headline metric:
A = D_r G D_c (32768 x 32768, G i.i.d. N(0,1), D log-uniform in [1e-2, 1e2]),
m = 128 contiguous row blocks of 256 rows, Q_i stored in BF16 (2 GiB), FP32
accumulation, FP64 setup.  One step = `--iters-per-step` APC iterations of
Eq. (cons) in one persistent launch; `value` is APC iterations per second with
everything resident in HBM.  Q (2 GiB) is far larger than L2 (129 MB), so no
flush is needed between steps.

Also reported on the same line: the FP32 path on the same matrix, the setup
time, `e2e` (the same metric through the C ABI with host buffers: H2D of the
right-hand side, least-norm reset, the iterations, D2H of xbar), the roofline
of the iteration kernel, and the FP64 CPU oracle timed on a bounded sample.

`--impl reference` times the FP64 CPU oracle alone (the paper has no code; the
oracle is the reference implementation of the method).
"""
from __future__ import annotations

import argparse
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


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            return float(d.get("hbm_gbs", 6800.0)), "measured"
        except Exception:
            pass
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
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
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) >= 9:
                for nm, v in zip(names, r[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return world, rank


def oracle_sample(A_rows_host, offs_sample, m_total, iters, warm=1):
    """Time the FP64 oracle's iteration on a sample of the row blocks.

    Returns seconds per full-workload iteration (sample time scaled by
    m_total / m_sample) and the thread count numpy used."""
    import numpy as np
    from oracle import apc_oracle as O
    m_s = len(offs_sample) - 1
    b = np.zeros(A_rows_host.shape[0])
    blocks = O.partition(A_rows_host, b, offs_sample)
    Qs = [O.block_qr(Ai)[0] for Ai, _ in blocks]
    n = A_rows_host.shape[1]
    rng = np.random.default_rng(0)
    xs = [rng.standard_normal(n) for _ in range(m_s)]
    xbar = sum(xs) / m_s
    for _ in range(warm):
        xs, xbar = O.apc_step(xs, xbar, Qs, 1.0, 1.5)
    t0 = time.perf_counter()
    for _ in range(iters):
        xs, xbar = O.apc_step(xs, xbar, Qs, 1.0, 1.5)
    dt = (time.perf_counter() - t0) / iters
    return dt * (m_total / m_s)


def _threads():
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS"):
        if os.environ.get(k):
            return int(os.environ[k])
    return os.cpu_count() or 1


def run_reference(args):
    world, rank = _dist()
    if rank != 0:
        return
    import numpy as np
    from paper_1708_01413_gb300 import inputs
    rows = 8 * 256
    A, _, _ = inputs.scaled_system(256, 0)  # warm numpy
    rng = np.random.default_rng(0)
    G = rng.standard_normal((rows, N_FULL))
    d_r = 10.0 ** rng.uniform(-2, 2, size=rows)
    d_c = 10.0 ** rng.uniform(-2, 2, size=N_FULL)
    A_s = (d_r[:, None] * G) * d_c[None, :]
    offs = np.arange(0, rows + 1, 256)
    times = []
    for s in range(args.warmup + args.steps):
        t = oracle_sample(A_s, offs, M_FULL, iters=1, warm=0)
        if s >= args.warmup:
            times.append(t)
    sec = statistics.mean(times)
    value = 1.0 / sec
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "iter/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "APC n=32768 D_r G D_c, m=128 blocks of 256, FP64 CPU oracle sample"},
        "cpu_baseline": {"value": value, "unit": "iter/s", "cores": _threads(), "kind": "oracle",
                         "sample": "8 of 128 row blocks (2048 x 32768 FP64), one Eq. (cons) iteration per step, "
                                   "time scaled x16 to all blocks"},
        "e2e": {"value": value, "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch
    from paper_1708_01413_gb300 import apc, inputs

    world, rank = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        local = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(local)
    dev = torch.device("cuda", torch.cuda.current_device())
    n, m = args.n, args.m
    A, x_true, b = inputs.scaled_system_torch(n, 1234 + rank, dev)
    offs = inputs.even_offsets(n, m)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx = apc.apc_setup(A, b, offs, precision=args.precision, cluster_size=args.cluster_size)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    info = ctx.info()
    gamma, eta = 1.0, 1.5  # any (gamma, eta) in S; the throughput does not depend on them
    ctx.reset()
    T = args.iters_per_step
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        ctx.iterate(gamma, eta, T)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(torch.cuda.current_device()) as clk:
        torch.cuda.synchronize()
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for s in range(args.steps):
            ev[s][0].record(stream)
            ctx.iterate(gamma, eta, T)
            ev[s][1].record(stream)
        t_end.record(stream)
        torch.cuda.synchronize()
    total_ms = t_start.elapsed_time(t_end)
    if world > 1:
        tt = torch.tensor([total_ms], device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(tt.item())
    launch_ms = [a.elapsed_time(bb) for a, bb in ev]
    iters = args.steps * T
    value = iters * world / (total_ms / 1e3)
    ms_per_step = total_ms / args.steps

    # roofline of the iteration kernel: algorithmic bytes per launch / launch time
    q_bytes = info["q_bytes"]
    state_bytes = 2 * m * n * 4 + 2 * n * 8  # x_i read + write, xbar read + write
    bytes_per_iter = q_bytes + state_bytes
    avg_launch_s = statistics.mean(launch_ms) / 1e3
    achieved = bytes_per_iter * T / avg_launch_s / 1e9
    peak, peak_kind = _peaks()

    # e2e through the C ABI with host buffers: H2D rhs, reset, T iterations, D2H xbar
    b_host = b.cpu().pin_memory()
    x_host = torch.empty(n, dtype=torch.float64).pin_memory()
    b_dev = torch.empty_like(b)
    x_dev = torch.empty(n, dtype=torch.float64, device=dev)
    e2e_steps = max(2, min(args.steps, 5))
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        b_dev.copy_(b_host, non_blocking=True)
        ctx.reset(b_dev)
        ctx.iterate(gamma, eta, T)
        ctx.xbar(out=x_dev)
        x_host.copy_(x_dev, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_value = e2e_steps * T / (e0.elapsed_time(e1) / 1e3)

    extra = {}
    if args.fp32 and rank == 0:
        ctx32 = apc.apc_setup(A, b, offs, precision="f32", cluster_size=0)
        ctx32.reset()
        ctx32.iterate(gamma, eta, 20)
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        ctx32.iterate(gamma, eta, T)
        a1.record(stream)
        torch.cuda.synchronize()
        s32 = a0.elapsed_time(a1) / 1e3
        b32 = ctx32.info()["q_bytes"] + state_bytes
        extra["fp32"] = {"iter_per_s": T / s32, "hbm_gbs": b32 * T / s32 / 1e9, "q_bytes": ctx32.info()["q_bytes"]}
        ctx32.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        rows = 8 * 256
        A_s = A[:rows].cpu().numpy()
        sec = oracle_sample(A_s, np.arange(0, rows + 1, 256), m, iters=2)
        cpu = {"value": 1.0 / sec, "unit": "iter/s", "cores": _threads(), "kind": "oracle",
               "sample": "8 of 128 row blocks (2048 x 32768 FP64) of the same matrix, 2 Eq. (cons) "
                         "iterations, time scaled x16 to all blocks"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "iter/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": f"APC n={n} A=D_r G D_c (log-uniform 1e-2..1e2), m={m} blocks of {n // m}, "
                                   f"Q {args.precision}, FP32 accumulation",
                       "iters_per_step": T, "l2": f"Q {q_bytes / 2**30:.2f} GiB > L2 129 MB, no flush",
                       "cluster_size": info["cluster_size"], "clusters": info["clusters"],
                       "setup_s": setup_s},
            "e2e": {"value": e2e_value, "unit": "iter/s", "h2d_bytes_per_step": n * 8, "d2h_bytes_per_step": n * 8},
            "gpu_launches": args.steps * (1 + (T > (1 << 20))),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                         "kernel": "apc_iter_kernel", "bytes_per_iter": bytes_per_iter},
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


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
    p.add_argument("--fp32", type=int, default=1)
    p.add_argument("--no-cpu", action="store_true")
    args = p.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        from paper_1708_01413_gb300 import build
        build.build()
        run_ours(args)


if __name__ == "__main__":
    main()
