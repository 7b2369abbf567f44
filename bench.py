#!/usr/bin/env python
"""Benchmark: filter TFLOP/s and time to nev eigenpairs at tol 1e-10 on one GB300.

One step = one full pass of the hot path on the synthetic workload: Lanczos
bounds, the filtered subspace iteration (filter, CholeskyQR2, oblique
Rayleigh-Ritz, residuals, locking, per-vector degrees) until nev pairs are
locked, and the eigenvalue-gradient backward of L = sum_i w_i lambda_i.  The
default workload is n16384: H of size 32768, nev 1000, nex 300, degrees up to
36, tol 1e-10, a dense band of 5 % of the eigenvalues at the bottom of the
spectrum, mixed precision (FP16x3 tensor-core filter, FP64-accurate products
elsewhere).

Printed JSON line (rank 0):
  value            filter TFLOP/s over the timed steps (algorithmic flops
                   64 n^2 sum_i deg_i of the filter / device time in the filter)
  time_to_solution seconds per step (device events, mean over the steps)
  e2e              the same metric through the Python/C-ABI entry points with
                   host buffers, host<->device copies inside the timed region
  roofline         the dominant kernel (the filter GEMM) against the measured peak
  cpu_baseline     the CPU oracle (a bounded sample) on the host cores
  eig_error        per-eigenvalue error bounds of the returned pairs, from FP64
                   products computed independently of the solver

Under torchrun (N > 1) every rank solves its own independent problem instance
(replicas: the method has no data-path exchange on one problem per GPU).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "filter TFLOP/s + time to nev eigenpairs at tol=1e-10, mixed vs FP64 on 1 GB300"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
# nominal dense rates (TFLOP/s) used to scale a measured bf16 peak to another dtype
NOMINAL = {"bf16": 2250.0, "fp16": 2250.0, "fp64": 1.25}
# workloads whose inputs are assembled on the device (the host QR of the Haar-unitary
# factor takes minutes at these sizes)
DEVICE_INPUTS_FROM = 8192
# the ncu summary that holds the DRAM traffic of the filter GEMM per workload
TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "tc_hop_fp16x3_traffic.md")
FILTER_SOURCE = os.path.join(ROOT, "paper_2601_10557_gb300", "csrc", "tc_filter.cu")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="n16384")
    p.add_argument("--precision", default="auto", choices=["auto", "fp64", "mixed", "fp16x3", "bf16x3", "bf16x6"])
    p.add_argument("--no-fp64-compare", action="store_true")
    p.add_argument("--e2e-steps", type=int, default=None,
                   help="end-to-end steps (default: 1 for n >= 16384, else --steps)")
    p.add_argument("--filter-only", action="store_true",
                   help="only the filter roofline measurement (one warm and one timed chase_bse_filter call)")
    p.add_argument("--deg", type=int, default=None, help="filter degree for --filter-only")
    p.add_argument("--profile-step", action="store_true",
                   help="one step (solve + gradient) of the workload and nothing else, for a profiler's launch list")
    return p.parse_args()


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return dict(PEAKS_FALLBACK), "fallback"


def filter_source_hash() -> str:
    with open(FILTER_SOURCE, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def traffic_for(workload: str):
    """DRAM bytes per filter-GEMM launch (dram__bytes_read.sum + dram__bytes_write.sum)
    from the committed ncu summary, or None when it has no line for this workload or
    was taken on another version of the kernel source."""
    if not os.path.exists(TRAFFIC_PROFILE):
        return None, "no capture"
    txt = open(TRAFFIC_PROFILE).read()
    m = re.search(r"kernel source sha256\[:16\]:\s*([0-9a-f]{16})", txt)
    if not m or m.group(1) != filter_source_hash():
        return None, "capture predates the current kernel source"
    m = re.search(rf"traffic_bytes_per_launch\[{re.escape(workload)}\]:\s*([0-9.e+]+)", txt)
    if not m:
        return None, f"no capture for {workload}"
    return float(m.group(1)), "ncu capture (profiles/" + os.path.basename(TRAFFIC_PROFILE) + ")"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def reduce_scalar(dist, x: float, op: str, device) -> float:
    """MAX or SUM of a per-rank scalar over the default process group (the
    scalar itself without one)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_tflops(dist, flops: float, ms: float, device) -> float:
    """Whole-job throughput of N replicas: the flops of all ranks over the
    slowest rank's time (ms)."""
    return reduce_scalar(dist, flops, "sum", device) / (reduce_scalar(dist, ms, "max", device) / 1e3) / 1e12


def make_inputs(wl: dict, seed: int, device=None):
    """(A, B, d, W0, V0, w): A, B as numpy arrays (host generator) or, for large n with
    a device given, torch tensors assembled on that device."""
    import bse_inputs as bi
    n = wl["n"]
    if device is not None and n >= DEVICE_INPUTS_FROM:
        A, B, d = bi.make_problem_device(n, seed, wl["spec"], wl["beta"], device=device)
    else:
        P = bi.make_problem(n, seed=seed, spec=wl["spec"], beta=wl["beta"])
        A, B, d = P.A, P.B, P.d
    nevex = wl["nev"] + wl["nex"]
    W0 = bi.start_block(n, nevex, seed)
    V0 = bi.lanczos_starts(n, 4, seed)
    w = bi.loss_weights(wl["nev"], seed)
    return A, B, d, W0, V0, w


def cpu_oracle_sample(A, B, W0, wl, ncols=None):
    """The oracle as it stands: one H^2 step of its Chebyshev filter (degree 1) over
    ncols columns (all nev + nex by default), timed on the host cores."""
    import numpy as np
    from oracle import chebyshev
    n = wl["n"]
    W = W0 if ncols is None else W0[:ncols]
    k = W.shape[0]
    lam_guess = (0.9, 2.0, 60.0)
    t0 = time.perf_counter()
    chebyshev.chebyshev_filter(A, B, W.T, np.ones(k, dtype=int), *lam_guess)
    dt = time.perf_counter() - t0
    flops = 64.0 * n * n * k
    return {"value": flops / dt / 1e12, "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"one H^2 step (degree 1) of the oracle filter, n={n}, {k} columns, "
                      f"{dt:.2f} s incl. forming H; the metric's unit scaled by 64 n^2 k flops"}


def sample_columns(wl):
    """Columns of the bounded CPU sample: all nev + nex up to n = 4096, 32 beyond."""
    return None if wl["n"] <= 4096 else 32


def host_inputs(wl, seed):
    """Inputs as numpy arrays for the CPU oracle (device assembly when large)."""
    import torch
    dev = torch.device("cuda", 0) if torch.cuda.is_available() else None
    A, B, d, W0, V0, w = make_inputs(wl, seed, device=dev)
    if not isinstance(A, type(W0)):
        A, B = A.cpu().numpy(), B.cpu().numpy()
    return A, B, W0


def config_dict(args, wl, precision, world):
    """The workload's description, the same in both arms' JSON lines."""
    n = wl["n"]
    return {"workload": args.workload, "n": n, "H": 2 * n, "nev": wl["nev"], "nex": wl["nex"],
            "deg": f"{wl['deg_min']}-{wl['deg_max']} adaptive, first {wl['deg']}", "tol": wl["tol"],
            "spectrum": wl["spec"], "beta": wl["beta"], "precision": precision,
            "l2": "inputs larger than L2 (A and B: %.0f MB)" % (2 * n * n * 16 / 1e6),
            "parallelism": f"replicas x{world}"}


def run_reference(args, wl, rank, world):
    if rank != 0:
        return
    import numpy as np
    A, B, W0 = host_inputs(wl, 0)
    ncols = sample_columns(wl)
    steps, warm = max(args.steps, 1), max(args.warmup, 0)
    samples = []
    for i in range(warm + steps):
        s = cpu_oracle_sample(A, B, W0, wl, ncols)
        if i >= warm:
            samples.append(s["value"])
    v = float(np.mean(samples))
    cols = W0.shape[0] if ncols is None else ncols
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": steps, "warmup": warm, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": config_dict(args, wl, "mixed" if args.precision == "auto" else args.precision, world),
            "cpu_baseline": {"value": v, "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"per step: one H^2 step (degree 1) of the oracle filter over {cols} "
                                       "columns of the same workload"},
            "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def filter_only(args, wl):
    import torch
    import paper_2601_10557_gb300 as pkg
    dev = torch.device("cuda", 0)
    A, B, d, W0n, _, _ = make_inputs(wl, 0, device=dev)
    A, B = (torch.as_tensor(A).to(dev), torch.as_tensor(B).to(dev))
    W = torch.from_numpy(W0n).to(dev)
    prec = args.precision if args.precision != "auto" else ("mixed" if pkg.has_mixed() else "fp64")
    deg = args.deg or wl["deg"]
    k = W.shape[0]
    pkg.filter(A, B, W.clone(), [deg] * k, 1.0, 2.0, 60.0, precision=prec)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    Wt = W.clone()
    e0.record()
    pkg.filter(A, B, Wt, [deg] * k, 1.0, 2.0, 60.0, precision=prec)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    fl = 64.0 * wl["n"] ** 2 * k * deg
    print(json.dumps({"filter_only": True, "precision": prec, "n": wl["n"], "k": k, "deg": deg, "ms": ms,
                      "tflops": fl / ms / 1e9}), flush=True)


def profile_step(args, wl):
    """One step of the workload (mixed solve + gradient) and nothing else."""
    import torch
    import paper_2601_10557_gb300 as pkg
    dev = torch.device("cuda", 0)
    A, B, d, W0n, V0n, wn = make_inputs(wl, 0, device=dev)
    A, B = torch.as_tensor(A).to(dev), torch.as_tensor(B).to(dev)
    prec = args.precision if args.precision != "auto" else ("mixed" if pkg.has_mixed() else "fp64")
    W0, V0, w = torch.from_numpy(W0n).to(dev), torch.from_numpy(V0n).to(dev), torch.from_numpy(wn).to(dev)
    torch.cuda.synchronize()
    # the profiler's capture range (ncu --profile-from-start off): the solve and the
    # gradient, not the assembly of the inputs
    torch.cuda.profiler.start()
    lam, V, st = pkg.solve(A, B, wl["nev"], wl["nex"], wl["deg"], wl["tol"], precision=prec, W0=W0, V0=V0,
                           deg_min=wl["deg_min"], deg_max=wl["deg_max"], maxiter=40)
    pkg.grad(V, w)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print(json.dumps({"profile_step": True, "workload": args.workload, "iterations": st["iterations"],
                      "ms_total": st["ms_total"], "launches": pkg.launch_count()}), flush=True)


def eig_error_bounds(A, B, lam, V, nsample: int = 100):
    """Per-eigenvalue error bounds of returned pairs against the exact eigenvalues (what
    an FP64 solve converges to), from FP64 products done here with torch, not by the
    solver: r = ||H v - lambda v|| and s = v^* S v give |lambda - lambda_exact| <= r/|s|
    to first order (v^* S is the left eigenvector, Theorem SH_HPD), and the S-Rayleigh
    quotient rho = v^* S H v / s differs from lambda by O(r^2).  Every nev/nsample-th pair."""
    import torch
    nev = lam.shape[0]
    idx = torch.arange(0, nev, max(1, nev // nsample), device=V.device)
    Vs = V[idx].T.contiguous()  # 2n x m
    n = A.shape[0]
    X, Y = Vs[:n], Vs[n:]
    # A, B are the (row-major) matrices themselves: H v = [A x + B y; -conj(B) x - conj(A) y]
    top = A @ X + B @ Y
    bot = -(B.conj() @ X) - A.conj() @ Y
    HV = torch.cat([top, bot], dim=0)
    lv = lam[idx]
    R = HV - Vs * lv[None, :]
    r = torch.linalg.vector_norm(R, dim=0)
    SV = torch.cat([X, -Y], dim=0)
    s = torch.real(torch.sum(SV.conj() * Vs, dim=0))
    rho = torch.real(torch.sum(SV.conj() * HV, dim=0)) / s
    bound = (r / s.abs()) / lv.abs()
    rq = (rho - lv).abs() / lv.abs()
    # second order: |rho - lambda_exact| <~ r^2 / (|s| gap), gap = distance to the nearest
    # other returned eigenvalue (no eigenvalue is missing from the returned set: the
    # completeness of the returned set is the inertia test's subject)
    srt = torch.sort(lam).values
    gaps = torch.empty_like(lam)
    d = srt[1:] - srt[:-1]
    gaps[0], gaps[-1] = d[0], d[-1]
    gaps[1:-1] = torch.minimum(d[1:], d[:-1])
    gsel = gaps[idx]
    bound2 = (r * r / (s.abs() * gsel)) / lv.abs()
    return {"reference": "exact eigenvalue; first-order bound ||Hv - lambda v|| / (|v^* S v| lambda), "
                         "second-order bound ||Hv - lambda v||^2 / (|v^* S v| gap lambda) and "
                         "|rho_S - lambda| / lambda with rho_S the S-Rayleigh quotient, FP64 torch products",
            "sampled_pairs": int(idx.numel()), "max_rel_bound": float(bound.max()),
            "max_rel_bound_second_order": float(bound2.max()),
            "max_rel_rayleigh_diff": float(rq.max()),
            "per_eigenvalue": [{"i": int(i), "lambda": float(l), "rel_bound": float(b), "rel_bound2": float(b2),
                                "rel_rq_diff": float(q)}
                               for i, l, b, b2, q in zip(idx.tolist(), lv.tolist(), bound.tolist(), bound2.tolist(),
                                                         rq.tolist())]}


def main():
    args = parse()
    import bse_inputs as bi
    wl = dict(bi.WORKLOADS[args.workload])
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, wl, rank, world)
        return
    if args.filter_only:
        filter_only(args, wl)
        return
    if args.profile_step:
        profile_step(args, wl)
        return

    import numpy as np
    import torch
    import paper_2601_10557_gb300 as pkg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    precision = args.precision
    if precision == "auto":
        precision = "mixed" if pkg.has_mixed() else "fp64"
    n, nev, nex = wl["n"], wl["nev"], wl["nex"]
    nevex = nev + nex
    A, B, d, W0n, V0n, wn = make_inputs(wl, rank, device=dev)
    A = torch.as_tensor(A).to(dev)
    B = torch.as_tensor(B).to(dev)
    W0 = torch.from_numpy(W0n).to(dev)
    V0 = torch.from_numpy(V0n).to(dev)
    w = torch.from_numpy(wn).to(dev)
    kw = dict(W0=W0, V0=V0, deg_min=wl["deg_min"], deg_max=wl["deg_max"], maxiter=40)

    def step(prec):
        lam, V, st = pkg.solve(A, B, nev, nex, wl["deg"], wl["tol"], precision=prec, **kw)
        gA, gB = pkg.grad(V, w)
        return lam, V, st, gA, gB

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    warm = max(args.warmup, 3)
    for _ in range(warm):
        step(precision)
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    l0 = pkg.launch_count()
    gemm_kind = "fp64" if precision == "fp64" else "tensor"
    pkg.gemm_timer(True)  # CUDA events around every filter GEMM launch of the timed steps
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    fl = fms = 0.0
    iters = []
    maxres = 0.0
    phases = {}
    for _ in range(args.steps):
        lam, V, st, gA, gB = step(precision)
        for key in ("ms_total", "ms_lanczos", "ms_filter", "ms_filter_mixed", "ms_filter_fp64", "ms_qr", "ms_rr",
                    "ms_resid"):
            phases[key] = phases.get(key, 0.0) + st[key] / args.steps
        fl += st["filter_flops"]
        fms += st["ms_filter"]
        iters.append(st["iterations"])
        maxres = max(maxres, st["max_residual"])
    ev1.record(stream)
    barrier()
    clocks.stop()
    launches = pkg.launch_count() - l0
    g_ms, g_flops, g_n = pkg.gemm_time(gemm_kind)
    pkg.gemm_timer(False)
    total_ms = ev0.elapsed_time(ev1)
    tts = total_ms / 1e3 / args.steps

    value = whole_job_tflops(dist, fl, fms, dev)
    tts_max = reduce_scalar(dist, tts, "max", dev)
    lam_np = lam.cpu().numpy()

    # ---- per-eigenvalue error bounds of the last timed result (independent FP64 products)
    eig_err = eig_error_bounds(A, B, lam, V) if rank == 0 else None
    torch.cuda.synchronize()

    # ---- e2e through the public API with host buffers
    e2e_steps = args.e2e_steps if args.e2e_steps is not None else (1 if n >= 16384 else args.steps)
    hA = A.cpu().pin_memory()
    hB = B.cpu().pin_memory()
    hW0 = torch.from_numpy(W0n).pin_memory()
    hV0 = torch.from_numpy(V0n).pin_memory()
    hw = torch.from_numpy(wn).pin_memory()
    out_l = torch.empty(nev, dtype=torch.float64).pin_memory()
    out_gA = torch.empty((n, n), dtype=torch.complex128).pin_memory()
    out_gB = torch.empty((n, n), dtype=torch.complex128).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in (hA, hB, hW0, hV0, hw))
    d2h = sum(t.numel() * t.element_size() for t in (out_l, out_gA, out_gB))
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    efl = 0.0
    for _ in range(max(e2e_steps, 1)):
        dA = hA.to(dev, non_blocking=True)
        dB = hB.to(dev, non_blocking=True)
        dW = hW0.to(dev, non_blocking=True)
        dV = hV0.to(dev, non_blocking=True)
        dw = hw.to(dev, non_blocking=True)
        lam2, V2, st2 = pkg.solve(dA, dB, nev, nex, wl["deg"], wl["tol"], precision=precision, W0=dW, V0=dV,
                                  deg_min=wl["deg_min"], deg_max=wl["deg_max"], maxiter=40)
        g2A, g2B = pkg.grad(V2, dw)
        out_l.copy_(lam2, non_blocking=True)
        out_gA.copy_(g2A, non_blocking=True)
        out_gB.copy_(g2B, non_blocking=True)
        efl += st2["filter_flops"]
        del dA, dB, g2A, g2B
    e1.record(stream)
    barrier()
    e2e_ms = reduce_scalar(dist, e0.elapsed_time(e1), "max", dev)
    e2e_val = whole_job_tflops(dist, efl, e2e_ms, dev)
    del hA, hB, out_gA, out_gB

    # ---- roofline of the dominant kernel, the filter GEMM: the algorithmic flops of its
    # launches in the timed steps (32 n^2 k for k vectors) over their summed device time
    # (a CUDA event pair around each launch, recorded by the library on the launch's
    # stream).  Cross-check on full-width launches: two filter calls over all nev + nex
    # columns that differ only in the degree (d1 and d2 H^2 steps: 2 (d2 - d1) more
    # launches of the same shape; the split of P, the packing and the final combination,
    # the same in both, cancel)
    d1, d2 = (2, 6) if n >= 16384 else (4, 20)

    def filter_ms(deg):
        Wr = W0.clone()
        barrier()
        r0 = torch.cuda.Event(enable_timing=True)
        r1 = torch.cuda.Event(enable_timing=True)
        r0.record(stream)
        pkg.filter(A, B, Wr, [deg] * nevex, 1.0, 2.0, 60.0, precision=precision)
        r1.record(stream)
        torch.cuda.synchronize()
        return r0.elapsed_time(r1)

    filter_ms(d1)  # warm
    rl0 = pkg.launch_count()
    t1 = min(filter_ms(d1) for _ in range(2))
    t2 = min(filter_ms(d2) for _ in range(2))
    rl = (pkg.launch_count() - rl0) // 4
    gemm_launches = 2 * (d2 - d1)
    full_launch_ms = (t2 - t1) / gemm_launches
    full_flops = 32.0 * n * n * nevex
    full_achieved = full_flops / (full_launch_ms / 1e3) / 1e12
    per_launch_ms = g_ms / max(g_n, 1)
    flops_per_launch = g_flops / max(g_n, 1)
    achieved = g_flops / (g_ms / 1e3) / 1e12 if g_ms > 0 else 0.0
    # launches timed inside steps of several seconds or more (the sustained peak was
    # measured over a 4 s loop) take the sustained measured peak as their denominator,
    # launches in shorter steps the burst peak; the full-width check times short calls
    # alone and takes the burst peak
    peaks, peak_src = load_peaks()
    long_steps = tts >= 4.0 and "bf16_tflops_sustained" in peaks
    sustained = peaks["bf16_tflops_sustained"] if long_steps else peaks["bf16_tflops"]
    kind_s = "sustained (steps of %.1f s)" % tts if long_steps else "burst (steps of %.2f s)" % tts
    if precision == "fp64":
        peak = sustained * NOMINAL["fp64"] / NOMINAL["bf16"]
        peak_burst = peaks["bf16_tflops"] * NOMINAL["fp64"] / NOMINAL["bf16"]
        peak_note = f"{peak_src} bf16 {kind_s} x nominal fp64/bf16 ratio (1.25/2250)"
    elif precision == "bf16x6":
        peak, peak_burst = sustained / 6.0, peaks["bf16_tflops"] / 6.0
        peak_note = f"{peak_src} bf16 {kind_s} / 6 (six 16-bit products per FP32-accurate product)"
    else:
        peak, peak_burst = sustained / 3.0, peaks["bf16_tflops"] / 3.0
        peak_note = (f"{peak_src} bf16 {kind_s} / 3 (three 16-bit products per FP32-accurate product; "
                     "the nominal FP16 and BF16 dense rates are equal)")
    traffic_full, traffic_src = traffic_for(args.workload) if precision in ("mixed", "fp16x3") else (None, "n/a")
    traffic = None
    if traffic_full is not None:
        # captured on full-width launches (k = nev + nex); scaled to the timed launches'
        # average width by the units processed (the operand re-reads grow with the
        # number of column tiles)
        traffic = traffic_full * flops_per_launch / full_flops
        traffic_src += f"; full-width launch {traffic_full:.4g} B scaled by the average width {flops_per_launch / full_flops:.3f}"
    roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": traffic, "traffic_source": traffic_src,
            "kernel": "hop_kernel (FP64 DFMA)" if precision == "fp64" else "tc_hop_kernel (tcgen05 filter GEMM)",
            "peak_source": peak_note, "launch_ms": per_launch_ms, "launches": g_n,
            "flops_per_launch": flops_per_launch,
            "method": "sum of 32 n^2 k over the filter GEMM launches of the timed steps / their summed "
                      "device time (a CUDA event pair around each launch on its stream)",
            "full_width_check": {
                "achieved": full_achieved, "frac": full_achieved / peak_burst, "peak": peak_burst,
                "peak_source": f"{peak_src} bf16 burst / 3 (short calls timed alone)", "launch_ms": full_launch_ms,
                "flops_per_launch": full_flops,
                "method": f"(t(degree {d2}) - t(degree {d1})) / {gemm_launches} launches, filter calls over "
                          f"{nevex} columns, CUDA events, best of 2",
                "launches_per_call_avg": rl, "filter_call_ms": {str(d1): t1, str(d2): t2}}}

    # ---- FP64 comparison: the plain FP64 solve (FP64 pipe) and the FP64-accurate solve with
    # every large product on the tensor cores (fp64_tc)
    fp64 = None
    if precision != "fp64" and not args.no_fp64_compare:
        if n <= 4096:
            barrier()
            f0 = torch.cuda.Event(enable_timing=True)
            f1 = torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            step("fp64")
            f1.record(stream)
            barrier()
            fp64 = {"time_to_solution_s": reduce_scalar(dist, f0.elapsed_time(f1) / 1e3, "max", dev),
                    "kind": "measured: one plain FP64 solve + gradient (unwarmed)"}
            step("fp64_tc")
            barrier()
            f0.record(stream)
            step("fp64_tc")
            f1.record(stream)
            barrier()
            fp64["fp64_tc_time_to_solution_s"] = reduce_scalar(dist, f0.elapsed_time(f1) / 1e3, "max", dev)
            fp64["fp64_tc_kind"] = ("measured: one FP64-accurate solve + gradient with every large product a "
                                    "sliced tensor-core GEMM (after one warm-up solve)")
        else:
            # the plain FP64 solve takes hours here: its filter alone, at the FP64 filter
            # rate measured on a short call, is a lower bound of its time
            kc = 64
            Wf = W0[:kc].clone()
            pkg.filter(A, B, Wf, [1] * kc, 1.0, 2.0, 60.0, precision="fp64")
            barrier()
            f0 = torch.cuda.Event(enable_timing=True)
            f1 = torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            pkg.filter(A, B, Wf, [2] * kc, 1.0, 2.0, 60.0, precision="fp64")
            f1.record(stream)
            barrier()
            rate = 64.0 * n * n * kc * 2 / (f0.elapsed_time(f1) / 1e3)
            flops_step = fl / max(args.steps, 1)
            fp64 = {"time_to_solution_s": flops_step / rate,
                    "kind": "extrapolated lower bound: the mixed solve's filter flops "
                            f"({flops_step:.3e}) at the FP64 filter rate measured on a degree-2 call over "
                            f"{kc} columns ({rate / 1e12:.3f} TFLOP/s); QR, Rayleigh-Ritz and the "
                            "FP64 filter's extra iterations not counted",
                    "fp64_filter_tflops": rate / 1e12}
            del Wf
            # the FP64-accurate filter on the tensor cores: a degree-1 call over all columns
            Wt = W0.clone()
            pkg.filter(A, B, Wt, [1] * nevex, 1.0, 2.0, 60.0, precision="fp64_tc")
            barrier()
            f0.record(stream)
            pkg.filter(A, B, Wt, [1] * nevex, 1.0, 2.0, 60.0, precision="fp64_tc")
            f1.record(stream)
            barrier()
            rate_tc = 64.0 * n * n * nevex / (f0.elapsed_time(f1) / 1e3)
            del Wt
            fp64["fp64_tc_time_to_solution_s"] = flops_step / rate_tc
            fp64["fp64_tc_kind"] = ("extrapolated lower bound: the same filter flops at the rate of the FP64-accurate "
                                    f"sliced tensor-core filter measured on a degree-1 call over {nevex} columns "
                                    f"({rate_tc / 1e12:.2f} TFLOP/s, slicing of H included)")
            fp64["fp64_tc_filter_tflops"] = rate_tc / 1e12

    # ---- the explicit-H^2 variant (not the paper's method): one measured solve + gradient
    h2x = None
    if precision not in ("fp64", "fp64_tc") and not args.no_fp64_compare:
        barrier()
        x0 = torch.cuda.Event(enable_timing=True)
        x1 = torch.cuda.Event(enable_timing=True)
        x0.record(stream)
        lamx, Vx, stx = pkg.solve(A, B, nev, nex, wl["deg"], wl["tol"], precision=precision, h2="explicit", **kw)
        pkg.grad(Vx, w)
        x1.record(stream)
        barrier()
        h2x = {"time_to_solution_s": reduce_scalar(dist, x0.elapsed_time(x1) / 1e3, "max", dev),
               "iterations": stx["iterations"], "max_residual": stx["max_residual"],
               "ms_h2": stx["ms_h2"], "ms_filter": stx["ms_filter"],
               "max_rel_diff_to_timed_lambda": float(((lamx - lam).abs() / lam.abs()).max()),
               "kind": "measured: one mixed solve + gradient with the blocks of H^2 formed once (FP64-accurate "
                       "sliced GEMMs) and one tensor-core product per filter step; not the paper's method"}
        del lamx, Vx

    cpu = None
    if rank == 0 and world == 1:
        hAn, hBn = A.cpu().numpy(), B.cpu().numpy()
        cpu = cpu_oracle_sample(hAn, hBn, W0n, wl, sample_columns(wl))
        del hAn, hBn

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": warm, "ms_per_step": tts_max * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if precision == "fp64" else "fp16x3+f64",
            "data": "synthetic",
            "config": config_dict(args, wl, precision, world),
            "time_to_solution_s": tts_max,
            "time_to_solution_fp64_s": (fp64 or {}).get("time_to_solution_s") if precision != "fp64" else tts_max,
            "fp64_comparison": fp64,
            "explicit_h2": h2x,
            "iterations": iters, "max_residual": maxres,
            "phases_ms_per_step": {k2: round(v2, 2) for k2, v2 in phases.items()},
            "lambda_min_max": [float(lam_np[0]), float(lam_np[-1])],
            "eig_error": eig_err,
            "e2e": {"value": e2e_val, "unit": "TFLOP/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": e2e_ms / max(e2e_steps, 1), "steps": max(e2e_steps, 1)},
            "gpu_launches": launches,
            "roofline": roof,
            "cpu_baseline": cpu,
            "clocks": clocks.summary(),
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
