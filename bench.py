#!/usr/bin/env python
"""Benchmark: parareal wall time to relative error 1e-8 against the serial
GPU solve, reported as fine steps x modes per second.

One "step" is one complete parareal solve (coarse sweep, F stages, coarse
sweeps with correction, stopping test) of the batched 1D workload: 256
instances with seeded uneven K in [64,256], N = 64 m with m in [16,64]
(N in [1024,4096]), alpha in {0.3,0.5,0.7,1.0}, P = 64 slices.  The error is
measured against the sequential fine sweep S_hyb (parareal's fixed point)
solved on the GPU in plain FP64.  The stopping rule is fixed in advance:
parareal stops once its increment e_k is below the target error (1e-8);
the loosest tolerance that still reaches 1e-8 (found with the reference
solution, which a user does not have) is reported beside it as context only.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
       python bench.py --workload uniform-history    (the uniform solver's history stream case)
Under torchrun each rank solves its own batch (seed + rank): weak scaling,
no collective on the data path; rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "parareal wall-time to rel err 1e-8 vs serial GPU solve; fine steps*modes/s"
UNIT = "fine_steps*modes/s"
TARGET = 1e-8
FIXED_TOL = TARGET             # increment tolerance of the stopping rule, fixed in advance
INEXACT_ABOVE = (1e-4, 1e-5, 3e-6)   # increments above which early iterations take the FP32 step (candidates)
REFINE_FACTORS = (1e-3, 1e-2, 1e-1)  # refined F steps of slices n > k stop at factor * e_{k-1} (candidates)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed", "fp32"])
    ap.add_argument("--workload", default="batched1d",
                    choices=["batched1d", "2d", "2d-batched", "uniform-history", "paper-model", "assembly",
                             "learned-g"],
                    help="batched1d: the headline 1D batch; 2d: one 32 x 32-mode instance, N = 2048, P = 128; "
                         "2d-batched: --batch instances of 64 x 64 modes, N = 8192, P = 256; uniform-history: "
                         "the uniform serial solve of 96 instances, K = 256, N = 1024 (history stream from HBM); "
                         "paper-model: the paper's model problem with its collocation scheme, FP64 (Sec. 4.2); "
                         "assembly: dense stiffness by tensor-core GEMM vs Toeplitz+Hankel moments, K = 256; "
                         "learned-g: the learned coarse propagator at its own size (K = 128, N = 4096, P = 64)")
    ap.add_argument("--batch", type=int, default=0, help="instances (0: 256 for batched1d, 16 for 2d-batched)")
    ap.add_argument("--seed", type=int, default=20251011)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="time the host-loop parareal instead of the graph")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-uniform", action="store_true", help="skip timing the uniform-history serial solve")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-step-seconds", type=float, default=0.0,
                    help="CPU seconds per reference-arm step (0: about 2 minutes in total)")
    ap.add_argument("--no-ref-context", action="store_true",
                    help="reference arm: skip the oracle's whole solves of the small configurations")
    ap.add_argument("--coarse", default="auto", choices=["auto", "l1", "l1x2", "l1x4", "l1x8", "learned"],
                    help="coarse propagator: the one-step L1 G, the L1 G with 2 or 4 substeps per slice, or the "
                         "learned correction; auto: the fastest to rel err 1e-8 in warm-up")
    ap.add_argument("--inexact", default="auto", choices=["auto", "on", "off"],
                    help="inexact early iterations (the FP32 step on slices not yet exact while the increment "
                         "exceeds a threshold, 1e-4, 1e-5 or 3e-6; mixed); auto: the fastest to rel err 1e-8 in warm-up")
    ap.add_argument("--sweep-split", type=int, default=0, choices=[0, 1, 2, 4, 8],
                    help="2D: CTAs of the cluster that shares each coarse-sweep step (0: the library's choice)")
    ap.add_argument("--train-batch", type=int, default=128, help="instances the learned correction trains on")
    ap.add_argument("--train-iters", type=int, default=8)
    ap.add_argument("--train-epochs", type=int, default=40)
    ap.add_argument("--reference", default="fp64", choices=["fp64", "same"],
                    help="precision of the serial S_hyb the error is measured against (same: profiling runs)")
    return ap.parse_args()


# ---------------------------------------------------------------- distributed
class Dist:
    def __init__(self, n_gpus: int, backend: str):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def sum(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.rows, self.proc = index, [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            for i, n in enumerate(names):
                if r[5 + i].lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


# ---------------------------------------------------------------- work accounting
def rel_err(U, S) -> float:
    """max over instances of max_n ||U_n - S_n||_2 / max_n ||S_n||_2."""
    return max(float(np.sqrt(((u - s) ** 2).sum(1)).max() / np.sqrt((s**2).sum(1)).max()) for u, s in zip(U, S))


# ---------------------------------------------------------------- CPU oracle sample
def oracle_prob(spec, P):
    import oracle as O
    return O.make_prob(dim=spec.dim, Mx=spec.modes[0], My=spec.modes[1], Qx=spec.qnodes[0] or None,
                       Qy=spec.qnodes[1] or None, N=spec.nsteps, P=P, alpha=spec.alpha, T=spec.T,
                       lo=spec.lo, hi=spec.hi, dpar=spec.dpar, fpar=spec.fpar, basis=spec.basis)


def make_workload(args, rank: int = 0):
    from paper_2510_11023_gb300 import workloads
    if args.workload == "2d":
        return workloads.cfg3()
    if args.workload == "2d-batched":
        return workloads.cfg5(B=args.batch or 16)
    return workloads.cfg2(B=args.batch or 256, seed=args.seed + rank)


def oracle_throughput_2d(wl, seconds: float) -> tuple:
    """2D: one oracle step of a reduced instance (half the modes per axis,
    same node ratio), repeated while time remains, scaled to the full size by
    the oracle's own cost model: its stiffness sum costs K^2 Q, 64x more at
    twice the modes per axis.  Returns (fine step-modes per second, seconds, steps)."""
    import dataclasses

    import oracle as O
    O.build()
    s = wl.specs[0]
    small = dataclasses.replace(s, modes=(s.modes[0] // 2, s.modes[1] // 2))
    op = oracle_prob(small, wl.P)
    c = np.zeros(small.K)
    c[0] = 0.5
    scale = (s.K / small.K) ** 2 * (s.Q / small.Q)
    t0, nstep = time.perf_counter(), 0
    while nstep == 0 or time.perf_counter() - t0 < seconds:
        O.step(op, c, 0.1, 0.01, c)
        nstep += 1
    dt = time.perf_counter() - t0
    return nstep * s.K / (dt * scale), dt, nstep


_HIST_CACHE: dict = {}


def oracle_throughput(wl, S, seconds: float, omp: bool = True) -> tuple:
    """The FP64 oracle on a bounded sample of the workload: for successive
    instances, the fine propagators F_n of the slices n = P/2 .. P/2 + T - 1
    (T = host threads of the OpenMP build, one slice per thread, as the paper
    runs its parallel stage; T = 1 for the serial build), until `seconds` of
    timed CPU work are spent.  Their history U_{0:n} comes from S (the GPU
    serial solve) or from the oracle's coarse sweep, computed outside the timed
    region.  Returns (fine step-modes per second, timed seconds, instances, T)."""
    import oracle as O
    if wl.specs[0].dim == 2:
        v, dt, n = oracle_throughput_2d(wl, seconds)
        return v, dt, n, 1
    O.build(omp=omp)
    T = O.threads(omp)
    n0 = wl.P // 2
    n1 = min(wl.P, n0 + T)
    work, timed, inst = 0.0, 0.0, 0
    while timed < seconds and inst < wl.B:
        s = wl.specs[inst]
        op = oracle_prob(s, wl.P)
        if S is not None:
            U = S[inst][:n1]
        else:
            key = (id(wl), inst)
            if key not in _HIST_CACHE:
                _HIST_CACHE[key] = O.coarse_sweep(op, wl.u0[inst])[:n1]
            U = _HIST_CACHE[key]
        t0 = time.perf_counter()
        O.fine_stage(op, U, n0, n1, omp=omp)
        timed += time.perf_counter() - t0
        work += (n1 - n0) * (s.nsteps // wl.P) * s.K
        inst += 1
    return work / timed, timed, inst, T


def oracle_paper_shapes() -> dict:
    """Whole solves by the oracle on the small configurations: the plain 1D
    case (K = 32, N = 256, P = 8) and the paper's model-problem shape
    (K = 16, P = 256, m = 32): S_uni, S_hyb and parareal (tolerance 1e-10, the
    paper's) on one thread, and parareal with its parallel stage on all host
    threads (OpenMP build).  Seconds per solve."""
    import oracle as O
    from paper_2510_11023_gb300 import workloads
    out = {}
    for name, wl in (("1d_plain_K32_N256_P8", workloads.cfg1()), ("paper_shape_K16_P256_m32", workloads.e1())):
        s = wl.specs[0]
        op = oracle_prob(s, wl.P)
        u0 = wl.u0[0]
        r = {"fine_steps_x_modes": s.nsteps * s.K}
        for key, fn in (("serial_uniform_s", lambda: O.serial_uni(op, u0)),
                        ("serial_hybrid_s", lambda: O.serial_hyb(op, u0))):
            t0 = time.perf_counter()
            fn()
            r[key] = time.perf_counter() - t0
        for omp in (False, True):
            t0 = time.perf_counter()
            _, _, k = O.parareal(op, u0, 1e-10, omp=omp)
            r["parareal_s_threads%d" % O.threads(omp)] = time.perf_counter() - t0
            r["parareal_iterations"] = k
        out[name] = r
    return out


def reference_arm(args, dist: Dist):
    if dist.rank != 0:
        return
    wl = make_workload(args)
    per_step = args.ref_step_seconds or max(2.0, 120.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_throughput(wl, None, per_step / 4)
    vals, secs, cores = [], [], 1
    for _ in range(args.steps):
        v, dt, ninst, cores = oracle_throughput(wl, None, per_step)
        vals.append(v)
        secs.append(dt)
    v = float(np.mean(vals))
    sample = (f"oracle fine propagators F_n, n = P/2 .. P/2+{cores - 1}, one per host thread (OpenMP build), "
              f"of successive instances of the batched workload, ~{per_step:.0f} s of timed work per step; "
              f"their coarse-sweep history computed outside the timed region")
    if wl.specs[0].dim == 2:
        sample = (f"oracle L1 steps of the instance with half the modes per axis, ~{per_step:.0f} s per step, "
                  f"scaled by the oracle's K^2 Q cost to the full size, 1 thread")
    extra = {}
    if wl.specs[0].dim == 1 and not args.no_ref_context:
        extra["oracle_paper_shapes"] = oracle_paper_shapes()
        # the serial solve S_hyb of a 16-instance subset of the batched workload, extrapolated
        # from the single-thread sample rate (an oracle step costs the same inside S_hyb)
        v1, dt1, n1, _ = oracle_throughput(wl, None, 10.0, omp=False)
        sub = wl.specs[:16]
        extra["oracle_batched_subset16"] = {
            "fine_steps_x_modes": float(sum(s_.nsteps * s_.K for s_ in sub)),
            "rate_1thread": v1, "rate_all_threads": v, "threads": cores,
            "serial_hybrid_s_extrapolated": float(sum(s_.nsteps * s_.K for s_ in sub)) / v1,
            "how": "rates of the fine-propagator sample above; S_hyb time = the subset's fine steps x modes / rate"}
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(secs)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl.name, "batch": wl.B, "P": wl.P},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "host_cpus": os.cpu_count()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}, **extra}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- algorithmic work
def alg_flops_step_1d(K: int, Q: int) -> float:
    """Algorithmic FLOPs of one linearised 1D step with the assembly in use:
    values at the Q nodes and the load vector (4 Q K), the 2K+1 quadrature
    moments of the Toeplitz+Hankel stiffness (2 Q (2K+1)), and the SPD solve
    counted as a direct solve (Cholesky K^3/3 and two triangular solves 2 K^2)."""
    return 4.0 * Q * K + 2.0 * Q * (2 * K + 1) + K**3 / 3.0 + 2.0 * K * K


TRAFFIC_SUMMARY = os.path.join(ROOT, "profiles", "k_fstage_dram_traffic_batched1d_256inst.md")


def source_digest() -> str:
    """sha256 over the library's CUDA sources and the public header: a DRAM-traffic
    figure taken by ncu is reported only while these are unchanged."""
    import glob
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2510_11023_gb300", "csrc")
    files = sorted(glob.glob(os.path.join(csrc, "*.cu")) + glob.glob(os.path.join(csrc, "*.cuh")) +
                   glob.glob(os.path.join(csrc, "*.h"))) + [os.path.join(ROOT, "include", "psl1.h")]
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def captured_traffic(config_key: str):
    """DRAM bytes (read + write) per k_fstage launch from the committed ncu summary, when
    it was captured on the current sources and on this configuration; else None."""
    try:
        fields = {}
        for line in open(TRAFFIC_SUMMARY):
            if line.startswith("- ") and ": " in line:
                k, v = line[2:].strip().split(": ", 1)
                fields[k.strip("`")] = v.strip().strip("`")
        if fields.get("sources_sha256") != source_digest() or fields.get("config") != config_key:
            return None
        return float(fields["bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


def fstage_alg_flops(wl, iters) -> tuple:
    """(algorithmic FLOPs of all F-stage launches of a solve, launches): at
    iteration k every instance still iterating runs its slices n = k..P-1."""
    total = 0.0
    for s, it in zip(wl.specs, iters):
        m = s.nsteps // wl.P
        steps = sum((wl.P - k) * m for k in range(int(it)))
        total += steps * alg_flops_step_1d(s.K, s.Q)
    return total, int(max(iters))


def uniform_history_case(args):
    """The uniform serial solve S_uni of 96 instances with K = 256 modes and
    N = 1024 fine steps (mixed precision): 2 MB of fine history per instance,
    192 MB in all, more than L2, so every history launch (k_uni_hist) streams
    from HBM.  The first solve tunes the stream and captures its graph; the
    second is timed."""
    import torch
    from paper_2510_11023_gb300 import psl1, workloads
    specs = [workloads.InstanceSpec(modes=(256, 1), nsteps=1024, alpha=0.5, dpar=workloads.D_CFG2,
                                    fpar=workloads.F_COS) for _ in range(96)]
    rng = np.random.default_rng(1)
    u0 = [rng.standard_normal(256) * np.arange(1, 257) ** -2.0 for _ in specs]
    wl = workloads.Workload("uniform history case: 96 x (K=256, N=1024)", 64, specs, u0)
    stream = torch.cuda.current_stream()
    out = {"workload": wl.name}
    with psl1.Problem(wl, precision="mixed", stream=stream.cuda_stream) as pr:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for kind in ("uniform", "uniform-soe"):
            pr.solve_serial(kind)
            e0.record(stream)
            pr.solve_serial(kind)
            e1.record(stream)
            torch.cuda.synchronize()
            out[kind.replace("-", "_") + "_solve_ms"] = e0.elapsed_time(e1)
            out[kind.replace("-", "_") + "_result"] = pr.get_coeffs("serial")
    out["soe_rel_diff"] = rel_err(out.pop("uniform_soe_result"), out.pop("uniform_result"))
    out["history_bytes"] = sum(s.K * 8 * s.nsteps * (s.nsteps - 1) / 2 for s in specs)
    print(json.dumps(out), flush=True)


def paper_model_case(args):
    """The paper's experiment on the GPU with its own spatial scheme (Sec.
    4.2): D = 1 + u, f = sin(pi x) e^{-t}, u0 = x^4 (1-x)^4, alpha = 0.5,
    Chebyshev-Lobatto collocation on 2^4 intervals, P = 2^8 slices of 2^5
    fine steps, FP64, parareal stopped at the paper's tolerance 1e-10.  The
    paper's speedup divides the sequential fine solver's time (the uniform
    scheme with the whole history) by parareal's; the sequential sweep S_hyb
    (parareal's limit) and the fast-history uniform solve are timed too.
    Times are device times (CUDA events) of the second of two solves."""
    import torch
    from paper_2510_11023_gb300 import psl1, workloads
    wl = workloads.e1_collocation()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"workload": wl.name, "precision": "fp64"}

    def timed(fn):
        fn()
        e0.record(stream)
        r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), r

    with psl1.Problem(wl, stream=stream.cuda_stream) as pr:
        for kind in ("uniform", "hybrid", "uniform-soe"):
            out[f"serial_{kind.replace('-', '_')}_ms"], _ = timed(lambda: pr.solve_serial(kind))
        S = pr.get_coeffs("serial")
        pr.solve_serial("hybrid")
        S = pr.get_coeffs("serial")
        pr.set_graph(True)
        out["parareal_ms"], k = timed(lambda: pr.solve_parareal(tol=1e-10))
        out["parareal_iterations"] = k
        out["parareal_rel_err_vs_serial_hybrid"] = rel_err(pr.get_coeffs("parareal"), S)
    out["speedup_vs_uniform_fine_solver"] = out["serial_uniform_ms"] / out["parareal_ms"]
    out["speedup_vs_serial_hybrid"] = out["serial_hybrid_ms"] / out["parareal_ms"]
    print(json.dumps(out), flush=True)


def assembly_case(args):
    """The stiffness assembly as a dense tensor-core contraction against the
    Toeplitz+Hankel moments the solver uses: 1024 units (sets of nodal D) of a
    K = 256, Q = 512 instance (the largest K of the batched workload), each
    method's kernel timed alone (CUDA events, second of two calls).  Work per
    unit: dense 2 K^2 Q FLOP (BF16 tensor cores); moments 2 Q (2K+1) + 3 K^2
    FLOP (FP32).  Both write the K x K FP32 matrix: K^2 4 bytes per unit."""
    import torch
    from paper_2510_11023_gb300 import psl1, workloads
    K, units = 256, 1024
    spec = workloads.InstanceSpec(modes=(K, 1), nsteps=64, alpha=0.5, dpar=workloads.D_CFG2, fpar=workloads.F_COS)
    rng = np.random.default_rng(3)
    D = 0.6 + rng.random((units, spec.Q))
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    bf16 = float(peaks.get("bf16_tflops", 1900.0))
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    _, fp32 = psl1.psl1_probe_peaks()
    out = {"workload": f"dense stiffness assembly, {units} units, K={K}, Q={spec.Q}"}
    with psl1.Problem([spec], 1, stream=torch.cuda.current_stream().cuda_stream) as pr:
        for method in ("tensor", "moments"):
            pr.assemble(0, D, method)
            _, ms = pr.assemble(0, D, method)
            flop = units * (2.0 * K * K * spec.Q if method == "tensor" else 2.0 * spec.Q * (2 * K + 1) + 3.0 * K * K)
            byts = units * (4.0 * K * K + 4.0 * spec.Q)
            tf = flop / (ms * 1e-3) / 1e12
            gbs = byts / (ms * 1e-3) / 1e9
            peak = bf16 if method == "tensor" else fp32
            out[method] = {"ms": ms, "tflops": tf, "frac_of_peak": tf / peak, "peak_tflops": peak,
                           "write_gbs": gbs, "frac_of_hbm": gbs / hbm}
    out["tensor_over_moments_time"] = out["tensor"]["ms"] / out["moments"]["ms"]
    out["peaks_source"] = "MEASURED_PEAKS.json bf16_tflops and hbm_gbs (burst); FP32 by psl1_probe_peaks"
    print(json.dumps(out), flush=True)


def learned_g_case(args):
    """The learned coarse propagator at its own size: an MLP (128 modal
    coefficients + 32 history features + alpha + t -> 128 modes, width 512, 4
    layers, BF16 weights, FP32 accumulation) trained on the 20,032 slice pairs
    of the sequential fine solutions of 313 instances (K = 128, N = 4096,
    P = 64, alpha ~ U[0.2, 1], seed 20251013), then parareal with the plain L1
    coarse propagator and with the learned one on 32 held-out instances (seed
    20251014): iterations and device wall time to rel. err 1e-8 against the
    FP64 sequential solution, at the fixed stopping rule (increment <= 1e-8).
    Mixed precision, host loop."""
    import torch
    from paper_2510_11023_gb300 import psl1, workloads
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"workload": "learned coarse propagator, K=128 N=4096 P=64, 313 training / 32 held-out instances"}
    t0 = time.perf_counter()
    tr = workloads.cfg4_trajectories(313, seed=20251013)
    mlp = psl1.MLP(128, 32, 512, 128, seed=1, stream=stream.cuda_stream)
    with psl1.Problem(tr, precision="mixed", stream=stream.cuda_stream) as data:
        data.solve_serial("hybrid")
        mlp.dataset(data, trajectories=True)
        log = mlp.train(data, epochs=args.train_epochs, batch=1024, lr=1e-3, seed=2)
    torch.cuda.synchronize()
    out["training"] = {"samples": 313 * 64, "epochs": args.train_epochs, "loss_first": float(log[0]),
                       "loss_last": float(log[-1]), "seconds": time.perf_counter() - t0}
    ho = workloads.cfg4_trajectories(32, seed=20251014)
    with psl1.Problem(ho, precision="fp64", stream=stream.cuda_stream) as ref:
        ref.solve_serial("hybrid")
        S = ref.get_coeffs("serial")
    d_u0 = torch.from_numpy(ho.u0_concat()).to("cuda")
    with psl1.Problem(ho, precision="mixed", stream=stream.cuda_stream) as pr:
        for name, m in (("l1", None), ("learned", mlp)):
            pr.set_coarse(m)
            for _ in range(2):
                pr.set_u0_dev(d_u0.data_ptr())
                e0.record(stream)
                pr.solve_parareal(tol=FIXED_TOL, allow_not_converged=True)
                e1.record(stream)
                torch.cuda.synchronize()
            out[name] = {"ms": e0.elapsed_time(e1), "iterations": int(pr.get_iterations().max()),
                         "rel_err": rel_err(pr.get_coeffs("parareal"), S)}
    mlp.close()
    out["learned_over_l1_time"] = out["learned"]["ms"] / out["l1"]["ms"]
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------- our arm
def main():
    args = parse()
    if args.impl == "reference":
        dist = Dist(args.gpus, "gloo")
        reference_arm(args, dist)
        dist.close()
        return
    import torch
    from paper_2510_11023_gb300 import psl1, workloads

    if args.workload == "uniform-history":
        psl1.load()
        uniform_history_case(args)
        return
    if args.workload == "paper-model":
        psl1.load()
        paper_model_case(args)
        return
    if args.workload == "assembly":
        psl1.load()
        assembly_case(args)
        return
    if args.workload == "learned-g":
        psl1.load()
        learned_g_case(args)
        return
    dist = Dist(args.gpus, "nccl")
    torch.cuda.set_device(dist.local)
    stream = torch.cuda.current_stream()
    psl1.load()
    fp64_tf, fp32_tf = psl1.psl1_probe_peaks()
    dmma_tf = psl1.psl1_probe_dmma()

    wl = make_workload(args, dist.rank)
    dim2 = wl.specs[0].dim == 2
    mmin = min(s.nsteps // wl.P for s in wl.specs)
    substeps = {"l1": 1, "l1x2": 2, "l1x4": 4, "l1x8": 8, "learned": 1}
    if args.coarse == "auto":
        coarse_list = [c for c in ("l1", "l1x2", "l1x4", "l1x8") if substeps[c] <= mmin]
        if not dim2:                 # the learned correction is defined for 1D instances
            coarse_list.append("learned")
    else:
        coarse_list = [args.coarse]
    u0 = wl.u0_concat()
    d_u0 = torch.from_numpy(u0).to("cuda")
    torch.cuda.synchronize()

    # plain serial FP64 GPU solve S_hyb: the reference solution and the baseline time
    ref = psl1.Problem(wl, precision="fp64" if args.reference == "fp64" else args.precision,
                       stream=stream.cuda_stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ref.solve_serial("hybrid")
    e1.record(stream)
    torch.cuda.synchronize()
    serial_fp64_ms = e0.elapsed_time(e1)
    S = ref.get_coeffs("serial")
    ref.close()

    pr = psl1.Problem(wl, precision=args.precision, stream=stream.cuda_stream)
    if dim2:
        pr.set_sweep_split(args.sweep_split)
    if args.precision != "fp64":
        e0.record(stream)
        pr.solve_serial("hybrid")
        e1.record(stream)
        torch.cuda.synchronize()
        serial_ms = e0.elapsed_time(e1)
    else:
        serial_ms = serial_fp64_ms
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2

    # autotuning of the F stage (inner CG tolerance per K bucket, persistent grid), off the clock
    pr.set_u0_dev(d_u0.data_ptr())
    import tempfile
    tune_cache = os.path.join(tempfile.gettempdir(), f"psl1_tune_{os.getpid()}.jsonl")
    t0 = time.perf_counter()
    from_cache = pr.autotune(tune_cache)
    tune_info = {"seconds": time.perf_counter() - t0, "from_cache": from_cache,
                 "choices": [json.loads(l) for l in open(tune_cache)] if os.path.exists(tune_cache) else []}

    # learned coarse correction, trained offline (not timed) on another seed of the
    # same instance distribution from the pairs parareal computes
    mlp, train_info = None, None
    if "learned" in coarse_list:
        t0 = time.perf_counter()
        twl = workloads.cfg2(B=args.train_batch, seed=args.seed + 7919 + dist.rank)
        with psl1.Problem(twl, precision=args.precision, stream=stream.cuda_stream) as data:
            mlp = psl1.MLP(128, 32, 512, 128, seed=1, stream=stream.cuda_stream)
            mlp.dataset(data, iterates=args.train_iters)
            log = mlp.train(data, epochs=args.train_epochs, batch=1024, lr=1e-3, seed=2)
        torch.cuda.synchronize()
        train_info = {"seconds": time.perf_counter() - t0, "instances": twl.B, "iterates": args.train_iters,
                      "epochs": args.train_epochs, "loss_first": float(log[0]), "loss_last": float(log[-1]),
                      "seed": args.seed + 7919}

    def configure(coarse, inexact):
        pr.set_coarse(None)
        pr.set_coarse_substeps(substeps[coarse])
        if coarse == "learned":
            pr.set_coarse(mlp)
        pr.set_inexact_fine(inexact)

    def timed_solve(tol_):
        pr.set_u0_dev(d_u0.data_ptr())
        e0.record(stream)
        pr.solve_parareal(tol=tol_, allow_not_converged=True)
        e1.record(stream)
        torch.cuda.synchronize()
        return {"tol": tol_, "ms": e0.elapsed_time(e1), "iterations": int(pr.get_iterations().max()),
                "rel_err": rel_err(pr.get_coeffs("parareal"), S)}

    last_ms = [0.0]

    def trial(coarse, inexact=0.0):
        """The solve at the fixed stopping rule with this configuration (after up to two
        warm-up solves; none once solves take seconds, where start-up costs vanish)."""
        configure(coarse, inexact)
        for _ in range(min(max(args.warmup - 1, 0), 2) if last_ms[0] < 5000.0 else 0):
            pr.set_u0_dev(d_u0.data_ptr())
            pr.solve_parareal(tol=FIXED_TOL, allow_not_converged=True)
        r = timed_solve(FIXED_TOL)
        last_ms[0] = r["ms"]
        r.update(coarse=coarse, inexact_above=inexact)
        return r

    # warm-up choice among configurations that reach the target error at the fixed rule:
    # every coarse propagator, each refined throughout and with inexact early iterations
    # (MIXED; the inexact iterations take the FP32 step in F and G)
    if args.precision == "mixed" and args.inexact != "off":
        inexact_list = ([] if args.inexact == "on" else [0.0]) + list(INEXACT_ABOVE)
    else:
        inexact_list = [0.0]
    cands = {f"{c}|{x:g}": trial(c, x) for c in coarse_list for x in inexact_list}
    ok = [k for k in cands if cands[k]["rel_err"] <= TARGET] or list(cands)
    best = cands[min(ok, key=lambda k: cands[k]["ms"])]
    coarse, inexact = best["coarse"], best["inexact_above"]
    # then looser refined steps while the increment is large (MIXED, with inexact iterations)
    refine = 0.0
    if inexact > 0.0:
        for fac in REFINE_FACTORS:
            pr.set_inexact_refinement(fac)
            c = trial(coarse, inexact)
            c["refine_factor"] = fac
            cands[f"{coarse}|{inexact:g}|refine={fac:g}"] = c
            if c["rel_err"] <= TARGET and c["ms"] < best["ms"]:
                best, refine = c, fac
        pr.set_inexact_refinement(refine)
    configure(coarse, inexact)

    # context only: the loosest increment tolerance that still reaches the target error,
    # found with the reference solution (information the method itself does not have)
    tol_t = 1.6e-7
    while True:
        pr.set_u0_dev(d_u0.data_ptr())
        pr.solve_parareal(tol=tol_t, allow_not_converged=True)
        if rel_err(pr.get_coeffs("parareal"), S) <= TARGET or tol_t < 1e-13:
            break
        tol_t /= 2.0
    tuned = timed_solve(tol_t)
    tol = FIXED_TOL

    # timed region: the solve runs as one CUDA graph (device-driven iteration loop)
    if not args.no_graph:
        pr.set_graph(True)
        pr.set_u0_dev(d_u0.data_ptr())
        pr.solve_parareal(tol=tol, allow_not_converged=True)   # builds the graph (untimed)
    dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(dist.local)
    clk.start()
    times, launches, iters_all = [], 0, []
    t_wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1.0)
        pr.set_u0_dev(d_u0.data_ptr())
        e0.record(stream)
        pr.solve_parareal(tol=tol, allow_not_converged=True)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        iters_all.append(int(pr.get_iterations().max()))
        launches += pr.stats()["kernel_launches"]
    torch.cuda.synchronize()
    dist.barrier()
    wall = time.perf_counter() - t_wall0
    clocks = clk.stop()
    err = rel_err(pr.get_coeffs("parareal"), S)

    # per-kernel device times for the roofline: the same solve once more through the
    # host loop, which records CUDA events around each F-stage and sweep launch
    pr.set_graph(False)
    flush.fill_(1.0)
    pr.set_u0_dev(d_u0.data_ptr())
    pr.solve_parareal(tol=tol, allow_not_converged=True)
    torch.cuda.synchronize()
    st = pr.stats()
    fine_ms, coarse_ms, flops_impl = st["ms_fine"], st["ms_coarse"], st["flop_fine"]
    iters_host = pr.get_iterations()
    solve_ms_events = fine_ms + coarse_ms
    if not args.no_graph:
        pr.set_graph(True)

    ms_step = dist.max(float(np.mean(times)))
    useful = float(sum(s.nsteps * s.K for s in wl.specs))
    value = dist.sum(useful) / (ms_step * 1e-3)

    # end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        h_out = np.zeros(int(pr.offU[-1]))
        et = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            pr.set_u0(u0)
            pr.solve_parareal(tol=tol, allow_not_converged=True)
            pr.L.psl1_get_coeffs(pr.h, 0, h_out.ctypes.data_as(psl1._D))
            et.append(time.perf_counter() - t0)
        e_ms = dist.max(1e3 * float(np.mean(et)))
        e2e = {"value": dist.sum(useful) / (e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": int(u0.nbytes),
               "d2h_bytes_per_step": int(h_out.nbytes)}

    # context: the uniform-history serial solve S_uni (the paper-style sequential L1
    # solver, full fine history) in the same precision, and its discretisation gap
    # to S_hyb (parareal's limit); the first call tunes the history stream and
    # captures the step graph, the second is timed
    uniform = None
    if not args.no_uniform:
        pr.solve_serial("uniform")
        flush.fill_(1.0)
        e0.record(stream)
        pr.solve_serial("uniform")
        e1.record(stream)
        torch.cuda.synchronize()
        uniform = {"ms": e0.elapsed_time(e1), "precision": args.precision,
                   "rel_gap_to_serial_hybrid": rel_err(pr.get_coeffs("serial"), S)}
        Wex = pr.get_coeffs("serial")
        # the same scheme with the fast (sum-of-exponentials) history
        pr.solve_serial("uniform-soe")
        flush.fill_(1.0)
        e0.record(stream)
        pr.solve_serial("uniform-soe")
        e1.record(stream)
        torch.cuda.synchronize()
        uniform["fast_history"] = {"ms": e0.elapsed_time(e1),
                                   "rel_diff_to_exact_history": rel_err(pr.get_coeffs("serial"), Wex)}

    # roofline of the dominant kernel (F stage).  1D: the algorithmic count of the
    # step (alg_flops_step_1d) times the fine steps each launch processes; the
    # library's own device counter of the work it did is kept beside it.  2D: the
    # device counter (matrix-free operator applications, the algorithm in use).
    fine_launches = int(iters_host.max())
    fine_avg_ms = fine_ms / max(fine_launches, 1)
    achieved_impl = flops_impl / max(fine_launches, 1) / (fine_avg_ms * 1e-3) / 1e12
    peak = fp64_tf if args.precision == "fp64" else fp32_tf
    if dim2:
        achieved, count = achieved_impl, "device counter of the implemented operator applications"
    else:
        alg, _ = fstage_alg_flops(wl, iters_host)
        achieved = alg / max(fine_launches, 1) / (fine_avg_ms * 1e-3) / 1e12
        count = ("4QK + 2Q(2K+1) + K^3/3 + 2K^2 per fine step (transforms, Toeplitz+Hankel moments, "
                 "direct-solve count) x the fine steps of each launch")
    # the refine factor is left out of the key: it moves the F stage's DRAM bytes by a few percent
    traffic_key = f"{args.workload}|B={wl.B}|{args.precision}|{coarse}|inexact={inexact:g}"
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "frac_impl": achieved_impl / peak, "traffic": captured_traffic(traffic_key),
            "traffic_config": traffic_key, "kernel": "k_fstage",
            "launches": fine_launches, "ms_per_launch": fine_avg_ms,
            "share_of_solve": {"k_fstage": fine_ms / max(solve_ms_events, 1e-9),
                               "k_coarse_sweep": coarse_ms / max(solve_ms_events, 1e-9)},
            "flops_source": count,
            "peak_source": ("measured FP64 FMA throughput (psl1_probe_peaks)" if args.precision == "fp64"
                            else "measured FP32 FMA throughput (psl1_probe_peaks)")}

    cpu = None
    if not args.no_cpu and dist.rank == 0 and dist.world == 1:
        v, dt, ninst, thr = oracle_throughput(wl, S, args.cpu_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": thr, "kind": "oracle", "host_cpus": os.cpu_count(),
               "sample": f"FP64 oracle (OpenMP build) fine propagators F_n, n = P/2 .. P/2+{thr - 1}, one per "
                         f"host thread, of the first {ninst} instances ({dt:.1f} s timed, history from the GPU "
                         f"serial solve)"}
        if dim2:
            cpu["sample"] = (f"FP64 oracle: {ninst} L1 steps of the instance with half the modes per axis "
                             f"({dt:.1f} s), scaled by the oracle's K^2 Q cost to the full size, 1 thread")

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
            "data": "synthetic",
            "config": {"workload": wl.name, "batch": wl.B, "P": wl.P, "precision": args.precision,
                       "stop_rule": f"increment e_k <= {FIXED_TOL:g} (the target error, fixed in advance)",
                       "l2": "flushed (256 MB write) before every timed step",
                       "seed": wl.meta.get("seed", args.seed),
                       "execution": "host loop" if args.no_graph else "one CUDA graph per solve (device-driven loop)"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
            "rel_err_vs_serial_fp64": err, "stop_tol": tol, "iterations": iters_all,
            "tuned_tolerance": tuned, "autotune": tune_info,
            "coarse_propagator": coarse, "inexact_early_iterations": {"above": inexact, "refine_factor": refine},
            "sweep_split_ctas": pr.sweep_split(),
            "configurations_tried": cands, "learned_training": train_info,
            "serial_fp64_ms": serial_fp64_ms, "serial_ms": serial_ms, "serial_uniform": uniform,
            "speedup_vs_serial_fp64": serial_fp64_ms / ms_step, "speedup_vs_serial_same_precision": serial_ms / ms_step,
            "measured_peaks_tflops": {"fp64": fp64_tf, "fp32": fp32_tf, "fp64_tensor": dmma_tf,
                                      "source": "psl1_probe_peaks (FMA chains), psl1_probe_dmma (mma.sync f64)"},
            "wall_s": wall}
    if dist.rank == 0:
        print(json.dumps(line), flush=True)
    pr.close()
    if mlp is not None:
        mlp.close()
    dist.close()


if __name__ == "__main__":
    main()
