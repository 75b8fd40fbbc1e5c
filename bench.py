#!/usr/bin/env python
"""Throughput benchmark of the form-factor hot path on B300.

One step = one full form-factor job on device-resident inputs: pair-prep
(Gaussian product theorem + coefficient folding), per-axis phase tables and
the q-evaluation over the whole product grid for every state, with the |f|^2
epilogue.  Metric: (q-point x state)/s.

Default workload: the 10-heavy-atom molecule (10 heavy + 10 H, double-zeta +
d basis, 170 Cartesian functions), 12 states, 128^3 grid on [-20, 20]
Bohr^-1, evaluated with the split-BF16 tensor-core path; the plain FP64 GPU
path is timed beside it.

Usage: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Under torchrun each rank evaluates its own job (weak scaling, no data-path
collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2512_18010_b300 import workloads as W  # noqa: E402

METRIC = "form-factor (q-point×state)/s and p50/p99 job latency vs plain FP64 GPU path"
UNIT = "(q-point*state)/s"
FP32_LANES_PER_SM = 128
N_SM = 148
SM_MAX_MHZ = 2032.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="scff", choices=["scff", "reference"])
    ap.add_argument("--workload", default="cfg3", choices=["cfg1", "cfg2", "cfg3"])
    ap.add_argument("--precision", default="tf32x3", choices=["tf32x3", "bf16x3", "bf16x2", "fp32", "fp64"])
    ap.add_argument("--fp64-steps", type=int, default=1, help="timed steps of the plain FP64 path (0 = skip)")
    ap.add_argument("--cpu-sample", type=int, default=2048, help="q points of the oracle CPU baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def workload(name: str, rank: int = 0):
    if name == "cfg1":
        job = W.config1(1000 + rank)
    elif name == "cfg2":
        job = W.config2(2000 + rank)
    else:
        job = W.config3(3000 + rank)
    desc = {
        "cfg1": "cfg1: 1 heavy + 2 H, 13 functions, 1 state, 16^3 on [-10,10]",
        "cfg2": "cfg2: benzene-scale ring, 66 functions, 12 states, 64^3 on [-15,15]",
        "cfg3": "cfg3: 10 heavy + 10 H, 170 functions (double-zeta + d), 12 states, 128^3 on [-20,20]",
    }[name]
    return job, desc


def pair_stats(mol):
    """Pair records and monomial rows of a basis (for the algorithmic flop count)."""
    per_heavy = {0: 1, 1: 3, 2: 6, -1: 4}
    lmax = {0: 0, 1: 1, 2: 2, -1: 1}
    recs = []
    for l, n in zip(mol.shell_l, mol.shell_nprim):
        recs += [lmax[int(l)]] * int(n)
    recs = np.array(recs)
    L = recs[:, None] + recs[None, :]
    iu = np.triu_indices(len(recs))
    Lp = L[iu]
    K = int(np.sum((Lp + 1) * (Lp + 2) * (Lp + 3) // 6))
    del per_heavy
    return len(Lp), K


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(job, n_points: int, seed: int = 99):
    import oracle
    idx = W.subset_indices(job.nq, n_points, seed)
    t0 = time.perf_counter()
    oracle.grid_form_factor(job, idx)
    dt = time.perf_counter() - t0
    return {"value": len(idx) * job.n_states / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{len(idx)} seeded q points of the same job, all {job.n_states} states, "
                      f"FP64 C oracle with OpenMP ({dt:.1f} s)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    job, desc = workload(args.workload)
    import oracle
    n_pts = {"cfg1": 4096, "cfg2": 1024, "cfg3": 256}[args.workload]
    idx_all = [W.subset_indices(job.nq, n_pts, 500 + k) for k in range(args.warmup + args.steps)]
    for k in range(args.warmup):
        oracle.grid_form_factor(job, idx_all[k])
    times = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        oracle.grid_form_factor(job, idx_all[args.warmup + k])
        times.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.mean(times))
    value = n_pts * job.n_states / (ms / 1e3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "sample_per_step": f"{n_pts} seeded q points x {job.n_states} states"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{n_pts} q points per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2512_18010_b300 import scff

    job, desc = workload(args.workload, rank)
    S, nq = job.n_states, job.nq
    prec = scff.PRECISIONS[args.precision]
    ctx = scff.Context(local)
    b = ctx.basis(job.mol)
    t = ctx.transitions(b, job.T)
    g = ctx.qgrid_product(job.qx, job.qy, job.qz)
    tdt = torch.float64 if prec == scff.FP64 else torch.float32
    dev = torch.device("cuda", local)
    f = torch.empty((S, nq, 2), dtype=tdt, device=dev)
    f2 = torch.empty((S, nq), dtype=tdt, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        ctx.form_factor(b, t, g, precision=prec, f_out=f, f2_out=f2, stream=stream)

    ctx.set_timing(True)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ctx.sync(stream)

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    l0 = ctx.kernel_launches()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    step_ms, qeval_ms = [], []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.fill_(float(k))  # L2 flush between timed steps (outside the events)
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
        qeval_ms.append(ctx.last_timing()[0])
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = ctx.kernel_launches() - l0
    clocks = sampler.stop()
    ctx.sync(stream)
    step_ms = [a.elapsed_time(bb) for a, bb in ev]
    ms = float(np.mean(step_ms))
    if dist:
        tt = torch.tensor([ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    units = S * nq
    value = world * units / (ms / 1e3)

    # plain FP64 GPU path on the same job
    fp64 = None
    if args.fp64_steps > 0 and prec != scff.FP64:
        f64 = torch.empty((S, nq, 2), dtype=torch.float64, device=dev)
        ctx.form_factor(b, t, g, precision=scff.FP64, f_out=f64, stream=stream)  # warm-up
        torch.cuda.synchronize()
        tms = []
        for _ in range(args.fp64_steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.form_factor(b, t, g, precision=scff.FP64, f_out=f64, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            tms.append(e0.elapsed_time(e1))
        fms = float(np.mean(tms))
        fp64 = {"value": units / (fms / 1e3), "unit": UNIT, "ms_per_step": fms, "steps": args.fp64_steps}
        del f64

    # roofline of the dominant kernel (the q-evaluation)
    n_pair, K = pair_stats(job.mol)
    flops_per_unit = 2 * K + 8 * n_pair
    kern_ms = float(np.mean(qeval_ms))
    achieved = flops_per_unit * units / (kern_ms / 1e3) / 1e12
    if prec in (scff.BF16X3, scff.TF32X3, scff.BF16X2):
        peak_src = "measured bf16 dense (MEASURED_PEAKS.json bf16_tflops)"
        try:
            peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"]
        except Exception:
            peak, peak_src = 1800.0, "fallback bf16 1.8 PFLOP/s"
        roof = {"bound": "tensor", "kernel": "tc_form_factor", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                "work": f"{flops_per_unit} algorithmic flop per (q*state)", "peak_source": peak_src}
    else:
        peak = N_SM * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
        if prec == scff.FP64:
            peak = 1.25
        roof = {"bound": "alu", "kernel": "direct_kernel", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "work": f"{flops_per_unit} algorithmic flop per (q*state)",
                "peak_source": "FP32: 148 SM x 128 lanes x 2 flop x 2032 MHz" if prec != scff.FP64
                else "FP64 nominal 1.25 TFLOP/s"}

    # end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        rdt = np.float64 if prec == scff.FP64 else np.float32
        hf = torch.empty((S, nq, 2), dtype=tdt, pin_memory=True)
        hf2 = torch.empty((S, nq), dtype=tdt, pin_memory=True)
        hT = torch.from_numpy(np.ascontiguousarray(job.T)).pin_memory()
        fview = hf.numpy()
        f2view = hf2.numpy()
        tlist = []
        for k in range(max(2, args.steps) + 1):
            t0 = time.perf_counter()
            bb = ctx.basis(job.mol)
            tt = ctx.transitions(bb, hT.numpy())
            gg = ctx.qgrid_product(job.qx, job.qy, job.qz)
            ctx.form_factor(bb, tt, gg, precision=prec, f_out=fview, f2_out=f2view)
            ctx.release(gg)
            ctx.release(bb)
            if k > 0:
                tlist.append(time.perf_counter() - t0)
        e2e_s = float(np.mean(tlist))
        h2d = job.T.nbytes + 8 * (len(job.qx) + len(job.qy) + len(job.qz)) + job.mol.xyz.nbytes + \
            job.mol.exponents.nbytes + job.mol.coefficients.nbytes + 12 * job.mol.n_shells
        d2h = S * nq * (2 + 1) * np.dtype(rdt).itemsize
        e2e = {"value": world * units / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * e2e_s}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(job, args.cpu_sample)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": {"tf32x3": "tf32x3->f32", "bf16x3": "bf16x3->f32", "bf16x2": "bf16x2->f32", "fp32": "f32", "fp64": "f64"}[args.precision],
                "data": "synthetic (seeded molecules, basis and transition matrices)",
                "config": {"workload": desc, "precision": args.precision, "n_pairs": n_pair,
                           "monomial_rows": K, "l2": "flushed between timed steps (256 MB write)",
                           "parallelism": f"dp{world} (one job per rank)"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
                "fp64_gpu_path": fp64, "clocks": clocks,
                "step_ms": step_ms, "qeval_ms": qeval_ms}
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
