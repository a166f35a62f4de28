#!/usr/bin/env python3
"""Throughput of the phaseless-AFQMC walker step on B300 (walker-steps/s).

Workload: the 108-orbital system with 21 alpha + 21 beta electrons, naux = 432
Cholesky vectors (spectrum decaying as exp(-gamma/40)), RHF trial, 640
walkers, dt = 0.005.  One step = the mixed local energy at the current walkers
+ one propagation step of every walker; QR every 5 steps and the comb every 10
steps, amortised.  Synthetic seeded inputs (the paper's molecular integrals are
not available).

Prints one JSON line.  --impl reference times the FP64 CPU oracle instead.
Under torchrun each rank runs an independent replica (different seed); the
value is the walker-steps of all ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "walker-steps/s at ≤0.1 mHa vs FP64 plain form; % tensor/HBM roofline"
UNIT = "walker-steps/s"
WORKLOAD = dict(norb=108, nalpha=21, nbeta=21, naux=432, tau=40.0, nwalkers=640, dt=0.005,
                energy_every=1, reortho_every=5, comb_every=10)
L2_BYTES = 126 * 2 ** 20
DTYPE = {"fp64": "f64", "fp32": "f32", "bf16": "bf16", "bf16x3": "bf16x3"}
# nominal per-GPU FP64 rate (recipe table); FP32 CUDA-core peak from 148 SMs x 128 lanes x 2 x 2032 MHz
FP64_PEAK_TFLOPS = 1.25
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12


def workload_name():
    w = WORKLOAD
    return (f"ph-AFQMC step N={w['norb']} {w['nalpha']}a+{w['nbeta']}b naux={w['naux']} RHF "
            f"W={w['nwalkers']} dt={w['dt']} (E every step, QR/5, comb/10)")


def make_problem():
    from synthetic_inputs import config_medium
    return config_medium()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------------------------------
def exchange_flops_per_walker(norb, ncol, naux, smul_blocks=1):
    """T^g = Ltilde^g Theta (real [n,N] x complex [N,n]) for every gamma: 2 real GEMMs."""
    return 2 * 2 * ncol * norb * ncol * naux * smul_blocks


def step_flops_per_walker(norb, ncol, naux, taylor=6):
    """Algorithmic FLOPs of one walker-step with the energy (restricted: one spin block propagated)."""
    exch = exchange_flops_per_walker(norb, ncol, naux)
    vhs = 2 * 2 * naux * norb * norb
    prop = 2 * (2 * 2 * norb * norb * ncol) + taylor * 8 * norb * norb * ncol
    ovl = 2 * (8 * norb * ncol * ncol)
    return dict(exchange=exch, vhs=vhs, propagate=prop, overlap=ovl, total=exch + vhs + prop + ovl)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


def source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2406_16238_b300", "csrc")
    for name in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_from_profiles(prec):
    """DRAM bytes per launch of the dominant kernel from a committed ncu summary, if the kernel is unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        data = json.load(f)
    ent = data.get(prec)
    if not ent or ent.get("source_hash") != source_hash():
        return None
    return ent.get("dram_bytes_per_launch")


# ------------------------------------------------------------------------------------------
def accuracy_vs_fp64(prob, prec, seed, nw, nsteps=10):
    """max |E_prec - E_fp64| (Ha) per step over a horizon with identical fields, no comb."""
    import paper_2406_16238_b300 as pkg
    if prec == "fp64":
        return 0.0
    e = {}
    for p in ("fp64", prec):
        ctx = pkg.Afqmc(prob.h1e, prob.chol, prob.ecore, prob.nalpha, prob.nbeta, prob.psiT, nwalkers=nw,
                        dt=WORKLOAD["dt"], seed=seed, prec=p)
        e[p] = ctx.run(nsteps, 1, WORKLOAD["reortho_every"], 0)
        ctx.close()
    return float(np.max(np.abs(e[prec][:, 0] / e[prec][:, 1] - e["fp64"][:, 0] / e["fp64"][:, 1])))


def cpu_baseline(prob, seed, budget_s=15.0):
    """The FP64 oracle as it stands, timed on a bounded sample of the workload on the host cores."""
    from oracle import afqmc as orc
    try:
        from threadpoolctl import threadpool_info
        cores = max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count()
    st = orc.build_setup(prob.h1e, prob.chol, prob.ecore, prob.nalpha, prob.nbeta, prob.psiT, WORKLOAD["dt"])
    nw = 16
    wk = orc.init_walkers(st, prob.psiT, nw)
    t0 = time.perf_counter()
    steps = 0
    while True:
        orc.energy_sums(st, wk)
        orc.phaseless_step(st, wk, seed, st.evar)
        steps += 1
        if wk.step % WORKLOAD["reortho_every"] == 0:
            orc.reorthogonalise(st, wk)
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": nw * steps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{nw} walkers x {steps} steps of the same workload (energy + step, QR/5), "
                      f"{dt:.1f} s on the host"}


# ------------------------------------------------------------------------------------------
def run_ours(args):
    import torch
    import paper_2406_16238_b300 as pkg

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    prob = make_problem()
    nw = WORKLOAD["nwalkers"]
    seed = 240616238 + 1000 * rank
    acc = accuracy_vs_fp64(prob, args.prec, seed, 64) if rank == 0 and not args.skip_extras else None

    stream = torch.cuda.current_stream(dev)
    ctx = pkg.Afqmc(prob.h1e, prob.chol, prob.ecore, prob.nalpha, prob.nbeta, prob.psiT, nwalkers=nw,
                    dt=WORKLOAD["dt"], seed=seed, prec=args.prec, device=dev, stream=stream)
    info = ctx.info()
    ncol = prob.nalpha if info["restricted"] else prob.nalpha + prob.nbeta
    ws_bytes = info["workspace_bytes"]
    ctx.run(args.warmup, WORKLOAD["energy_every"], WORKLOAD["reortho_every"], WORKLOAD["comb_every"])
    torch.cuda.synchronize(dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    per_step_flush = ws_bytes < 2 * L2_BYTES
    if world > 1:
        torch.distributed.barrier()
    ctx.profile(True)
    l0 = ctx.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step_ms = []
    with ClockSampler(dev.index) as clk:
        torch.cuda.synchronize(dev)
        if per_step_flush:
            for _ in range(args.steps):
                flush.zero_()
                ev0.record(stream)
                ctx.run(1, WORKLOAD["energy_every"], WORKLOAD["reortho_every"], WORKLOAD["comb_every"])
                ev1.record(stream)
                ev1.synchronize()
                step_ms.append(ev0.elapsed_time(ev1))
            total_ms = sum(step_ms)
        else:
            ev0.record(stream)
            ctx.run(args.steps, WORKLOAD["energy_every"], WORKLOAD["reortho_every"], WORKLOAD["comb_every"])
            ev1.record(stream)
            ev1.synchronize()
            total_ms = ev0.elapsed_time(ev1)
        torch.cuda.synchronize(dev)
    launches = ctx.launch_count() - l0
    stages = ctx.stage_times()
    ctx.profile(False)
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * nw * args.steps / (total_ms / 1e3)

    if args.skip_extras:
        ctx.close()
        return None if rank != 0 else {"value": value, "ms_per_step": total_ms / args.steps,
                                       "stages_ms_per_step": {k: v[0] / args.steps for k, v in stages.items()}}
    # end to end through the public API from pinned host buffers: create (H2D of h1e, L, psiT)
    # + the same steps with the energy sums read back to the host every step
    h1e_p = torch.from_numpy(prob.h1e).pin_memory().numpy()
    chol_p = torch.from_numpy(prob.chol).pin_memory().numpy()
    psiT_p = torch.from_numpy(prob.psiT).pin_memory().numpy()
    ctx.close()
    del ctx
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    ctx2 = pkg.Afqmc(h1e_p, chol_p, prob.ecore, prob.nalpha, prob.nbeta, psiT_p, nwalkers=nw, dt=WORKLOAD["dt"],
                     seed=seed + 1, prec=args.prec, device=dev, stream=stream)
    for s in range(args.steps):
        ctx2.local_energy()
        ctx2.propagate(1)
        if (s + 1) % WORKLOAD["reortho_every"] == 0:
            ctx2.reortho()
        if (s + 1) % WORKLOAD["comb_every"] == 0:
            ctx2.popcontrol()
    ctx2.synchronize(600.0)
    e2e_s = time.perf_counter() - t0
    ctx2.close()
    h2d = prob.h1e.nbytes + prob.chol.nbytes + prob.psiT.nbytes
    if world > 1:
        t = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_s = float(t.item())

    if rank != 0:
        return None
    peaks, peak_src = measured_peaks()
    fl = step_flops_per_walker(prob.norb, ncol, prob.naux)
    exch_ms, exch_n = stages["exchange"]
    exch_flops_launch = exchange_flops_per_walker(prob.norb, ncol, prob.naux) * nw
    achieved = exch_flops_launch / (exch_ms / exch_n / 1e3) / 1e12 if exch_n else None
    if args.prec == "fp64":
        bound, peak, unit, peak_note = "alu", FP64_PEAK_TFLOPS, "TFLOP/s", "nominal FP64 (recipe table)"
    elif args.prec == "fp32":
        bound, peak, unit, peak_note = "alu", FP32_PEAK_TFLOPS, "TFLOP/s", "FP32 CUDA-core: 148 SM x 128 x 2 x 2.032 GHz"
    else:
        scale = 1.0 if args.prec == "bf16" else 1.0 / 3.0
        bound, peak, unit = "tensor", peaks["bf16_tflops_sustained"] * scale, "TFLOP/s"
        peak_note = f"bf16 sustained ({peak_src})" + (" / 3 products" if scale < 1 else "")
    traffic = traffic_from_profiles(args.prec)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE[args.prec], "data": "synthetic",
        "config": {"workload": workload_name(), "form": args.prec, "norb": prob.norb, "nalpha": prob.nalpha,
                   "nbeta": prob.nbeta, "naux": prob.naux, "walkers_per_gpu": nw, "dt": WORKLOAD["dt"],
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": ("L2 flushed before every timed step" if per_step_flush else
                          f"inputs larger than L2 (workspace {ws_bytes / 2**20:.0f} MiB > 2 x L2)"),
                   "max_abs_dE_vs_fp64_Ha_10steps": acc,
                   "meets_0.1mHa": None if acc is None else bool(acc <= 1e-4)},
        "roofline": {"kernel": "exchange (T = Ltilde Theta, fused Tr T and Tr T T)", "bound": bound,
                     "achieved": achieved, "peak": peak, "unit": unit, "peak_source": peak_note,
                     "frac": achieved / peak if achieved else None, "traffic": traffic,
                     "algorithmic_flops_per_launch": exch_flops_launch},
        "stages_ms_per_step": {k: v[0] / args.steps for k, v in stages.items()},
        "step_flops_per_walker": fl,
        "clocks": clk.summary(),
        "gpu_launches": int(launches),
        "e2e": {"value": world * nw * args.steps / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": 32,
                "note": "create from pinned host arrays + steps with the 4 energy sums read back every step"},
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(prob, seed, args.cpu_budget)
    return line


def run_reference(args):
    """The oracle arm: the FP64 CPU oracle on the same workload, a bounded walker sample per step."""
    rank, world, _ = dist_env()
    if rank != 0:
        return None
    from oracle import afqmc as orc
    prob = make_problem()
    st = orc.build_setup(prob.h1e, prob.chol, prob.ecore, prob.nalpha, prob.nbeta, prob.psiT, WORKLOAD["dt"])
    nw = args.ref_walkers
    wk = orc.init_walkers(st, prob.psiT, nw)
    seed = 240616238

    def one():
        orc.energy_sums(st, wk)
        orc.phaseless_step(st, wk, seed, st.evar)
        if wk.step % WORKLOAD["reortho_every"] == 0:
            orc.reorthogonalise(st, wk)
        if wk.step % WORKLOAD["comb_every"] == 0:
            orc.population_control(wk, seed)

    for _ in range(args.warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    dt = time.perf_counter() - t0
    value = nw * args.steps / dt
    cores = os.cpu_count()
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(), "form": "fp64 CPU oracle", "walkers_per_step_sample": nw},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{nw} of {WORKLOAD['nwalkers']} walkers per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="bf16x3", choices=["fp64", "fp32", "bf16", "bf16x3"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-walkers", type=int, default=8)
    ap.add_argument("--skip-extras", action="store_true",
                    help="time the steps only (no accuracy check, e2e or CPU baseline), e.g. under ncu")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    line = run_reference(args) if args.impl == "reference" else run_ours(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
