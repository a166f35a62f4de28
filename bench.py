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


class _CtypesNvml:
    """The few NVML calls the clock sampler makes, through ctypes on the driver's libnvidia-ml (for
    images without the pynvml module).  Names and return values follow pynvml's."""

    NVML_CLOCK_SM = 1

    def __init__(self):
        import ctypes
        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")

    def _ok(self, rc, what):
        if rc != 0:
            raise RuntimeError(f"{what} failed ({rc})")

    def nvmlInit(self):
        self._ok(self.lib.nvmlInit_v2(), "nvmlInit_v2")

    def nvmlDeviceGetHandleByPciBusId(self, bus):
        h = self.ct.c_void_p()
        self._ok(self.lib.nvmlDeviceGetHandleByPciBusId_v2(self.ct.c_char_p(bus), self.ct.byref(h)),
                 "nvmlDeviceGetHandleByPciBusId_v2")
        return h

    def nvmlDeviceGetHandleByIndex(self, i):
        h = self.ct.c_void_p()
        self._ok(self.lib.nvmlDeviceGetHandleByIndex_v2(self.ct.c_uint(i), self.ct.byref(h)),
                 "nvmlDeviceGetHandleByIndex_v2")
        return h

    def _uint(self, fn, *args):
        v = self.ct.c_uint()
        self._ok(getattr(self.lib, fn)(*args, self.ct.byref(v)), fn)
        return v.value

    def nvmlDeviceGetClockInfo(self, h, clk):
        return self._uint("nvmlDeviceGetClockInfo", h, self.ct.c_int(clk))

    def nvmlDeviceGetMaxClockInfo(self, h, clk):
        return self._uint("nvmlDeviceGetMaxClockInfo", h, self.ct.c_int(clk))

    def nvmlDeviceGetPowerUsage(self, h):
        return self._uint("nvmlDeviceGetPowerUsage", h)

    def nvmlDeviceGetCurrentClocksEventReasons(self, h):
        v = self.ct.c_ulonglong()
        self._ok(self.lib.nvmlDeviceGetCurrentClocksThrottleReasons(h, self.ct.byref(v)),
                 "nvmlDeviceGetCurrentClocksThrottleReasons")
        return v.value


class ClockSampler:
    """SM clock, its maximum, power and clock-event (throttle) reasons, polled through NVML every
    ~2 ms in a background thread (nvidia-smi's 200 ms loop sees nothing of a 10 ms timed region).
    mark_start()/mark_end() bracket the timed region; summary() reports the samples inside it (and,
    separately, every sample of the run).  Falls back to nvidia-smi when NVML is unavailable."""

    REASONS = {"hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40,
               "sw_power_cap": 0x4}

    def __init__(self, device):
        self.device = device
        self.samples = []          # (t, sm_mhz, max_mhz, power_w, reasons bitmask)
        self.t0 = self.t1 = None
        self._stop = threading.Event()
        self.thread = None
        self.nvml = None

    def _handle(self):
        try:
            import pynvml
        except ImportError:
            pynvml = _CtypesNvml()
        import torch
        pynvml.nvmlInit()
        self.nvml = pynvml
        try:
            props = torch.cuda.get_device_properties(self.device)
            bus = f"{props.pci_domain_id:08x}:{props.pci_bus_id:02x}:{props.pci_device_id:02x}.0"
            return pynvml.nvmlDeviceGetHandleByPciBusId(bus.encode())
        except Exception:
            return pynvml.nvmlDeviceGetHandleByIndex(self.device.index or 0)

    def _poll(self, h):
        nv = self.nvml
        mx = nv.nvmlDeviceGetMaxClockInfo(h, nv.NVML_CLOCK_SM)
        while not self._stop.is_set():
            try:
                sm = nv.nvmlDeviceGetClockInfo(h, nv.NVML_CLOCK_SM)
                rs = nv.nvmlDeviceGetCurrentClocksEventReasons(h)
                pw = nv.nvmlDeviceGetPowerUsage(h) / 1000.0
                self.samples.append((time.perf_counter(), float(sm), float(mx), pw, int(rs)))
            except Exception:
                break
            time.sleep(0.002)

    SMI_FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                  "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                  "clocks_event_reasons.sw_power_cap")

    def _smi(self):
        """Fallback: nvidia-smi's own loop at 10 ms, each line stamped on arrival."""
        import torch
        bits = [self.REASONS[k] for k in ("hw_slowdown", "sw_thermal_slowdown", "hw_thermal_slowdown",
                                          "sw_power_cap")]
        try:
            props = torch.cuda.get_device_properties(self.device)
            sel = f"{props.pci_domain_id:08x}:{props.pci_bus_id:02x}:{props.pci_device_id:02x}.0"
        except Exception:   # noqa: BLE001
            sel = str(self.device.index or 0)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", sel, f"--query-gpu={self.SMI_FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "10"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError as e:
            self.error = (self.error or "") + f"; nvidia-smi: {e}"
            return
        for ln in self.proc.stdout:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                rs = sum(b for b, v in zip(bits, parts[3:7]) if v.lower() == "active")
                self.samples.append((time.perf_counter(), float(parts[0]), float(parts[1]), float(parts[2]), rs))
            except ValueError:
                continue
            if self._stop.is_set():
                break

    def __enter__(self):
        self.error = None
        self.proc = None
        self.mode = "NVML, polled every ~2 ms"
        try:
            h = self._handle()
            self.thread = threading.Thread(target=self._poll, args=(h,), daemon=True)
        except Exception as e:   # noqa: BLE001  (reported in the summary)
            self.error = f"NVML: {type(e).__name__}: {e}"
            self.mode = "nvidia-smi -lms 10"
            self.thread = threading.Thread(target=self._smi, daemon=True)
        self.thread.start()
        return self

    def mark_start(self):
        self.t0 = time.perf_counter()

    def mark_end(self):
        self.t1 = time.perf_counter()

    def __exit__(self, *a):
        self._stop.set()
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    @staticmethod
    def _summarise(rows):
        sm = [r[1] for r in rows]
        reasons = set()
        for r in rows:
            for nm, bit in ClockSampler.REASONS.items():
                if r[4] & bit:
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": rows[-1][2] if rows else None,
                "power_w_max": max(r[3] for r in rows) if rows else None, "reasons": sorted(reasons),
                "samples": len(rows)}

    def summary(self):
        rows = self.samples
        inside = [r for r in rows if self.t0 is not None and self.t1 is not None and self.t0 <= r[0] <= self.t1]
        out = self._summarise(inside)
        out["source"] = self.mode + " during the timed region" + (f" ({self.error})" if self.error else "")
        out["whole_run"] = self._summarise(rows)
        return out


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


def traffic_from_profiles(prec, stage):
    """DRAM bytes per launch of a stage's main kernel from the committed ncu summary, if the source is unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        data = json.load(f)
    ent = data.get(f"{prec}:{stage}")
    if not ent or ent.get("source_hash") != source_hash():
        return None
    return ent.get("dram_bytes_per_launch")


def fp64_gemm_tflops(dev, n=4096, reps=5):
    """Binary64 rate measured on this GPU: a cuBLAS DGEMM (n x n x n) timed with CUDA events."""
    import torch
    a = torch.randn(n, n, dtype=torch.float64, device=dev)
    b = torch.randn(n, n, dtype=torch.float64, device=dev)
    c = a @ b
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        c = a @ b
    e1.record()
    e1.synchronize()
    del a, b, c
    return 2.0 * n ** 3 * reps / (e0.elapsed_time(e1) / 1e3) / 1e12


def stage_rooflines(prec, norb, ncol, naux, nw, stages, fp64_peak=None):
    """Algorithmic work per launch of the main stages against the peak of the unit that bounds them."""
    peaks, src = measured_peaks()
    tensor = prec in ("bf16", "bf16x3")
    # the stage times come from a short pass (~20 steps, ~10 ms of GPU time) of direct launches: the
    # burst bf16 rate is the matching peak (the sustained one applies to a seconds-long loop)
    tpeak = peaks["bf16_tflops"] * (1.0 if prec == "bf16" else 1.0 / 3.0)
    tnote = f"bf16 burst ({src})" + ("" if prec == "bf16" else " / 3 products")
    alu = (fp64_peak or FP64_PEAK_TFLOPS) if prec == "fp64" else FP32_PEAK_TFLOPS
    anote = (("binary64 rate measured on this GPU (cuBLAS DGEMM 4096^3)" if fp64_peak else "nominal FP64 (recipe table)")
             if prec == "fp64" else "FP32 CUDA cores: 148 SM x 128 x 2 x 2.032 GHz")
    fl = step_flops_per_walker(norb, ncol, naux)
    n = ncol
    lu_fp64 = 8 * n ** 3 / 3                            # LU with partial pivoting, complex (binary64)
    work = {
        "exchange": (fl["exchange"] * nw, "tensor" if tensor else "alu", tpeak if tensor else alu,
                     tnote if tensor else anote),
        "propagate": (fl["propagate"] * nw, "tensor" if tensor else "alu", tpeak if tensor else alu,
                      tnote if tensor else anote),
        "vhs": (fl["vhs"] * nw, "tensor" if tensor else "alu", tpeak if tensor else alu, tnote if tensor else anote),
        "overlap": (lu_fp64 * nw, "alu", fp64_peak or FP64_PEAK_TFLOPS,
                    ("binary64 rate measured on this GPU (cuBLAS DGEMM 4096^3)" if fp64_peak else
                     "nominal FP64 (recipe table)") + "; binary64 LU work only"),
    }
    out = {}
    for k, (flops, bound, peak, note) in work.items():
        ms, cnt = stages.get(k, (0.0, 0))
        if not cnt:
            continue
        per = ms / cnt
        ach = flops / (per / 1e3) / 1e12
        out[k] = {"bound": bound, "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                  "peak_source": note, "algorithmic_flops_per_launch": flops, "ms_per_launch": per,
                  "launches_per_step": cnt / max(1, stages.get("_steps", (1, 1))[0]),
                  "traffic": traffic_from_profiles(prec, k)}   # DRAM bytes per launch (ncu), while unchanged
    return out


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
    clk = ClockSampler(dev).__enter__()
    ctx.run(args.warmup, WORKLOAD["energy_every"], WORKLOAD["reortho_every"], WORKLOAD["comb_every"])
    torch.cuda.synchronize(dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    per_step_flush = ws_bytes < 2 * L2_BYTES
    if world > 1:
        torch.distributed.barrier()
    l0 = ctx.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step_ms, sums_timed = [], []
    torch.cuda.synchronize(dev)
    clk.mark_start()
    if per_step_flush:
        for _ in range(args.steps):
            flush.zero_()
            ev0.record(stream)
            sums_timed.append(ctx.run(1, WORKLOAD["energy_every"], WORKLOAD["reortho_every"],
                                      WORKLOAD["comb_every"]))
            ev1.record(stream)
            ev1.synchronize()
            step_ms.append(ev0.elapsed_time(ev1))
        total_ms = sum(step_ms)
    else:
        ev0.record(stream)
        sums_timed.append(ctx.run(args.steps, WORKLOAD["energy_every"], WORKLOAD["reortho_every"],
                                  WORKLOAD["comb_every"]))
        ev1.record(stream)
        ev1.synchronize()
        total_ms = ev0.elapsed_time(ev1)
    torch.cuda.synchronize(dev)
    clk.mark_end()
    launches = ctx.launch_count() - l0
    # stage times from a separate pass with per-stage events (direct launches, no graph replay)
    nprof = min(args.steps, 20)
    ctx.profile(True)
    ctx.run(nprof, WORKLOAD["energy_every"], WORKLOAD["reortho_every"], WORKLOAD["comb_every"])
    torch.cuda.synchronize(dev)
    stages = ctx.stage_times()
    stages["_steps"] = (nprof, 1)
    ctx.profile(False)
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * nw * args.steps / (total_ms / 1e3)

    if args.skip_extras:
        clk.__exit__(None, None, None)
        ctx.close()
        return None if rank != 0 else {"value": value, "ms_per_step": total_ms / args.steps,
                                       "stages_ms_per_step": {k: v[0] / nprof for k, v in stages.items()
                                                              if not k.startswith("_")}}
    fp64_form = None
    if rank == 0 and args.prec != "fp64":   # the plain FP64 form on the same workload (context for the ratio)
        c64 = pkg.Afqmc(prob.h1e, prob.chol, prob.ecore, prob.nalpha, prob.nbeta, prob.psiT, nwalkers=nw,
                        dt=WORKLOAD["dt"], seed=seed, prec="fp64", device=dev, stream=stream)
        c64.run(3, 1, 5, 10)
        torch.cuda.synchronize(dev)
        ev0.record(stream)
        c64.run(5, 1, 5, 10)
        ev1.record(stream)
        ev1.synchronize()
        ms64 = ev0.elapsed_time(ev1) / 5
        fp64_form = {"value": nw / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64, "steps": 5}
        c64.close()
        del c64
    free_proj = None
    if rank == 0:   # free projection (unshifted fields, complex weights, no comb) on the same workload
        cfp = pkg.Afqmc(prob.h1e, prob.chol, prob.ecore, prob.nalpha, prob.nbeta, prob.psiT, nwalkers=nw,
                        dt=WORKLOAD["dt"], seed=seed, prec=args.prec, device=dev, stream=stream)
        cfp.set_free_projection(True)
        cfp.run(3, 1, WORKLOAD["reortho_every"], 0)
        torch.cuda.synchronize(dev)
        ev0.record(stream)
        efp = cfp.run(10, 1, WORKLOAD["reortho_every"], 0)
        ev1.record(stream)
        ev1.synchronize()
        msfp = ev0.elapsed_time(ev1) / 10
        if not np.all(np.isfinite(efp)):
            raise RuntimeError("free projection: non-finite estimator sums")
        free_proj = {"value": nw / (msfp / 1e3), "unit": UNIT, "ms_per_step": msfp, "steps": 10,
                     "form": args.prec, "note": "energy every step, QR every 5, no comb (Section "
                     "\"Free projection AFQMC\")"}
        cfp.close()
        del cfp
    # end to end through the public API from pinned host buffers: create (H2D of h1e, L, psiT)
    # + the same steps with each step's energy sums copied to pinned host memory (stream-ordered,
    # asynchronous), the host waiting once at the end
    h1e_p = torch.from_numpy(prob.h1e).pin_memory().numpy()
    chol_p = torch.from_numpy(prob.chol).pin_memory().numpy()
    psiT_p = torch.from_numpy(prob.psiT).pin_memory().numpy()
    ctx.close()
    del ctx
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    ctx2 = pkg.Afqmc(h1e_p, chol_p, prob.ecore, prob.nalpha, prob.nbeta, psiT_p, nwalkers=nw, dt=WORKLOAD["dt"],
                     seed=seed + 1, prec=args.prec, device=dev, stream=stream)
    t1 = time.perf_counter()
    sums_host = torch.zeros(4 * args.steps, dtype=torch.float64).pin_memory().numpy()
    # first step alone (captures the step graphs on first use), then the remaining steps
    ctx2.run_async(1, sums_host[:4], WORKLOAD["energy_every"], WORKLOAD["reortho_every"], WORKLOAD["comb_every"])
    ctx2.synchronize(600.0)
    t2 = time.perf_counter()
    if args.steps > 1:
        ctx2.run_async(args.steps - 1, sums_host[4:], WORKLOAD["energy_every"], WORKLOAD["reortho_every"],
                       WORKLOAD["comb_every"])
    ctx2.synchronize(600.0)
    t3 = time.perf_counter()
    e2e_s = t3 - t0
    e2e_split = {"create_ms": 1e3 * (t1 - t0), "first_step_ms": 1e3 * (t2 - t1),
                 "steady_value": (world * nw * (args.steps - 1) / (t3 - t2)) if args.steps > 1 else None}
    if not np.all(np.isfinite(sums_host)) or not np.all(sums_host[1::4] > 0):
        raise RuntimeError("end-to-end run: non-finite energy sums or a zero weight total")
    ctx2.close()
    clk.__exit__(None, None, None)
    clocks = clk.summary()
    h2d = prob.h1e.nbytes + prob.chol.nbytes + prob.psiT.nbytes
    if world > 1:
        t = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_s = float(t.item())

    if rank != 0:
        return None
    fl = step_flops_per_walker(prob.norb, ncol, prob.naux)
    # error bar per second (reblocked mixed-energy series of the timed steps, first 20 % dropped):
    # eta = 1 / (sigma_E^2 t_wall)
    from paper_2406_16238_b300.analysis import energy_series, error_bar
    e_timed = energy_series(np.concatenate(sums_timed))
    e_kept = e_timed[len(e_timed) // 5:]
    eb = error_bar(e_kept) if len(e_kept) >= 16 else float("nan")
    eta = {"mean_energy_Ha": float(e_kept.mean()) if len(e_kept) else None,
           "error_bar_Ha": eb if np.isfinite(eb) else None,
           "eta_per_Ha2_s": (1.0 / (eb * eb * total_ms / 1e3)) if np.isfinite(eb) and eb > 0 else None,
           "note": f"{len(e_kept)} of {len(e_timed)} timed steps' energies (first 20 % dropped), "
                   "Flyvbjerg-Petersen reblocking; t_wall = the timed region"}
    rooflines = stage_rooflines(args.prec, prob.norb, ncol, prob.naux, nw, stages, fp64_peak=fp64_gemm_tflops(dev))
    dominant = max(rooflines, key=lambda k: rooflines[k]["ms_per_launch"] * rooflines[k]["launches_per_step"])
    roof = dict(rooflines[dominant])
    roof["kernel"] = dominant
    roof["traffic"] = traffic_from_profiles(args.prec, dominant)
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
        "roofline": roof,
        "rooflines": rooflines,
        "stages_ms_per_step": {k: v[0] / nprof for k, v in stages.items() if not k.startswith("_")},
        "stages_note": f"per-stage CUDA events over {nprof} separately run steps (direct launches); "
                       "value and ms_per_step come from the graph-replayed timed region",
        "step_flops_per_walker": fl,
        "error_bar_per_second": eta,
        "fp64_form": fp64_form,
        "free_projection": free_proj,
        "clocks": clocks,
        "gpu_launches": int(launches),
        "e2e": {"value": world * nw * args.steps / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": 32,
                "create_ms": e2e_split["create_ms"], "first_step_ms": e2e_split["first_step_ms"],
                "steady_value": e2e_split["steady_value"],
                "note": "create from pinned host arrays (workspace allocation, H2D of h1e, L and psiT, device "
                        "set-up) + afqmc_run_async (graph-replayed steps, the step graphs captured during the first "
                        "step, each step's 4 energy sums copied to pinned host memory by an asynchronous "
                        "stream-ordered copy), checked finite after the final synchronisation; steady_value = the "
                        "steps after the first, from the host's clock"},
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(prob, seed, args.cpu_budget)
    if not args.no_large and world == 1:
        line["large_system"] = run_large(args, dev, stream)
    if not args.no_batched and world == 1:
        bargs = argparse.Namespace(**vars(args))
        bargs.steps, bargs.warmup = 20, 3
        b = run_batched(bargs)
        line["batched"] = {k: b[k] for k in ("value", "unit", "ms_per_step", "steps", "warmup", "config", "clocks",
                                             "gpu_launches", "roofline", "rooflines", "stage_ms_per_step",
                                             "graphs_form", "energies_finite") if k in b}
    return line


def batched_rooflines(prec, systems, stages, steps):
    """Work per grouped launch (sums over the systems) of the grouped stages against the tensor peak."""
    peaks, src = measured_peaks()
    tpeak = peaks["bf16_tflops"] * (1.0 if prec == "bf16" else 1.0 / 3.0)
    tnote = f"bf16 burst ({src})" + ("" if prec == "bf16" else " / 3 products")
    work = {"exchange": 0.0, "vhs": 0.0, "propagate": 0.0}
    for norb, ncol, naux, nw in systems:
        fl = step_flops_per_walker(norb, ncol, naux)
        for k in work:
            work[k] += fl[k] * nw
    out = {}
    for k, flops in work.items():
        ms, cnt = stages.get(k, (0.0, 0))
        if not cnt:
            continue
        # the propagation stage is one small-form launch plus, for N > 128, one launch per product
        per = ms / steps
        ach = flops / (per / 1e3) / 1e12
        out[k] = {"bound": "tensor", "achieved": ach, "peak": tpeak, "unit": "TFLOP/s", "frac": ach / tpeak,
                  "peak_source": tnote, "algorithmic_flops_per_step": flops, "ms_per_step": per,
                  "launches_per_step": cnt / steps, "traffic": None}
    return out


def run_batched(args):
    """32 uneven systems (N ~ U[50, 300], n = N/6, naux = 4N), 256 walkers each, split-bf16 GEMMs
    with fp32 accumulation, autotuned per system, one CUDA graph launch per step: in the grouped form
    every stage is one launch over the work of all systems (the per-system graphs form is timed beside
    it on the same systems)."""
    import torch
    import paper_2406_16238_b300 as pkg
    from paper_2406_16238_b300._lib import Batch
    from synthetic_inputs import config_batched
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    probs = config_batched(nsys=args.nsys)
    ctxs, tunings, sizes, shapes = [], [], [], []
    for i, p in enumerate(probs):
        c = pkg.Afqmc(p.h1e, p.chol, p.ecore, p.nalpha, p.nbeta, p.psiT, nwalkers=256, dt=WORKLOAD["dt"],
                      seed=240616238 + i, prec=args.prec, device=dev, stream=stream)
        tunings.append(c.autotune(steps=2))
        ctxs.append(c)
        sizes.append(p.norb)
        info = c.info()
        shapes.append((p.norb, info["nalpha"] if info["restricted"] else info["nalpha"] + info["nbeta"], info["naux"],
                       256))
        p.chol = None
    b = Batch(ctxs, mode=args.batch_mode)
    form = b.mode()

    def timed(nsteps):
        torch.cuda.synchronize(dev)
        l0 = sum(c.launch_count() for c in ctxs)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(dev) as clk:
            torch.cuda.synchronize(dev)
            clk.mark_start()
            ev0.record(stream)
            e = b.run(nsteps, 1, 5, 10)
            ev1.record(stream)
            ev1.synchronize()
            clk.mark_end()
        return ev0.elapsed_time(ev1), e, sum(c.launch_count() for c in ctxs) - l0, clk.summary()

    b.run(args.warmup, 1, 5, 10)
    ms, e, launches, clocks = timed(args.steps)
    total_ws = len(ctxs) * 256 * args.steps
    extra = {}
    if form == "grouped":
        # stage trace of the grouped launches (direct launches between CUDA events)
        b.profile(True)
        nprof = 10
        b.run(nprof, 1, 5, 10)
        st = b.stage_times()
        b.profile(False)
        rl = batched_rooflines(args.prec, shapes, st, nprof)
        extra["rooflines"] = rl
        if "exchange" in rl:
            r = dict(rl["exchange"])
            r["kernel"] = "k_tc_gemm<0, 0, true> (grouped exchange over every system's tiles)"
            extra["roofline"] = r
        extra["stage_ms_per_step"] = {k: v[0] / nprof for k, v in st.items() if v[1]}
        # the per-system graphs form on the same systems, for comparison
        b.set_mode("graphs")
        b.run(2, 1, 5, 10)
        gms, _, gl, _ = timed(args.steps)
        extra["graphs_form"] = {"value": total_ws / (gms / 1e3), "ms_per_step": gms / args.steps,
                                "gpu_launches": int(gl)}
    return {"metric": METRIC, "value": total_ws / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE[args.prec], "data": "synthetic",
            "config": {"workload": f"batched uneven systems: {len(ctxs)} x (N in [50,300], n=N/6, naux=4N, W=256), "
                                   "one CUDA graph launch per step", "form": args.prec, "batch_form": form,
                       "norb": sizes, "tuning": tunings, "l2": "inputs larger than L2"},
            "energies_finite": bool(np.isfinite(e).all()), "clocks": clocks, "gpu_launches": int(launches), **extra}


def run_cv(args):
    """N=300, 25a+25b, naux=1500, 2048 walkers: learned control variate vs the plain form."""
    import torch
    import paper_2406_16238_b300 as pkg
    from paper_2406_16238_b300.analysis import energy_series, error_bar
    from synthetic_inputs import config_cv
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    prob = config_cv()
    nw = 2048
    ctx = pkg.Afqmc(prob.h1e, prob.chol, prob.ecore, prob.nalpha, prob.nbeta, prob.psiT, nwalkers=nw,
                    dt=WORKLOAD["dt"], seed=240616243, prec=args.prec, device=dev, stream=stream)
    ctx.cv_attach(capacity=args.cv_pairs, batch=1024, sample_frac=0.125, seed=7)
    t0 = time.perf_counter()
    npairs = ctx.cv_collect((args.cv_pairs + nw - 1) // nw, 5, 10)
    losses = ctx.cv_train(args.cv_epochs, lr=1e-3)
    t_train = time.perf_counter() - t0
    psi, logo, w, step = ctx.get_walkers()
    out = {}
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for form in ("plain", "cv"):
        ctx.set_walkers(psi, w, step)
        ctx.cv_enable(form == "cv")
        ctx.run(args.warmup, 1, 5, 10)
        ev0.record(stream)
        sums = ctx.run(args.steps, 1, 5, 10)
        ev1.record(stream)
        ev1.synchronize()
        ms = ev0.elapsed_time(ev1)
        e = energy_series(sums)
        eb = error_bar(e[len(e) // 5:])
        t = ms / 1e3
        out[form] = {"walker_steps_per_s": nw * args.steps / t, "ms_per_step": ms / args.steps,
                     "mean_energy": float(e[len(e) // 5:].mean()), "error_bar": eb,
                     "error_bar_per_second": 1.0 / (eb * eb * t) if eb > 0 else None}
    ctx.cv_enable(False)
    return {"metric": METRIC, "value": out["cv"]["walker_steps_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": out["cv"]["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.prec],
            "data": "synthetic",
            "config": {"workload": "learned control variate: N=300 25a+25b naux=1500 W=2048 dt=0.005, exact exchange "
                                   "on 1/8 of the walkers per step", "form": args.prec, "training_pairs": npairs,
                       "epochs": args.cv_epochs, "final_loss": float(losses[-1]) if len(losses) else None,
                       "collect_and_train_s": t_train},
            "forms": out}


def large_rooflines(prec, norb, nblocks, nocc, naux, nw, stages):
    """Rooflines of the large system's stages: the exchange and the propagation against the tensor
    peak, the VHS build against HBM bandwidth (its bytes are L's bf16 copy, read once per step)."""
    peaks, src = measured_peaks()
    tpeak = peaks["bf16_tflops"] * (1.0 if prec == "bf16" else 1.0 / 3.0)
    tnote = f"bf16 burst ({src})" + ("" if prec == "bf16" else " / 3 products")
    parts = 1 if prec == "bf16" else 2
    kx = (naux + 63) // 64 * 64
    ncol = nblocks * nocc
    exch = nblocks * exchange_flops_per_walker(norb, nocc, naux) * nw
    prop = (2 * (2 * 2 * norb * norb * ncol) + 6 * 8 * norb * norb * ncol) * nw
    # L^T holds the packed upper triangle (N (N + 1) / 2 rows) where N > 128; the V planes are written whole
    rows = norb * (norb + 1) // 2 if norb > 128 else norb * norb
    vhs_bytes = parts * rows * kx * 2 + nw * 2 * parts * kx * 2 + nw * 4 * norb * norb * 2
    work = {"exchange": (exch, "tensor", tpeak, "TFLOP/s", 1e12, tnote),
            "propagate": (prop, "tensor", tpeak, "TFLOP/s", 1e12, tnote),
            "vhs": (vhs_bytes, "hbm", peaks["hbm_gbs"], "GB/s", 1e9,
                    f"HBM copy bandwidth ({src}); bytes = packed L^T bf16 {'hi + lo' if parts == 2 else 'hi'} read "
                    "once, coefficients, V planes written")}
    out = {}
    for k, (amount, bound, peak, unit, scale, note) in work.items():
        ms, cnt = stages.get(k, (0.0, 0))
        if not cnt:
            continue
        per = ms / cnt
        ach = amount / (per / 1e3) / scale
        out[k] = {"bound": bound, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
                  "peak_source": note, ("algorithmic_flops_per_launch" if bound == "tensor" else
                                        "algorithmic_bytes_per_launch"): amount,
                  "ms_per_launch": per, "traffic": None}
    return out


def run_large(args, dev=None, stream=None, steps=10, warmup=2):
    """The large system: N=1512, 42a+42b, naux=7560, UHF trial, 128 walkers; L drawn on the GPU in
    binary32 chunks of 120 vectors and passed through the chunked set-up (never on the host)."""
    import torch
    import paper_2406_16238_b300 as pkg
    from synthetic_inputs import config_large
    dev = dev or torch.device("cuda", 0)
    stream = stream or torch.cuda.current_stream(dev)
    prob = config_large(naux=getattr(args, "large_naux", None) or 7560)
    nw = 128
    prec = "bf16" if args.prec == "bf16" else "bf16x3"
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    ctx = pkg.Afqmc(prob.h1e, prob.chunks(120, device=dev), prob.ecore, prob.nalpha, prob.nbeta, prob.psiT,
                    nwalkers=nw, dt=WORKLOAD["dt"], seed=240616241, prec=prec, naux=prob.naux, device=dev,
                    stream=stream)
    create_s = time.perf_counter() - t0
    ws = ctx.info()["workspace_bytes"]
    ctx.run(warmup, 1, WORKLOAD["reortho_every"], WORKLOAD["comb_every"])
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = ctx.launch_count()
    ev0.record(stream)
    e = ctx.run(steps, 1, WORKLOAD["reortho_every"], WORKLOAD["comb_every"])
    ev1.record(stream)
    ev1.synchronize()
    ms = ev0.elapsed_time(ev1)
    launches = ctx.launch_count() - l0
    if not np.all(np.isfinite(e)):
        raise RuntimeError("large system: non-finite estimator sums")
    ctx.profile(True)
    ctx.run(3, 1, WORKLOAD["reortho_every"], WORKLOAD["comb_every"])
    torch.cuda.synchronize(dev)
    stages = ctx.stage_times()
    ctx.profile(False)
    ctx.close()
    del ctx
    roof = large_rooflines(prec, prob.norb, 2, prob.nalpha, prob.naux, nw, stages)
    return {"value": nw * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps, "steps": steps,
            "warmup": warmup, "form": prec, "dtype": DTYPE[prec], "gpu_launches": int(launches),
            "workload": f"large single system N=1512 42a+42b naux={prob.naux} (tau=756) UHF W=128 dt=0.005 (E every "
                        "step, QR/5, comb/10); L drawn on the GPU, binary32 chunks",
            "create_s": create_s, "workspace_GiB": ws / 2 ** 30,
            "l2": "inputs larger than L2 (L^T bf16 copy of tens of GB)",
            "mean_energy_Ha": float(np.mean(e[:, 0] / e[:, 1])),
            "stages_ms_per_step": {k: v[0] / 3 for k, v in stages.items()},
            "rooflines": roof}


REF_BUDGET_S = 150.0


def run_reference(args):
    """The oracle arm: the FP64 CPU oracle on the same workload, a bounded walker sample per step."""
    rank, world, _ = dist_env()
    if rank != 0:
        return None
    from oracle import afqmc as orc
    prob = make_problem()
    st = orc.build_setup(prob.h1e, prob.chol, prob.ecore, prob.nalpha, prob.nbeta, prob.psiT, WORKLOAD["dt"])
    seed = 240616238
    # walker sample per step: at most --ref-walkers, fewer when --steps is large, so that the whole
    # run stays within about REF_BUDGET_S seconds (calibrated on one step of two walkers)
    cal = orc.init_walkers(st, prob.psiT, 2)
    t0 = time.perf_counter()
    orc.energy_sums(st, cal)
    orc.phaseless_step(st, cal, seed, st.evar)
    per_walker = (time.perf_counter() - t0) / 2
    nw = int(max(1, min(args.ref_walkers, REF_BUDGET_S / max(1e-9, per_walker * (args.steps + args.warmup)))))
    wk = orc.init_walkers(st, prob.psiT, nw)

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
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 2000 for the medium workload, 50 for batched and cv)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="bf16x3", choices=["fp64", "fp32", "bf16", "bf16x3"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-walkers", type=int, default=8)
    ap.add_argument("--workload", default="medium", choices=["medium", "batched", "cv", "large"])
    ap.add_argument("--no-large", action="store_true", help="leave the large-system measurement out of the line")
    ap.add_argument("--large-naux", type=int, default=None,
                    help="the large system truncated to its first naux Cholesky vectors (a small case for ncu)")
    ap.add_argument("--nsys", type=int, default=32)
    ap.add_argument("--no-batched", action="store_true", help="leave the uneven-batch measurement out of the line")
    ap.add_argument("--batch-mode", default="auto", choices=["auto", "grouped", "graphs"],
                    help="batched workload: one launch per stage over all systems, or per-system graphs")
    ap.add_argument("--cv-pairs", type=int, default=100000)
    ap.add_argument("--cv-epochs", type=int, default=30)
    ap.add_argument("--skip-extras", action="store_true",
                    help="time the steps only (no accuracy check, e2e or CPU baseline), e.g. under ncu")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = (2000 if args.workload == "medium" and args.impl == "ours" else
                      10 if args.workload == "large" else 50)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        line = run_reference(args)
    elif args.workload == "batched":
        line = run_batched(args)
    elif args.workload == "cv":
        line = run_cv(args)
    elif args.workload == "large":
        r = run_large(args, steps=args.steps, warmup=args.warmup)
        roof = max(r["rooflines"].values(), key=lambda v: v["ms_per_launch"]) if r["rooflines"] else None
        line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": 1, "steps": r["steps"],
                "warmup": r["warmup"], "ms_per_step": r["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": r["dtype"], "data": "synthetic",
                "config": {"workload": r["workload"], "form": r["form"], "l2": r["l2"]},
                "roofline": roof, "rooflines": r["rooflines"], "gpu_launches": r["gpu_launches"],
                "stages_ms_per_step": r["stages_ms_per_step"], "create_s": r["create_s"]}
    else:
        line = run_ours(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
