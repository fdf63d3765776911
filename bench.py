#!/usr/bin/env python3
"""Throughput benchmark of the lattice leapfrog (one JSON line on rank 0).

Workload (default): 3D 256^3 periodic lattice, 2 fields phi, chi with
V = phi^4/4 + (q/2) phi^2 chi^2, q = 1.2, L = 20, dt = 0.02, expansion on,
seeded Gaussian-random-field initial conditions (paper_0712_0813_gb300.icgen),
fields and velocities in FP32 with FP64 global sums and scale factor.
A "step" is one leapfrog step of the whole lattice (drift, Laplacian, model
force, kick, global sums, scale-factor update).

Metric: Gsite-updates/s = sites * steps / seconds / 1e9 (one site update
advances all fields at one site by one step).  The state (537 MB) is larger
than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (serial FP64 C, test infrastructure) on
the host cores, each step on a bounded sub-lattice of the same model.
Multi-GPU: replicas only (independent lattices per rank, no data-path
collective); launched with torchrun, rank 0 prints the aggregate.
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
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

def _courant(N, q):
    from paper_0712_0813_gb300.icgen import courant_dt
    return courant_dt(3, N, 20.0, 1.0, q)


# 256cube is the default (the bench line); the others are the large-lattice configurations.
WORKLOADS = {
    "256cube": dict(name="3d_256cube_2field_expanding", dims=3, N=256, L=20.0, dt=0.02, nf=2,
                    q=(1.2,), expansion=True, phi0=1.0, seed=1, steps=5000),
    "1024cube": dict(name="3d_1024cube_2field_expanding", dims=3, N=1024, L=20.0, dt=None, nf=2,
                     q=(1.2,), expansion=True, phi0=1.0, seed=1, steps=2000),
    "512cube_4field": dict(name="3d_512cube_4field_expanding", dims=3, N=512, L=20.0, dt=None, nf=4,
                           q=(0.8, 5.0, 40.0), expansion=True, phi0=1.0, seed=1, steps=1000),
}
WORKLOAD = WORKLOADS["256cube"]
METRIC = "Gsite-updates/s"
STEP_SOURCES = {"k_step_sweep": ("ce_sweep3d.cuh", "ce_sweep3d_f32.cu", "ce_tma.cuh", "ce_device.cuh", "ce_internal.h"),
                "k_step_generic": ("ce_generic.cu", "ce_device.cuh", "ce_internal.h")}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash(kernel_name: str) -> str:
    h = hashlib.sha1()
    for name in STEP_SOURCES[kernel_name]:
        with open(os.path.join(ROOT, "paper_0712_0813_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def ncu_traffic(kernel_name: str, precision: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source (same hash); else None."""
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.md")
    if not os.path.exists(path):
        return None
    pat = re.compile(rf"^traffic\s+{re.escape(kernel_name)}\s+{precision}\s+src=(\w+)\s+bytes_per_launch=(\d+)")
    cur = kernel_source_hash(kernel_name)
    with open(path) as fh:
        for line in fh:
            m = pat.match(line.strip())
            if m and m.group(1) == cur:
                return int(m.group(2))
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        self.out = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.out = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        if not self.out:
            return None
        sm, smax, reasons = [], 0.0, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.out:
            parts = [p.strip() for p in ln.split(",")]
            try:
                sm.append(float(parts[0]))
                smax = max(smax, float(parts[1]))
            except (ValueError, IndexError):
                continue
            for n, p in zip(names, parts[3:]):
                if p.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def make_inputs(rank: int):
    from paper_0712_0813_gb300.icgen import lattice_ics
    w = WORKLOAD
    big = w["N"] ** w["dims"] >= 1 << 24
    from paper_0712_0813_gb300.replicas import replica_seed
    return lattice_ics(w["dims"], w["N"], w["L"], w["nf"], phi0=w["phi0"], q=w["q"],
                       seed=replica_seed(w["seed"], rank), backend="torch" if big else "numpy")


def sim_config(precision: str, stream, hints=None):
    w = WORKLOAD
    cfg = dict(dims=w["dims"], N=w["N"], L=w["L"], dt=w["dt"], nfields=w["nf"], q=w["q"],
               expansion=w["expansion"], phi0=w["phi0"], precision=precision, stream=stream)
    cfg.update(hints or {})
    return cfg


def time_device_steps(capi, torch, f0, u0, precision, steps, warmup, barrier, sampler_gpu=None, hints=None):
    """Device-resident timing: CUDA events on the library's stream around `steps` launches."""
    stream = torch.cuda.Stream()
    sim = capi.Simulation(**sim_config(precision, stream.cuda_stream, hints))
    sim.set_fields(f0, u0)
    sim.step(warmup)
    sim.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    clocks = None
    barrier()
    torch.cuda.synchronize()
    if sampler_gpu is not None:
        cs = ClockSampler(sampler_gpu)
        cs.__enter__()
        time.sleep(0.25)
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    if sampler_gpu is not None:
        cs.__exit__(None, None, None)
        clocks = cs.summary()
    barrier()
    sim.synchronize()  # surfaces any latched device error
    ms = e0.elapsed_time(e1)
    kernel = {1: "generic", 2: "sweep", 3: "rows"}[sim.kernel]
    plan = sim.sweep_plan
    sim.close()
    return ms, kernel, clocks, plan


def time_e2e(capi, torch, f0, u0, precision, steps, hints=None):
    """End to end through the public API with pinned host buffers: upload of the
    initial state, start-up, `steps` steps, download of the final state."""
    nf, S = f0.shape
    pin_f = torch.empty(nf * S, dtype=torch.float64, pin_memory=True).numpy()
    pin_u = torch.empty(nf * S, dtype=torch.float64, pin_memory=True).numpy()
    out_f, out_v = pin_f, pin_u          # the inputs are consumed by set_fields: reuse them for the outputs
    pin_f[:] = f0.reshape(-1)
    pin_u[:] = u0.reshape(-1)
    stream = torch.cuda.Stream()
    sim = capi.Simulation(**sim_config(precision, stream.cuda_stream, hints))
    sim.set_fields(pin_f, pin_u)  # warm (first-touch, module load)
    torch.cuda.synchronize()
    pin_f[:] = f0.reshape(-1)
    pin_u[:] = u0.reshape(-1)
    t0 = time.perf_counter()
    sim.set_fields(pin_f, pin_u)
    sim.step(steps)
    capi.ce_get_fields(sim.handle, nf, S, capi.CE_VEL_SYNC, out=(out_f, out_v))
    t1 = time.perf_counter()
    sim.close()
    nbytes = 2 * nf * S * 8
    return t1 - t0, nbytes


def batched_leg(capi, torch, steps: int, warmup: int, seq_steps: int, hbm_peak: float):
    """Mixed-size workload (96 lattices of 1D/2D/3D): the batched FP32 persistent
    kernel against the same lattices stepped one by one with the plain FP64 path
    and with the plain FP32 path (device-resident, CUDA events)."""
    from paper_0712_0813_gb300 import workloads as W
    specs = W.mixed_batch_specs()
    ics = [W.make_ics(sp) for sp in specs]
    total = sum(W.sites(sp) for sp in specs)
    stream = torch.cuda.Stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    sims = []
    for sp, (f0, u0) in zip(specs, ics):
        sim = capi.Simulation(**W.sim_kwargs(sp, "f32"), kernel="generic")
        sim.set_fields(f0, u0)
        sims.append(sim)
    from paper_0712_0813_gb300 import autotune
    tune = autotune.autotune_batch(sims, stream=stream)   # outside the timed region
    b = capi.Batch(sims, sweep_len=tune["sweep_len"], stream=stream.cuda_stream, ctas_per_sm=tune["ctas_per_sm"])
    info = b.info
    b.step(warmup)
    b.synchronize()
    torch.cuda.synchronize()
    e0.record(stream)
    b.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    b.synchronize()
    b.close()
    for sim in sims:
        sim.close()
    batched = total * steps / (ms / 1e3) / 1e9

    def sequential(precision: str, nsteps: int):
        t_ms, site_steps = 0.0, 0
        for sp, (f0, u0) in zip(specs, ics):
            with capi.Simulation(**W.sim_kwargs(sp, precision), stream=stream.cuda_stream) as sim:
                sim.set_fields(f0, u0)
                sim.step(3)
                sim.synchronize()
                e0.record(stream)
                sim.step(nsteps)
                e1.record(stream)
                e1.synchronize()
                t_ms += e0.elapsed_time(e1)
                site_steps += W.sites(sp) * nsteps
        return site_steps / (t_ms / 1e3) / 1e9

    fp64_seq = sequential("f64", seq_steps)
    f32_seq = sequential("f32", seq_steps)
    alg = 16 * 2 * total
    achieved = alg / (ms / 1e3 / steps) / 1e9
    return {"workload": "96 lattices: 32 x 1D 65536, 32 x 2D 1024^2, 32 x 3D side in {64..192}; 2 fields, "
                        "per-lattice q, phi0, Courant dt, expansion on half",
            "sites": total, "steps": steps, "ms_per_step": ms / steps, "items": info["items"],
            "sweep_len": tune["sweep_len"], "ctas_per_sm": tune["ctas_per_sm"], "autotune": tune["table"],
            "blocks": info["blocks"], "value_f32_batched": batched, "fp64_plain_sequential": fp64_seq,
            "f32_plain_sequential": f32_seq, "batched_over_fp64_plain": batched / fp64_seq,
            "sequential_steps": seq_steps,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "kernel": "k_step_batched",
                         "algorithmic_bytes_per_launch": alg}}


def cpu_oracle_rate(f0, u0, target_s: float, N_sample: int | None = None):
    """Sites/s of the CPU oracle (serial, 1 thread) on the bench model."""
    import oracle
    from paper_0712_0813_gb300.icgen import lattice_ics
    w = WORKLOAD
    if N_sample is None or N_sample == w["N"]:
        N = w["N"]
        fs, us = f0, u0
    else:
        N = N_sample
        fs, us = lattice_ics(w["dims"], N, w["L"], w["nf"], phi0=w["phi0"], q=w["q"], seed=w["seed"])
    p = oracle.Params(dims=w["dims"], N=N, L=w["L"], dt=w["dt"], nf=w["nf"], q=w["q"], expansion=w["expansion"])
    st = oracle.init(p, fs, us)
    t0 = time.perf_counter()
    oracle.step(st, 1)
    one = time.perf_counter() - t0
    k = max(1, int(target_s / max(one, 1e-6)) - 1)
    t0 = time.perf_counter()
    oracle.step(st, k)
    el = time.perf_counter() - t0
    return (N ** w["dims"]) * (k + 1) / (el + one), k + 1, N, el + one


def run_reference(args):
    """Reference arm: the CPU oracle, as it stands, on this host's cores."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_0712_0813_gb300.icgen import lattice_ics
    oracle.build()
    w = WORKLOAD
    # size each step's sub-lattice so that warmup + steps stay within ~150 s
    probe_N = 32
    rate, _, _, _ = cpu_oracle_rate(None, None, 0.5, N_sample=probe_N)
    budget = 150.0 / max(1, args.steps + args.warmup)
    N = 8
    for cand in (8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256):
        if cand ** 3 / rate <= budget:
            N = cand
    fs, us = lattice_ics(w["dims"], N, w["L"], w["nf"], phi0=w["phi0"], q=w["q"], seed=w["seed"])
    p = oracle.Params(dims=w["dims"], N=N, L=w["L"], dt=w["dt"], nf=w["nf"], q=w["q"], expansion=w["expansion"])
    st = oracle.init(p, fs, us)
    oracle.step(st, args.warmup)
    t0 = time.perf_counter()
    oracle.step(st, args.steps)
    el = time.perf_counter() - t0
    value = (N ** 3) * args.steps / el / 1e9
    sample = f"each step = one oracle step of a {N}^3 sub-lattice of the same model (bounded sample of the 256^3 workload)"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
        "device": "host CPU (the oracle; no GPU work)",
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": w["name"], "sample_N": N, "precision": "f64",
                                        "expansion": True, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--workload", default="256cube", choices=sorted(WORKLOADS))
    ap.add_argument("--steps", type=int, default=None, help="timed steps (default: the workload's)")
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="f32", choices=["f32", "f64"])
    ap.add_argument("--fp64-steps", type=int, default=1000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--serve-jobs", type=int, default=16, help="jobs in the serving leg (0: skip)")
    ap.add_argument("--batch-steps", type=int, default=300)
    ap.add_argument("--no-batch", action="store_true", help="skip the mixed-size batched leg")
    ap.add_argument("--plan", default=None,
                    help="force the z-sweep plan rows,stages,zchunks for the FP32 leg (skips autotuning)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="use the library's default launch plan instead of the autotuned one")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    global WORKLOAD
    WORKLOAD = dict(WORKLOADS[args.workload])
    if WORKLOAD["dt"] is None:
        WORKLOAD["dt"] = _courant(WORKLOAD["N"], WORKLOAD["q"])
    if args.steps is None:
        args.steps = WORKLOAD["steps"]
    if args.workload != "256cube":
        args.no_batch = True
        args.serve_jobs = 0
        args.fp64_steps = min(args.fp64_steps, 20)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        print(json.dumps({"error": "no CUDA device"}), flush=True)
        return 1
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_0712_0813_gb300 import replicas

    def barrier():
        replicas.barrier(dist)

    def max_over_ranks(x: float) -> float:
        return replicas.max_over_ranks(x, dist, device="cuda")

    from paper_0712_0813_gb300 import build as pkg_build
    pkg_build.build()
    from paper_0712_0813_gb300 import capi

    w = WORKLOAD
    S = w["N"] ** w["dims"]
    f0, u0 = make_inputs(rank)
    gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local]) \
        if os.environ.get("CUDA_VISIBLE_DEVICES") else local

    # launch-plan autotuning (outside the timed region)
    hints, tune_info = None, None
    if args.plan:
        r_, s_, z_ = (int(x) for x in args.plan.split(","))
        hints = {"tile_rows": r_, "stages": s_, "zchunks": z_}
        tune_info = {"forced": hints}
    elif not args.no_autotune and w["dims"] == 3:
        from paper_0712_0813_gb300 import autotune
        common = dict(N=w["N"], L=w["L"], dt=w["dt"], nfields=w["nf"], q=w["q"], expansion=w["expansion"],
                      phi0=w["phi0"])
        t0 = time.perf_counter()
        res = autotune.autotune_sweep(f0, u0, precision=args.precision, **common)
        hints = res.hints()
        tune_info = {"candidates": len(res.table), "seconds": time.perf_counter() - t0,
                     "best": hints, "best_ms_per_step": res.ms_per_step,
                     "table": [list(t) for t in res.table]}
    ms, kernel, clocks, plan = time_device_steps(capi, torch, f0, u0, args.precision, args.steps, args.warmup,
                                                 barrier, sampler_gpu=gpu_index if rank == 0 else None,
                                                 hints=hints)
    ms = max_over_ranks(ms)
    secs = ms / 1e3
    value = replicas.aggregate_throughput(ws, S * args.steps, secs) / 1e9

    # plain FP64 path on the same lattice (context for the FP32/FP64 ratio): the
    # library's automatic FP64 choice
    ms64, kernel64, _, plan64 = time_device_steps(capi, torch, f0, u0, "f64", args.fp64_steps, args.warmup,
                                                  barrier)
    ms64 = max_over_ranks(ms64)
    value64 = ws * S * args.fp64_steps / (ms64 / 1e3) / 1e9

    e2e = None
    if not args.no_e2e:
        t_e2e, nbytes = time_e2e(capi, torch, f0, u0, args.precision, args.steps, hints=hints)
        t_e2e = max_over_ranks(t_e2e)
        e2e = {"value": ws * S * args.steps / t_e2e / 1e9, "unit": METRIC,
               "h2d_bytes_per_step": nbytes / args.steps, "d2h_bytes_per_step": nbytes / args.steps,
               "job": f"set_fields(host f,u) + {args.steps} steps + get_fields(host f,u), pinned host buffers"}

    hbm_peak, peak_kind = peaks()
    esize = 4 if args.precision == "f32" else 8
    alg_bytes = 4 * esize * w["nf"] * S          # read f, w; write f, w per field and site
    launch_s = secs / args.steps                  # one step kernel per step
    achieved = alg_bytes / launch_s / 1e9
    kname = {"sweep": "k_step_sweep", "rows": "k_step_batched"}.get(kernel, "k_step_generic")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": ncu_traffic(kname, args.precision),
                "kernel": kname, "algorithmic_bytes_per_launch": alg_bytes, "peak_kind": peak_kind}

    batch = None
    if not args.no_batch:
        batch = batched_leg(capi, torch, args.batch_steps, max(args.warmup // 10, 3), 10, hbm_peak)

    serving = None
    if args.serve_jobs > 0 and rank == 0:
        from paper_0712_0813_gb300 import serve
        cap = batch["value_f32_batched"] * 1e9 if batch else None
        serving = serve.run_serving_benchmark(n_jobs=args.serve_jobs, capacity=cap)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        Ns_sample = 256 if w["N"] > 256 else None    # a bounded sample of the large lattices
        rate, k, Ns, el = cpu_oracle_rate(f0, u0, args.cpu_seconds, N_sample=Ns_sample)
        cpu = {"value": rate / 1e9, "unit": METRIC, "cores": 1, "kind": "oracle",
               "sample": f"{k} oracle steps of the full {Ns}^3 lattice ({el:.1f} s, serial FP64 C)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": w["name"], "N": w["N"], "fields": w["nf"], "expansion": w["expansion"],
                       "dt": w["dt"], "L": w["L"], "precision": args.precision,
                       "storage": "fields+velocities " + args.precision + ", global sums and a(t) f64",
                       "kernel": kernel, "sweep_plan": {"tile_rows": plan[0], "stages": plan[1],
                                                         "zchunks": plan[2]},
                       "autotune": tune_info,
                       "parallelism": "replicas" if ws > 1 else "single",
                       "l2": f"state {4 * esize * w['nf'] * S / 1e6:.0f} MB > L2 (129 MB); no flush needed"},
            "fp64_plain": {"value": value64, "ms_per_step": ms64 / args.fp64_steps, "steps": args.fp64_steps,
                           "kernel": kernel64, "sweep_plan": list(plan64), "f32_over_f64": value / value64},
            "roofline": roofline,
            "batched_mix": batch,
            "serving": serving,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": args.steps,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
