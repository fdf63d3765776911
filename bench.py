#!/usr/bin/env python3
"""Throughput benchmark of the lattice leapfrog (one JSON line on rank 0).

Workload (default): 3D 1024^3 periodic lattice, 2 fields phi, chi with
V = phi^4/4 + (q/2) phi^2 chi^2, q = 1.2, L = 20, dt from the Courant rule
(0.0051), expansion on, seeded Gaussian-random-field initial conditions
(paper_0712_0813_gb300.icgen), fields and velocities in FP32 with FP64 global
sums and scale factor.  A "step" is one leapfrog step of the whole lattice
(drift, Laplacian, model force, kick, global sums, scale-factor update).

Metric: Gsite-updates/s = sites * steps / seconds / 1e9 (one site update
advances all fields at one site by one step).  The state (34.4 GB) is far
larger than L2, so no flush is needed between steps.

Beside the headline the line carries: the same lattice in FP64 (the plain
path), the end-to-end figure through host buffers, the expanding 256^3
lattice (timed, and its FP32 and FP64 outputs against the oracle's stored
values of the same run), the 96-lattice mixed batch against the same
lattices one at a time, the serving loop against plain FP64 one job at a
time, and the oracle timed on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --shapes     # per-shape timings of the batched and single-lattice kernels

--impl reference times the CPU oracle (its OpenMP copy, all host cores) on a
bounded sub-lattice of the same model.  Multi-GPU: replicas only
(independent lattices per rank, no data-path collective); launched with
torchrun, rank 0 prints the aggregate.
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


# 1024cube is the default (the bench line); the others run with --workload.
WORKLOADS = {
    "1024cube": dict(name="3d_1024cube_2field_expanding", dims=3, N=1024, L=20.0, dt=None, nf=2,
                     q=(1.2,), expansion=True, phi0=1.0, seed=1, steps=2000),
    "256cube": dict(name="3d_256cube_2field_expanding", dims=3, N=256, L=20.0, dt=0.02, nf=2,
                    q=(1.2,), expansion=True, phi0=1.0, seed=1, steps=5000),
    "512cube_4field": dict(name="3d_512cube_4field_expanding", dims=3, N=512, L=20.0, dt=None, nf=4,
                           q=(0.8, 5.0, 40.0), expansion=True, phi0=1.0, seed=1, steps=1000),
}
WORKLOAD = WORKLOADS["1024cube"]
METRIC = "Gsite-updates/s"
GOLDEN_256 = os.path.join(ROOT, "tests", "golden", "longrun_256cube.json")
STEP_SOURCES = {"k_step_sweep": ("ce_sweep3d.cuh", "ce_sweep3d_f32.cu", "ce_tma.cuh", "ce_device.cuh",
                                 "ce_internal.h"),
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


def ncu_traffic(kernel_name: str, precision: str, sites: int, nf: int):
    """DRAM bytes per launch from the committed ncu record, if it was taken on
    the current kernel source (same hash) with the same field count, scaled
    from the captured lattice's sites to `sites` (the traffic of the streaming
    kernel grows with the sites it processes); else None.  Returns (bytes, note)."""
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.md")
    if not os.path.exists(path):
        return None, None
    pat = re.compile(rf"^traffic\s+{re.escape(kernel_name)}\s+{precision}\s+nf={nf}\s+src=(\w+)\s+"
                     rf"bytes_per_launch=(\d+)\s+sites=(\d+)")
    cur = kernel_source_hash(kernel_name)
    with open(path) as fh:
        for line in fh:
            m = pat.match(line.strip())
            if m and m.group(1) == cur:
                b, s = int(m.group(2)), int(m.group(3))
                note = None if s == sites else f"captured on {s} sites, scaled by {sites / s:g}"
                return int(round(b * sites / s)), note
    return None, None


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


def make_inputs(w: dict, rank: int, backend: str | None = None, pinned: bool = False):
    from paper_0712_0813_gb300.icgen import lattice_ics
    from paper_0712_0813_gb300.replicas import replica_seed
    big = w["N"] ** w["dims"] >= 1 << 25
    return lattice_ics(w["dims"], w["N"], w["L"], w["nf"], phi0=w["phi0"], q=w["q"],
                       seed=replica_seed(w["seed"], rank), backend=backend or ("torch" if big else "numpy"),
                       pinned=pinned and big)


def sim_config(w: dict, precision: str, stream, hints=None):
    cfg = dict(dims=w["dims"], N=w["N"], L=w["L"], dt=w["dt"], nfields=w["nf"], q=w["q"],
               expansion=w["expansion"], phi0=w["phi0"], precision=precision, stream=stream)
    cfg.update(hints or {})
    return cfg


def tune_budget(N: int) -> dict:
    """Autotuner effort: large lattices take fewer timed steps per candidate."""
    if N >= 1024:
        return dict(steps=10, warmup=2, repeats=1)
    if N >= 512:
        return dict(steps=16, warmup=4, repeats=1)
    return dict(steps=40, warmup=8, repeats=2)


def lattice_stats(sim) -> dict:
    en = sim.energy()
    mean, var = sim.means_variances()
    return {"step": int(en["step"]), "mean": [float(x) for x in mean], "var": [float(x) for x in var],
            "E": float(en["E"]), "a": float(en["a"]), "ap": float(en["ap"])}


def stats_error(got: dict, ref: dict) -> dict:
    """Relative errors of lattice statistics (a mean against the field's spread)."""
    spread = np.maximum(np.abs(np.asarray(ref["mean"])), np.sqrt(np.asarray(ref["var"])))
    return {"mean": [float(x) for x in np.abs(np.asarray(got["mean"]) - np.asarray(ref["mean"])) / spread],
            "var": [float(x) for x in np.abs(np.asarray(got["var"]) / np.asarray(ref["var"]) - 1.0)],
            "E": abs(got["E"] / ref["E"] - 1.0), "a": abs(got["a"] / ref["a"] - 1.0),
            "ap": abs(got["ap"] / ref["ap"] - 1.0) if ref["ap"] else None}


def time_device_steps(capi, torch, w, f0, u0, precision, steps, warmup, barrier, sampler_gpu=None,
                      hints=None, tune=False, stats=False):
    """Device-resident timing: CUDA events on the library's stream around
    `steps` launches.  With tune=True the z-sweep plan is autotuned on this
    same handle first (ce_replan between candidates; outside the timed
    region), so a large lattice is uploaded once."""
    from paper_0712_0813_gb300 import autotune
    stream = torch.cuda.Stream()
    tune_info = None
    kw = sim_config(w, precision, stream.cuda_stream, hints)
    if tune:
        kw["kernel"] = "sweep"
    sim = capi.Simulation(**kw)
    sim.set_fields(f0, u0)
    if tune:
        t0 = time.perf_counter()
        table = autotune.tune_handle(sim, stream, w["N"], **tune_budget(w["N"]))
        best = min(table, key=lambda t: t[3])
        sim.replan(best[0], best[1], best[2])
        tune_info = {"candidates": len(table), "seconds": time.perf_counter() - t0,
                     "best": {"tile_rows": best[0], "stages": best[1], "zchunks": best[2]},
                     "best_ms_per_step": best[3], "table": [list(t) for t in table]}
    sim.step(warmup)
    sim.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    clocks = None
    barrier()
    torch.cuda.synchronize()
    cs = None
    if sampler_gpu is not None:
        cs = ClockSampler(sampler_gpu)
        cs.__enter__()
        time.sleep(0.25)
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    if cs is not None:
        cs.__exit__(None, None, None)
        clocks = cs.summary()
    barrier()
    sim.synchronize()  # surfaces any latched device error
    ms = e0.elapsed_time(e1)
    kernel = {1: "generic", 2: "sweep", 3: "rows", 4: "planes"}[sim.kernel]
    plan = sim.sweep_plan
    st = lattice_stats(sim) if stats else None
    sim.close()
    if stats:
        return ms, kernel, clocks, plan, tune_info, st
    return ms, kernel, clocks, plan, tune_info


def time_e2e(capi, torch, w, f0, u0, precision, steps, hints=None, inputs_pinned=False):
    """End to end through the public API with pinned host buffers: upload of the
    initial state, start-up, `steps` steps, download of the final state.  With
    inputs_pinned the inputs' own page-locked memory serves as the buffers and
    receives the final state (the caller's last use of them)."""
    nf, S = f0.shape
    if inputs_pinned:
        pin_f, pin_u = f0.reshape(-1), u0.reshape(-1)
    else:
        pin_f = torch.empty(nf * S, dtype=torch.float64, pin_memory=True).numpy()
        pin_u = torch.empty(nf * S, dtype=torch.float64, pin_memory=True).numpy()
        pin_f[:] = f0.reshape(-1)
        pin_u[:] = u0.reshape(-1)
    out_f, out_v = pin_f, pin_u          # the inputs are consumed by set_fields: reuse them for the outputs
    stream = torch.cuda.Stream()
    sim = capi.Simulation(**sim_config(w, precision, stream.cuda_stream, hints))
    sim.set_fields(pin_f, pin_u)  # warm (first-touch, module load); reads the buffers only
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.set_fields(pin_f, pin_u)
    sim.step(steps)
    capi.ce_get_fields(sim.handle, nf, S, capi.CE_VEL_SYNC, out=(out_f, out_v))
    t1 = time.perf_counter()
    sim.close()
    del pin_f, pin_u, out_f, out_v
    nbytes = 2 * nf * S * 8
    return t1 - t0, nbytes


def roofline_of(w, precision, ms_per_step, hbm_peak, peak_kind, kernel):
    S = w["N"] ** w["dims"]
    esize = 4 if precision == "f32" else 8
    alg = 4 * esize * w["nf"] * S          # read f, w; write f, w per field and site
    achieved = alg / (ms_per_step / 1e3) / 1e9
    kname = {"sweep": "k_step_sweep", "rows": "k_step_batched",
             "planes": "k_step_cols" if w["dims"] == 3 else "k_step_lines"}.get(kernel, "k_step_generic")
    traffic, note = ncu_traffic(kname, precision, S, w["nf"]) if kname in STEP_SOURCES else (None, None)
    out = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
           "traffic": traffic, "kernel": kname, "algorithmic_bytes_per_launch": alg, "peak_kind": peak_kind}
    if note:
        out["traffic_note"] = note
    return out


# FP64 instructions per site of the generic kernel's two-pass FP64 step, 3D, 2
# fields (ncu, 256^3: k_drift_g 2 per field and site, k_kick_from_g 14.1; each
# DADD, DMUL or DFMA takes one slot of the FP64 pipe), and the pipe's rate:
# GB300's nominal FP64 1.25 TFLOP/s counts a DFMA as 2 flops, so 0.625 T
# instructions/s (152 SMs x 2 FP64 lanes x 2.07 GHz = 0.629 T).
FP64_OPS_PER_SITE_2F_3D = 32.2
FP64_PIPE_PEAK_TOPS = 0.625


def fp64_alu_roofline(w, gsites_per_s: float, kernel: str, hbm_peak: float):
    """The plain FP64 path is bound by GB300's FP64 pipe, not by HBM: its
    roofline in FP64 instructions per second (2-field 3D lattices on the generic
    kernel's two passes, whose per-site count was measured)."""
    if not (w["dims"] == 3 and w["nf"] == 2 and kernel == "generic"):
        return None
    achieved = gsites_per_s * FP64_OPS_PER_SITE_2F_3D / 1e3
    return {"bound": "alu", "achieved": achieved, "peak": FP64_PIPE_PEAK_TOPS, "unit": "T FP64 instructions/s",
            "frac": achieved / FP64_PIPE_PEAK_TOPS, "ops_per_site": FP64_OPS_PER_SITE_2F_3D,
            "peak_kind": "nominal FP64 rate (1.25 TFLOP/s, a DFMA = 2 flops = one pipe slot)",
            "hbm_frac": gsites_per_s * 4 * 8 * w["nf"] / hbm_peak}


def cube256_leg(capi, torch, steps: int, warmup: int, hbm_peak: float, peak_kind: str):
    """The expanding 256^3 lattice (the 5000-step configuration), FP32 with the
    autotuned z-sweep plan, timed for `steps` steps on the device."""
    w = dict(WORKLOADS["256cube"])
    f0, u0 = make_inputs(w, 0, backend="numpy")
    ms, kernel, _, plan, tune = time_device_steps(capi, torch, w, f0, u0, "f32", steps, warmup,
                                                  lambda: None, tune=True)
    S = w["N"] ** 3
    return {"workload": w["name"], "value": S * steps / (ms / 1e3) / 1e9, "unit": METRIC, "steps": steps,
            "ms_per_step": ms / steps, "kernel": kernel, "sweep_plan": list(plan),
            "autotune_best": tune["best"] if tune else None,
            "roofline": roofline_of(w, "f32", ms / steps, hbm_peak, peak_kind, kernel)}


def fp32_error_leg(capi, torch, golden_path: str = GOLDEN_256):
    """FP32 (and FP64) outputs of the expanding 256^3 run against the oracle's
    stored values of the same run (tests/golden/longrun_256cube.json, written
    by the serial FP64 oracle only): f and f'(t+dt/2) at the stored sample of
    sites after 100 steps (max |gpu - oracle| / max over the lattice of
    |oracle|, per field), and means, variances, E, a, a' at every stored
    checkpoint up to 5000 steps (relative; a mean against the field's spread)."""
    if not os.path.exists(golden_path):
        return {"unavailable": f"{os.path.relpath(golden_path, ROOT)} is missing"}
    with open(golden_path) as fh:
        gold = json.load(fh)
    c = gold["config"]
    w = dict(WORKLOADS["256cube"])
    assert (c["N"], c["dt"], c["nf"], tuple(c["q"]), c["seed"]) == (w["N"], w["dt"], w["nf"], w["q"], w["seed"])
    f0, u0 = make_inputs(w, 0, backend=c["ic_backend"])
    sites = np.asarray(gold["sample_sites"], dtype=np.int64)
    out = {"oracle_run": f"serial FP64 oracle, {c['N']}^3, {gold['checkpoints'][-1]['step']} steps"
                         + ("" if gold.get("complete") else " (incomplete file)")}
    for precision in ("f32", "f64"):
        stream = torch.cuda.Stream()
        sim = capi.Simulation(**sim_config(w, precision, stream.cuda_stream))
        sim.set_fields(f0, u0)
        res = {"kernel": {1: "generic", 2: "sweep", 3: "rows", 4: "planes"}[sim.kernel], "checkpoints": []}
        worst = {}
        done = 0
        for cp in gold["checkpoints"]:
            sim.step(cp["step"] - done)
            done = cp["step"]
            got = lattice_stats(sim)
            if cp["step"] == gold["sample_step"] and "samples" in gold:
                f, v, _ = sim.sample_fields(sites)
                smp = gold["samples"]
                res["f_relmax_step100"] = [float(np.abs(f[i] - np.asarray(smp["f"][i])).max() / smp["f_absmax"][i])
                                           for i in range(w["nf"])]
                res["v_relmax_step100"] = [float(np.abs(v[i] - np.asarray(smp["v_staggered"][i])).max()
                                                 / smp["v_absmax"][i]) for i in range(w["nf"])]
            e = dict(step=cp["step"], **stats_error(got, cp))
            res["checkpoints"].append(e)
            for k in ("mean", "var"):
                worst[k] = max(worst.get(k, 0.0), max(e[k]))
            for k in ("E", "a", "ap"):
                if e[k] is not None:
                    worst[k] = max(worst.get(k, 0.0), e[k])
        res["max_rel_error"] = worst
        res["final"] = res["checkpoints"][-1]
        sim.close()
        out[precision] = res
    return out


def batched_leg(capi, torch, steps: int, warmup: int, seq_steps: int, hbm_peak: float):
    """Mixed-size workload (96 lattices of 1D/2D/3D): the batched FP32 persistent
    kernel against the same lattices stepped one by one with the plain FP64 path
    and with the plain FP32 path (device-resident, CUDA events; each lattice
    timed over seq_steps steps after 3 warm-up steps, graphs of 32 launches)."""
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

    fp64_seq = sequential("f64", seq_steps) if seq_steps > 0 else None
    f32_seq = sequential("f32", seq_steps) if seq_steps > 0 else None
    alg = 16 * 2 * total
    achieved = alg / (ms / 1e3 / steps) / 1e9
    return {"workload": "96 lattices: 32 x 1D 65536, 32 x 2D 1024^2, 32 x 3D side in {64..192}; 2 fields, "
                        "per-lattice q, phi0, Courant dt, expansion on half",
            "sites": total, "steps": steps, "ms_per_step": ms / steps, "items": info["items"],
            "sweep_len": tune["sweep_len"], "ctas_per_sm": tune["ctas_per_sm"], "autotune": tune["table"],
            "blocks": info["blocks"], "value_f32_batched": batched, "fp64_plain_sequential": fp64_seq,
            "f32_plain_sequential": f32_seq, "batched_over_fp64_plain": batched / fp64_seq if fp64_seq else None,
            "sequential_steps": seq_steps,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "kernel": "k_step_batched",
                         "algorithmic_bytes_per_launch": alg}}


def cpu_oracle_rate(w, target_s: float, N_sample: int, parallel: bool, f0=None, u0=None):
    """Sites/s of the CPU oracle on the bench model, on a lattice of N_sample^3
    sites: the serial oracle (1 thread) or its OpenMP copy (all host cores)."""
    import oracle
    from paper_0712_0813_gb300.icgen import lattice_ics
    if f0 is None:
        f0, u0 = lattice_ics(w["dims"], N_sample, w["L"], w["nf"], phi0=w["phi0"], q=w["q"], seed=w["seed"])
    p = oracle.Params(dims=w["dims"], N=N_sample, L=w["L"], dt=w["dt"], nf=w["nf"], q=w["q"],
                      expansion=w["expansion"])
    init, step = (oracle.omp_init, oracle.omp_step) if parallel else (oracle.init, oracle.step)
    threads = oracle.omp_threads() if parallel else 1
    st = init(p, f0, u0)
    t0 = time.perf_counter()
    step(st, 1)
    one = time.perf_counter() - t0
    k = max(1, int(target_s / max(one, 1e-6)) - 1)
    t0 = time.perf_counter()
    step(st, k)
    el = time.perf_counter() - t0
    return (N_sample ** w["dims"]) * (k + 1) / (el + one), k + 1, el + one, threads


def cpu_baseline_leg(w, seconds: float):
    """The oracle timed on the host cores: the OpenMP copy of its loops on all
    cores (the reported value) and the serial oracle on one core beside it, on
    a bounded sample of the workload (a 256^3 lattice of the same model)."""
    import oracle
    from paper_0712_0813_gb300.icgen import lattice_ics
    oracle.build()
    Ns = min(w["N"], 256)
    f0, u0 = lattice_ics(w["dims"], Ns, w["L"], w["nf"], phi0=w["phi0"], q=w["q"], seed=w["seed"])
    par, kp, elp, threads = cpu_oracle_rate(w, seconds, Ns, True, f0, u0)
    ser, ks, els, _ = cpu_oracle_rate(w, seconds, Ns, False, f0, u0)
    return {"value": par / 1e9, "unit": METRIC, "cores": threads, "kind": "oracle",
            "sample": (f"{kp} steps of a {Ns}^3 lattice of the same model ({elp:.1f} s) by the OpenMP copy "
                       f"of the oracle's loops on {threads} threads (os.cpu_count() = {os.cpu_count()})"),
            "serial_1core": {"value": ser / 1e9, "unit": METRIC, "cores": 1,
                             "sample": f"{ks} steps of the same lattice ({els:.1f} s), serial FP64 C oracle"}}


def run_reference(args, w):
    """Reference arm: the CPU oracle (its OpenMP copy, all host cores)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_0712_0813_gb300.icgen import lattice_ics
    oracle.build()
    threads = oracle.omp_threads()
    # size each step's sub-lattice so that warmup + steps stay within ~150 s
    rate, _, _, _ = cpu_oracle_rate(w, 0.5, 32, True)
    budget = 150.0 / max(1, args.steps + args.warmup)
    N = 8
    for cand in (8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512):
        if cand ** 3 / rate <= budget and cand <= w["N"]:
            N = cand
    fs, us = lattice_ics(w["dims"], N, w["L"], w["nf"], phi0=w["phi0"], q=w["q"], seed=w["seed"])
    p = oracle.Params(dims=w["dims"], N=N, L=w["L"], dt=w["dt"], nf=w["nf"], q=w["q"], expansion=w["expansion"])
    st = oracle.omp_init(p, fs, us)
    oracle.omp_step(st, args.warmup)
    t0 = time.perf_counter()
    oracle.omp_step(st, args.steps)
    el = time.perf_counter() - t0
    value = (N ** 3) * args.steps / el / 1e9
    sample = (f"each step = one oracle step of a {N}^3 sub-lattice of the same model (bounded sample of the "
              f"{w['N']}^3 workload), OpenMP copy of the oracle's loops on {threads} threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
        "device": "host CPU (the oracle; no GPU work)",
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": w["name"], "sample_N": N, "precision": "f64",
                                        "expansion": True, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _shape_timed(torch, stream, fn_step, steps: int, warmup: int) -> float:
    fn_step(warmup)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fn_step(steps)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / steps * 1e3        # us per step


def _shape_batch_row(capi, torch, stream, sims, sites, item_lengths, steps, warmup, peak):
    out = {}
    for L in item_lengths:
        with capi.Batch(sims, sweep_len=L, stream=stream.cuda_stream) as b:
            us = _shape_timed(torch, stream, b.step, steps, warmup)
            items = b.info["items"]
            b.synchronize()
        out[f"L{L}"] = {"us": us, "gsite_per_s": sites / us / 1e3, "frac": 32.0 * sites / us / 1e3 / peak,
                        "items": items}
    return out


def shapes_mode(steps: int = 100, warmup: int = 20, item_lengths=(64, 128)) -> int:
    """Per-shape timings of the batched kernel and of the single-lattice
    kernels, one JSON line per case (FP32 storage, 2 fields, expansion on):

    * mix_class: the 96-lattice mixed batch and its 1D, 2D and 3D parts alone,
      one k_step_batched launch per step, at two item lengths;
    * batch_3d: homogeneous batches of about 100 M sites of one 3D side;
    * single: one lattice stepped by ce_step with the generic kernel, the row
      kernel (CE_KERNEL_ROWS, sides that are multiples of 4) and the column /
      line-sweep kernel (CE_KERNEL_PLANES, 3D / 2D), FP32 and FP64.

    CUDA events on the library's stream around `steps` steps after `warmup`;
    frac = the algorithmic 16 B per field and site / time / measured HBM."""
    import torch
    from paper_0712_0813_gb300 import build as pkg_build
    pkg_build.build()
    from paper_0712_0813_gb300 import capi, workloads
    from paper_0712_0813_gb300.icgen import courant_dt, lattice_ics
    peak, _ = peaks()
    stream = torch.cuda.Stream()
    specs = workloads.mixed_batch_specs()
    ics = [workloads.make_ics(sp) for sp in specs]
    groups = {"1d": [k for k, s in enumerate(specs) if s["dims"] == 1],
              "2d": [k for k, s in enumerate(specs) if s["dims"] == 2],
              "3d": [k for k, s in enumerate(specs) if s["dims"] == 3],
              "all": list(range(len(specs)))}
    for name, idx in groups.items():
        sims = []
        for k in idx:
            sim = capi.Simulation(**workloads.sim_kwargs(specs[k], "f32"), kernel="generic")
            sim.set_fields(*ics[k])
            sims.append(sim)
        sites = sum(workloads.sites(specs[k]) for k in idx)
        row = {"case": "mix_class", "class": name, "lattices": len(idx), "sites": sites}
        row.update(_shape_batch_row(capi, torch, stream, sims, sites, item_lengths, steps, warmup, peak))
        print(json.dumps(row), flush=True)
        for sim in sims:
            sim.close()
    for N, count in ((64, 384), (96, 113), (128, 48), (160, 24), (192, 14)):
        f0, u0 = lattice_ics(3, N, 20.0, 2, q=(1.2,), seed=3, amp=1e-2,
                             backend="torch" if N ** 3 >= 1 << 22 else "numpy")
        dt = courant_dt(3, N, 20.0, 1.0, (1.2,))
        sims = []
        for _ in range(count):
            sim = capi.Simulation(dims=3, N=N, L=20.0, dt=dt, nfields=2, q=(1.2,), expansion=True,
                                  precision="f32", kernel="generic")
            sim.set_fields(f0, u0)
            sims.append(sim)
        sites = count * N ** 3
        row = {"case": "batch_3d", "N": N, "lattices": count, "sites": sites}
        row.update(_shape_batch_row(capi, torch, stream, sims, sites, item_lengths, steps, warmup, peak))
        print(json.dumps(row), flush=True)
        for sim in sims:
            sim.close()
    for dims, N in ((1, 65536), (2, 257), (2, 385), (2, 1023), (2, 1024), (2, 6000), (2, 6001), (3, 48), (3, 64),
                    (3, 95), (3, 96),
                    (3, 160), (3, 192), (3, 255), (3, 288), (3, 383), (3, 448), (3, 511)):
        big = N ** dims >= 1 << 22
        f0, u0 = lattice_ics(dims, N, 20.0, 2, q=(1.2,), seed=3, amp=1e-2, backend="torch" if big else "numpy")
        dt = courant_dt(dims, N, 20.0, 1.0, (1.2,))
        row = {"case": "single", "dims": dims, "N": N}
        kernels = ("generic",) + (("rows",) if N % 4 == 0 else ()) + (("planes",) if dims >= 2 else ())
        for prec in ("f32", "f64"):
            for kern in kernels:
                with capi.Simulation(dims=dims, N=N, L=20.0, dt=dt, nfields=2, q=(1.2,), expansion=True,
                                     precision=prec, kernel=kern, stream=stream.cuda_stream) as sim:
                    sim.set_fields(f0, u0)
                    n = max(10, min(2 * steps, int(2e9 / (N ** dims * 8 * (4 if prec == "f32" else 8)))))
                    us = _shape_timed(torch, stream, sim.step, n, min(2 * warmup, n))
                    row[f"{prec}_{kern}_us"] = us
                    row[f"{prec}_{kern}_frac"] = (4 * (4 if prec == "f32" else 8) * 2 * N ** dims
                                                  / (us * 1e-6) / 1e9 / peak)
        print(json.dumps(row), flush=True)
    return 0


def single_mode(spec: str, steps: int, warmup: int) -> int:
    """One lattice, one kernel: `dims,N,kernel[,precision[,fields]]` (kernel auto,
    generic, sweep, rows or planes), 2 fields by default, expansion on, q = 1.2
    (fields 4: q = 0.8, 5, 40), Courant dt.  Prints one JSON line with the time
    per step (CUDA events) and the fraction of measured HBM the algorithmic
    16 (FP32) / 32 (FP64) bytes per field and site reach.  Small cases of this
    mode are what the ncu captures under profiles/ run."""
    import torch
    from paper_0712_0813_gb300 import build as pkg_build
    pkg_build.build()
    from paper_0712_0813_gb300 import capi
    from paper_0712_0813_gb300.icgen import courant_dt, lattice_ics
    parts = spec.split(",")
    dims, N, kernel = int(parts[0]), int(parts[1]), parts[2]
    precision = parts[3] if len(parts) > 3 else "f32"
    nf = int(parts[4]) if len(parts) > 4 else 2
    q = (1.2,) if nf == 2 else (0.8, 5.0, 40.0)[:nf - 1]
    peak, _ = peaks()
    S = N ** dims
    f0, u0 = lattice_ics(dims, N, 20.0, nf, q=q, seed=3, backend="torch" if S >= 1 << 25 else "numpy")
    stream = torch.cuda.Stream()
    with capi.Simulation(dims=dims, N=N, L=20.0, dt=courant_dt(dims, N, 20.0, 1.0, q), nfields=nf, q=q,
                         expansion=True, precision=precision, kernel=kernel, stream=stream.cuda_stream) as sim:
        sim.set_fields(f0, u0)
        us = _shape_timed(torch, stream, sim.step, steps, warmup)
        sim.synchronize()
        used = {1: "generic", 2: "sweep", 3: "rows", 4: "planes"}[sim.kernel]
    alg = 4 * (4 if precision == "f32" else 8) * nf * S
    print(json.dumps({"case": "single", "dims": dims, "N": N, "fields": nf, "precision": precision,
                      "kernel": used, "steps": steps, "us_per_step": us, "gsite_per_s": S / us / 1e3,
                      "frac": alg / (us * 1e-6) / 1e9 / peak}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--workload", default="1024cube", choices=sorted(WORKLOADS))
    ap.add_argument("--steps", type=int, default=None, help="timed steps (default: the workload's)")
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="f32", choices=["f32", "f64"])
    ap.add_argument("--fp64-steps", type=int, default=None,
                    help="timed steps of the FP64 leg (default: 20 at 1024^3, 1000 below)")
    ap.add_argument("--cube256-steps", type=int, default=2000,
                    help="timed steps of the 256^3 leg (0: skip; skipped when it is the workload)")
    ap.add_argument("--no-fp32-error", action="store_true", help="skip the 256^3 errors against the oracle")
    ap.add_argument("--golden", default=GOLDEN_256,
                    help="stored oracle values of the 256^3 run for the fp32_error key")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="CPU seconds per oracle leg")
    ap.add_argument("--serve-jobs", type=int, default=16, help="jobs in the serving leg (0: skip)")
    ap.add_argument("--serve-fp64", default="measured", choices=["measured", "model"])
    ap.add_argument("--batch-steps", type=int, default=3000, help="steps of the batched mix (its full run)")
    ap.add_argument("--seq-steps", type=int, default=64, help="steps per lattice of the one-at-a-time baselines")
    ap.add_argument("--no-batch", action="store_true", help="skip the mixed-size batched leg")
    ap.add_argument("--plan", default=None,
                    help="force the z-sweep plan rows,stages,zchunks for the FP32 leg (skips autotuning)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="use the library's default launch plan instead of the autotuned one")
    ap.add_argument("--shapes", action="store_true",
                    help="per-shape timings of the batched and single-lattice kernels (JSON lines), then exit")
    ap.add_argument("--single", default=None, metavar="DIMS,N,KERNEL[,PREC[,FIELDS]]",
                    help="time one lattice on one kernel for --steps steps (JSON line), then exit")
    ap.add_argument("--batch-only", action="store_true",
                    help="run only the mixed-batch leg (--batch-steps, no one-at-a-time baselines), then exit")
    args = ap.parse_args()
    if args.shapes:
        return shapes_mode()
    if args.single:
        return single_mode(args.single, args.steps or 20, args.warmup)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    w = dict(WORKLOADS[args.workload])
    if w["dt"] is None:
        w["dt"] = _courant(w["N"], w["q"])
    if args.steps is None:
        args.steps = w["steps"]
    if args.fp64_steps is None:
        args.fp64_steps = 20 if w["N"] >= 1024 else 1000
    if args.impl == "reference":
        return run_reference(args, w)

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

    hbm_peak, peak_kind = peaks()
    if args.batch_only:
        print(json.dumps({"batched_mix": batched_leg(capi, torch, args.batch_steps, 3, 0, hbm_peak)}), flush=True)
        return 0
    S = w["N"] ** w["dims"]
    # large inputs in page-locked memory: the e2e leg (last) copies from and into them
    f0, u0 = make_inputs(w, rank, pinned=True)
    inputs_pinned = S >= 1 << 25
    gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local]) \
        if os.environ.get("CUDA_VISIBLE_DEVICES") else local

    hints, tune = None, False
    if args.plan:
        r_, s_, z_ = (int(x) for x in args.plan.split(","))
        hints = {"tile_rows": r_, "stages": s_, "zchunks": z_}
    elif not args.no_autotune and w["dims"] == 3 and args.precision == "f32":
        tune = True   # (FP64 keeps the automatic choice: the generic kernel's two passes, faster in FP64)
    ms, kernel, clocks, plan, tune_info = time_device_steps(
        capi, torch, w, f0, u0, args.precision, args.steps, args.warmup, barrier,
        sampler_gpu=gpu_index if rank == 0 else None, hints=hints, tune=tune)
    if args.plan:
        tune_info = {"forced": hints}
    if tune_info and "best" in tune_info:
        hints = dict(tune_info["best"])
    ms = max_over_ranks(ms)
    secs = ms / 1e3
    value = replicas.aggregate_throughput(ws, S * args.steps, secs) / 1e9
    roofline = roofline_of(w, args.precision, ms / args.steps, hbm_peak, peak_kind, kernel)
    if args.precision == "f64":   # bound by the FP64 pipe, not by HBM: that roofline when it is known
        roofline = fp64_alu_roofline(w, value / ws, kernel, hbm_peak) or roofline   # per GPU

    # plain FP64 path on the same lattice: the library's automatic FP64 choice
    w64 = min(args.warmup, 5)
    ms64, kernel64, _, plan64, _, st64 = time_device_steps(capi, torch, w, f0, u0, "f64", args.fp64_steps, w64,
                                                           barrier, stats=True)
    ms64 = max_over_ranks(ms64)
    value64 = ws * S * args.fp64_steps / (ms64 / 1e3) / 1e9
    # the headline lattice in FP32 (the timed launch plan) after the same number of
    # steps, against the FP64 path (which matches the oracle to 1e-11 over 100
    # steps on the lattices the oracle can run)
    fp32_vs_fp64 = None
    if rank == 0:
        stream = torch.cuda.Stream()
        with capi.Simulation(**sim_config(w, "f32", stream.cuda_stream, hints)) as sim32:
            sim32.set_fields(f0, u0)
            sim32.step(st64["step"])
            st32 = lattice_stats(sim32)
        fp32_vs_fp64 = {"steps": st64["step"], "errors": stats_error(st32, st64), "fp64": st64,
                        "note": "FP32 storage against the FP64 path of the library on the same inputs"}

    # end to end through the public API (last use of the inputs: with page-locked
    # inputs their memory is the transfer buffer and receives the final state)
    e2e = None
    if not args.no_e2e:
        t_e2e, nbytes = time_e2e(capi, torch, w, f0, u0, args.precision, args.steps, hints=hints,
                                 inputs_pinned=inputs_pinned)
        t_e2e = max_over_ranks(t_e2e)
        e2e = {"value": ws * S * args.steps / t_e2e / 1e9, "unit": METRIC,
               "h2d_bytes_per_step": nbytes / args.steps, "d2h_bytes_per_step": nbytes / args.steps,
               "job": f"set_fields(host f,u) + {args.steps} steps + get_fields(host f,u), pinned host buffers"}
    del f0, u0

    cube256 = None
    if args.cube256_steps > 0 and args.workload != "256cube" and rank == 0:
        cube256 = cube256_leg(capi, torch, args.cube256_steps, args.warmup, hbm_peak, peak_kind)

    fp32_error = None
    if not args.no_fp32_error and rank == 0:
        fp32_error = fp32_error_leg(capi, torch, args.golden)

    batch = None
    if not args.no_batch:
        batch = batched_leg(capi, torch, args.batch_steps, max(args.warmup // 10, 3), args.seq_steps, hbm_peak)

    serving = None
    if args.serve_jobs > 0 and rank == 0:
        from paper_0712_0813_gb300 import serve
        cap = batch["value_f32_batched"] * 1e9 if batch else None
        serving = serve.run_serving_benchmark(n_jobs=args.serve_jobs, capacity=cap, fp64_baseline=args.serve_fp64)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_leg(w, args.cpu_seconds)

    if rank == 0:
        esize = 4 if args.precision == "f32" else 8
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
                           "kernel": kernel64, "sweep_plan": list(plan64), "f32_over_f64": value / value64,
                           "roofline": fp64_alu_roofline(w, value64 / ws, kernel64, hbm_peak)},
            "roofline": roofline,
            "fp32_vs_fp64": fp32_vs_fp64,
            "cube256": cube256,
            "fp32_error": fp32_error,
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
