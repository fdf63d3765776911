"""Serving loop: continuous batching of lattice-simulation jobs on one GPU.

Jobs (lattice spec, initial fields, number of steps) arrive over time.  The
server admits them first-come first-served while their device footprint fits
an HBM budget; admitted jobs keep their state resident on the GPU and advance
together, a chunk of steps at a time, in the batched persistent kernel
(`ce_batch_*`: one launch advances every active lattice by one step).
Between chunks finished jobs leave (their outputs are read back and their
memory freed) and newly admitted jobs join.  A job that arrives while a chunk
runs is created and uploaded on its own stream at once, so its host-to-device
copies overlap the running chunk; it joins at the next chunk boundary.

Because a lattice's work items and their summation order depend only on that
lattice, every job's result is bit-identical whether it runs alone or inside
any mix, and whatever the chunk boundaries are.

The loop is written against a small backend interface; `GpuBackend` drives
the C ABI, and the test-suite drives the same loop with a host-only fake to
check admission, cancellation and failure handling without a GPU.
"""
from __future__ import annotations

import argparse
import json
import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import workloads


@dataclass
class Job:
    id: int
    spec: dict
    steps: int
    arrival: float                      # seconds after the server starts
    f0: np.ndarray | None = None
    u0: np.ndarray | None = None
    state: str = "pending"              # pending, running, done, rejected, cancelled, failed
    steps_done: int = 0
    admitted_at: float | None = None
    finished_at: float | None = None
    result: dict = field(default_factory=dict)
    error: str | None = None

    @property
    def latency(self) -> float | None:
        return None if self.finished_at is None else self.finished_at - self.arrival

    @property
    def site_steps(self) -> int:
        return workloads.sites(self.spec) * self.steps


class GpuBackend:
    """Runs jobs through libclusterlat: one handle per job, one batch per chunk."""

    def __init__(self, precision: str = "f32", keep_fields: bool = False):
        from . import capi
        import torch
        self.capi = capi
        self.torch = torch
        self.precision = precision
        self.keep_fields = keep_fields
        self.stream = torch.cuda.Stream()

    def footprint(self, spec: dict) -> int:
        S = workloads.sites(spec)
        staging = min(S, 1 << 22) * spec["nf"] * 8
        return workloads.state_bytes(spec, self.precision) + staging + (1 << 20)

    def create(self, job: Job):
        sim = self.capi.Simulation(**workloads.sim_kwargs(job.spec, self.precision), kernel="generic")
        sim.set_fields(job.f0, job.u0)
        return sim

    def make_batch(self, handles):
        return self.capi.Batch(handles, stream=self.stream.cuda_stream)

    def free_batch(self, batch):
        batch.close()

    def step(self, batch, n: int):
        batch.step(n)

    def wait(self, batch):
        batch.synchronize()

    def member_errors(self, batch) -> dict:
        """{member index: latched error code} of the members that failed."""
        return {k: c for k, c in enumerate(batch.member_status()) if c != 0}

    def result(self, handle) -> dict:
        en = handle.energy()
        mean, var = handle.means_variances()
        out = {"E": en["E"], "a": en["a"], "t": en["t"], "step": en["step"],
               "mean": mean.tolist(), "var": var.tolist()}
        if self.keep_fields:
            f, v, sc = handle.get_fields(self.capi.CE_VEL_STAGGERED)
            out["f"], out["v"] = f, v
        return out

    def free(self, handle):
        handle.close()


class Server:
    """First-come first-served admission under an HBM budget, chunked batched stepping."""

    def __init__(self, backend, hbm_budget: float, chunk_steps: int = 256, clock=time.perf_counter,
                 sleep=time.sleep):
        self.backend = backend
        self.budget = float(hbm_budget)
        self.chunk_steps = int(chunk_steps)
        self.clock = clock
        self.sleep = sleep
        self.used = 0.0
        self.peak_used = 0.0
        self.active: list = []            # (job, handle, footprint)
        self.cancel_requests: set = set()
        self.chunks = 0
        self.rebuilds = 0

    def cancel(self, job_id: int):
        """Ask for a job to be dropped at the next chunk boundary (or before admission)."""
        self.cancel_requests.add(job_id)

    # -- internals ---------------------------------------------------------
    def _admit(self, pending: list, now: float) -> bool:
        changed = False
        while pending and pending[0].arrival <= now:
            job = pending[0]
            if job.id in self.cancel_requests:
                job.state = "cancelled"
                pending.pop(0)
                continue
            fp = self.backend.footprint(job.spec)
            if fp > self.budget:
                job.state = "rejected"
                job.error = f"footprint {fp} B exceeds the HBM budget {self.budget:.0f} B"
                pending.pop(0)
                continue
            if self.used + fp > self.budget:
                break                      # head of line waits until memory frees up
            pending.pop(0)
            try:
                handle = self.backend.create(job)
            except Exception as e:       # the job fails, the server carries on
                job.state = "failed"
                job.error = f"admission: {e}"
                continue
            job.state = "running"
            job.admitted_at = self.clock() - self._t0
            self.used += fp
            self.peak_used = max(self.peak_used, self.used)
            self.active.append((job, handle, fp))
            changed = True
        return changed

    def _retire(self, keep_if) -> bool:
        changed = False
        still = []
        for job, handle, fp in self.active:
            if keep_if(job):
                still.append((job, handle, fp))
                continue
            if job.state == "running" and job.steps_done >= job.steps:
                try:
                    job.result = self.backend.result(handle)
                    job.state = "done"
                except Exception as e:
                    job.state = "failed"
                    job.error = f"read-out: {e}"
            job.finished_at = self.clock() - self._t0
            self.backend.free(handle)
            self.used -= fp
            changed = True
        self.active = still
        return changed

    def run(self, jobs: list) -> dict:
        pending = sorted(jobs, key=lambda j: (j.arrival, j.id))
        self._t0 = self.clock()
        batch = None
        members: list = []                # the jobs inside the current batch, in member order
        dirty = True
        while pending or self.active:
            dirty |= self._admit(pending, self.clock() - self._t0)
            # cancellations take effect at the chunk boundary
            for job, _, _ in self.active:
                if job.id in self.cancel_requests and job.state == "running":
                    job.state = "cancelled"
            dirty |= self._retire(lambda j: j.state == "running")
            if not self.active:
                if pending:
                    self.sleep(max(0.0, min(0.01, pending[0].arrival - (self.clock() - self._t0))))
                continue
            if dirty:
                if batch is not None:
                    self.backend.free_batch(batch)
                batch = self.backend.make_batch([h for _, h, _ in self.active])
                members = [j for j, _, _ in self.active]
                self.rebuilds += 1
                dirty = False
            n = min(min(j.steps - j.steps_done for j in members), self.chunk_steps)
            try:
                self.backend.step(batch, n)
                # arrivals during the chunk are created now: their uploads overlap
                # the GPU work, and they join the batch at the next boundary
                dirty |= self._admit(pending, self.clock() - self._t0)
                self.backend.wait(batch)
            except Exception as e:
                # Members evolve independently: when the batch can say which
                # members latched an error, only those fail and the others keep
                # the completed chunk; otherwise the whole chunk fails.
                bad = self._member_errors(batch)
                for k, job in enumerate(members):
                    if bad and k not in bad:
                        job.steps_done += n
                    elif job.state == "running":
                        job.state = "failed"
                        job.error = f"chunk: {e}" if not bad else f"chunk: member error {bad[k]} ({e})"
                self.backend.free_batch(batch)
                batch = None
                members = []
                self._retire(lambda j: j.state == "running" and j.steps_done < j.steps)
                dirty = True
                continue
            self.chunks += 1
            for job in members:
                job.steps_done += n
            dirty |= self._retire(lambda j: j.state == "running" and j.steps_done < j.steps)
        if batch is not None:
            self.backend.free_batch(batch)
        return self.stats(jobs)

    def _member_errors(self, batch) -> dict:
        if not hasattr(self.backend, "member_errors"):
            return {}
        try:
            return self.backend.member_errors(batch)
        except Exception:
            return {}

    def stats(self, jobs: list) -> dict:
        done = [j for j in jobs if j.state == "done"]
        lat = sorted(j.latency for j in done)
        work = sum(j.site_steps for j in done)
        if done:
            span = max(j.finished_at for j in done) - min(j.arrival for j in done)
        else:
            span = 0.0
        return {
            "jobs": len(jobs), "done": len(done),
            "rejected": sum(j.state == "rejected" for j in jobs),
            "cancelled": sum(j.state == "cancelled" for j in jobs),
            "failed": sum(j.state == "failed" for j in jobs),
            "p50_latency_s": percentile(lat, 50), "p99_latency_s": percentile(lat, 99),
            "aggregate_gsite_updates_per_s": work / span / 1e9 if span > 0 else None,
            "span_s": span, "chunks": self.chunks, "batch_rebuilds": self.rebuilds,
            "peak_hbm_bytes": self.peak_used, "budget_bytes": self.budget,
            "errors": [[j.id, j.state, j.error] for j in jobs if j.error],
        }


def percentile(sorted_vals: list, p: float):
    """Nearest-rank percentile of an ascending list (None if empty)."""
    if not sorted_vals:
        return None
    k = max(0, min(len(sorted_vals) - 1, math.ceil(p / 100.0 * len(sorted_vals)) - 1))
    return float(sorted_vals[k])


def poisson_arrivals(n: int, rate: float, seed: int = 4) -> list:
    rng = np.random.default_rng(seed)
    return list(np.cumsum(rng.exponential(1.0 / rate, size=n)))


def fifo_sequential_latencies(jobs: list, seconds_per_job: list) -> dict:
    """Latencies of running the same jobs one at a time, first come first served."""
    t = 0.0
    lat = []
    work = 0
    for job, sec in sorted(zip(jobs, seconds_per_job), key=lambda x: x[0].arrival):
        start = max(t, job.arrival)
        t = start + sec
        lat.append(t - job.arrival)
        work += job.site_steps
    lat.sort()
    span = t - min(j.arrival for j in jobs)
    return {"p50_latency_s": percentile(lat, 50), "p99_latency_s": percentile(lat, 99),
            "aggregate_gsite_updates_per_s": work / span / 1e9 if span > 0 else None, "span_s": span}


def _measure_capacity(backend, jobs, steps: int = 20) -> float:
    """Batched throughput (site-updates/s) of all the jobs' lattices stepped together."""
    torch = backend.torch
    handles = [backend.create(j) for j in jobs]
    batch = backend.make_batch(handles)
    batch.step(3)
    batch.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(backend.stream)
    batch.step(steps)
    e1.record(backend.stream)
    e1.synchronize()
    batch.close()
    for h in handles:
        h.close()
    return sum(workloads.sites(j.spec) for j in jobs) * steps / (e0.elapsed_time(e1) / 1e3)


def _fp64_seconds_per_step(backend, jobs, steps: int = 10) -> dict:
    """Plain FP64 single-lattice path: seconds per step for each distinct lattice shape."""
    from . import capi
    torch = backend.torch
    out = {}
    for j in jobs:
        key = (j.spec["dims"], j.spec["N"])
        if key in out:
            continue
        with capi.Simulation(**workloads.sim_kwargs(j.spec, "f64"), stream=backend.stream.cuda_stream) as sim:
            sim.set_fields(j.f0, j.u0)
            sim.step(3)
            sim.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(backend.stream)
            sim.step(steps)
            e1.record(backend.stream)
            e1.synchronize()
            out[key] = e0.elapsed_time(e1) / 1e3 / steps
    return out


def _fp64_job_seconds(backend, jobs) -> list:
    """Each job run alone on the plain FP64 single-lattice path, start to result:
    handle creation and upload, all of its steps, and the same read-out a
    served job gets (energies, means and variances); wall-clock seconds."""
    from . import capi
    out = []
    for j in sorted(jobs, key=lambda x: (x.arrival, x.id)):
        t0 = time.perf_counter()
        with capi.Simulation(**workloads.sim_kwargs(j.spec, "f64"), stream=backend.stream.cuda_stream) as sim:
            sim.set_fields(j.f0, j.u0)
            sim.step(j.steps)
            sim.energy()
            sim.means_variances()
        out.append((j.id, time.perf_counter() - t0))
    by_id = dict(out)
    return [by_id[j.id] for j in jobs]


def run_serving_benchmark(n_jobs: int = 40, load: float = 0.8, budget_gb: float = 150.0, chunk: int = 256,
                          seed: int = 4, capacity: float | None = None, fp64_baseline: str = "measured") -> dict:
    """Poisson arrivals of jobs from the mixed workload (plus 5% 3D 512^3), served
    with continuous batching; p50/p99 job latency and aggregate throughput, beside
    the same jobs run one at a time, first come first served, on the plain FP64
    path.  fp64_baseline "measured": every job is run alone on the FP64 path and
    its start-to-result time measured; the FIFO queue over the same arrival
    times is then exact arithmetic on those durations (one job at a time, so a
    job starts when it has arrived and the previous one has finished).  "model":
    durations from measured per-step times of each lattice shape."""
    specs = workloads.serving_job_specs(n_jobs, seed=seed)
    jobs = [Job(k, sp, sp["steps"], 0.0) for k, sp in enumerate(specs)]
    for j in jobs:
        j.f0, j.u0 = workloads.make_ics(j.spec)
    backend = GpuBackend("f32")
    if not capacity:
        capacity = _measure_capacity(backend, jobs)
    mean_work = float(np.mean([j.site_steps for j in jobs]))
    rate = load * capacity / mean_work
    for j, t in zip(jobs, poisson_arrivals(n_jobs, rate, seed)):
        j.arrival = float(t)
    server = Server(backend, budget_gb * 1e9, chunk)
    stats = server.run(jobs)
    if fp64_baseline == "measured":
        durations = _fp64_job_seconds(backend, jobs)
        kind = ("measured: every job run alone on the plain FP64 path (create, upload, all steps, read-out; "
                "wall clock), FIFO over the same arrival times")
    else:
        t64 = _fp64_seconds_per_step(backend, jobs)
        durations = [j.steps * t64[(j.spec["dims"], j.spec["N"])] for j in jobs]
        kind = ("model: same arrivals, one job at a time on the plain FP64 path; durations from measured "
                "per-step times of each lattice shape")
    baseline = fifo_sequential_latencies(jobs, durations)
    baseline["job_seconds"] = [round(d, 4) for d in durations]
    return {"serving": stats, "arrival_rate_per_s": rate, "offered_load": load,
            "capacity_gsite_updates_per_s": capacity / 1e9, "chunk_steps": chunk,
            "jobs_512cube": sum(j.spec["N"] == 512 for j in jobs),
            "fp64_sequential_fifo": baseline, "fp64_baseline_kind": kind,
            "p50_over_fp64": (baseline["p50_latency_s"] / stats["p50_latency_s"]
                              if stats["p50_latency_s"] else None),
            "p99_over_fp64": (baseline["p99_latency_s"] / stats["p99_latency_s"]
                              if stats["p99_latency_s"] else None)}


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--jobs", type=int, default=40)
    ap.add_argument("--load", type=float, default=0.8)
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--chunk", type=int, default=256)
    ap.add_argument("--seed", type=int, default=4)
    ap.add_argument("--fp64-baseline", default="measured", choices=["measured", "model"])
    args = ap.parse_args(argv)
    from . import build
    build.build()
    print(json.dumps(run_serving_benchmark(args.jobs, args.load, args.budget_gb, args.chunk, args.seed,
                                           fp64_baseline=args.fp64_baseline)), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
