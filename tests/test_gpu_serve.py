"""Serving loop on the GPU: jobs arriving over time are admitted into the
running batch (continuous batching) and every job's final state is
bit-identical to the same job advanced alone (batch of one) for the same number
of steps, with and without a budget tight enough to make jobs queue."""
import numpy as np
import pytest

from paper_0712_0813_gb300 import workloads
from paper_0712_0813_gb300.icgen import courant_dt
from paper_0712_0813_gb300.serve import GpuBackend, Job, Server

pytestmark = pytest.mark.gpu

SHAPES = [(3, 32), (3, 48), (2, 128), (1, 4096), (3, 24), (2, 64)]


def jobs_for(n, seed=0):
    rng = np.random.default_rng(seed)
    jobs = []
    for k in range(n):
        dims, N = SHAPES[k % len(SHAPES)]
        q = float(rng.uniform(0.5, 20.0))
        phi0 = float(rng.uniform(0.5, 1.5))
        sp = {"dims": dims, "N": N, "L": 20.0, "nf": 2, "q": (q,), "phi0": phi0,
              "dt": courant_dt(dims, N, 20.0, phi0, (q,)), "expansion": k % 2 == 0, "seed": 500 + k}
        j = Job(k, sp, int(rng.integers(40, 160)), arrival=0.004 * k)
        j.f0, j.u0 = workloads.make_ics(sp)
        jobs.append(j)
    return jobs


@pytest.mark.parametrize("budget_jobs", [100, 2])
def test_served_jobs_match_running_alone(gpu_capi, budget_jobs):
    capi = gpu_capi
    jobs = jobs_for(9)
    be = GpuBackend("f32", keep_fields=True)
    budget = budget_jobs * max(be.footprint(j.spec) for j in jobs)
    server = Server(be, hbm_budget=budget, chunk_steps=16)
    st = server.run(jobs)
    assert st["done"] == len(jobs), [(j.id, j.state, j.error) for j in jobs]
    assert st["p50_latency_s"] is not None and st["p99_latency_s"] >= st["p50_latency_s"]
    assert st["peak_hbm_bytes"] <= budget and server.used == 0
    if budget_jobs == 2:
        assert st["batch_rebuilds"] >= len(jobs) // 2
    for j in jobs:
        assert j.result["step"] == j.steps
        with capi.Simulation(**workloads.sim_kwargs(j.spec, "f32"), kernel="generic") as sim:
            sim.set_fields(j.f0, j.u0)
            with capi.Batch([sim]) as b:
                b.step(j.steps)
            f, v, _ = sim.get_fields(capi.CE_VEL_STAGGERED)
        assert np.array_equal(f, j.result["f"]) and np.array_equal(v, j.result["v"]), j.id
