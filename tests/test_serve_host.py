"""Serving loop logic on the host (no GPU): admission under the HBM budget,
first-come first-served order, rejection, cancellation, a failure injected in
the backend, and the latency statistics."""
import pytest

from paper_0712_0813_gb300.serve import Job, Server, fifo_sequential_latencies, percentile


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-4)


class FakeBackend:
    def __init__(self, clock, step_cost=1e-3, fail_chunk=None):
        self.clock = clock
        self.step_cost = step_cost
        self.fail_chunk = fail_chunk
        self.chunk = 0
        self.batches = []
        self.freed = []

    def footprint(self, spec):
        return spec["bytes"]

    def create(self, job):
        if job.spec.get("fail_create"):
            raise RuntimeError("device allocation failed")
        return {"id": job.id, "steps": 0}

    def make_batch(self, handles):
        self.batches.append([h["id"] for h in handles])
        return list(handles)

    def free_batch(self, batch):
        pass

    def step(self, batch, n):
        self.chunk += 1
        if self.fail_chunk is not None and self.chunk == self.fail_chunk:
            raise RuntimeError("injected device error")
        for h in batch:
            h["steps"] += n
        self.clock.t += n * self.step_cost

    def wait(self, batch):
        if any(h.get("status") for h in batch):
            raise RuntimeError("a member reported non-finite sums")

    def member_errors(self, batch):
        return {k: h["status"] for k, h in enumerate(batch) if h.get("status")}

    def result(self, h):
        return {"steps": h["steps"]}

    def free(self, h):
        self.freed.append(h["id"])


def spec(nbytes, **kw):
    d = {"dims": 3, "N": 8, "nf": 2, "bytes": nbytes}
    d.update(kw)
    return d


def make_jobs(n, steps=100, gap=0.01, nbytes=10):
    return [Job(k, spec(nbytes), steps + 7 * k, arrival=gap * k) for k in range(n)]


def test_every_job_runs_exactly_its_steps_and_latency_is_measured():
    clock = FakeClock()
    be = FakeBackend(clock)
    jobs = make_jobs(12)
    st = Server(be, hbm_budget=1000, chunk_steps=32, clock=clock, sleep=clock.sleep).run(jobs)
    assert st["done"] == 12 and st["failed"] == 0
    for j in jobs:
        assert j.result["steps"] == j.steps           # newcomers never advance in a chunk they were not in
        assert j.latency >= j.steps * be.step_cost - 1e-9
    assert st["p50_latency_s"] <= st["p99_latency_s"]
    assert sorted(be.freed) == list(range(12))


def test_budget_is_never_exceeded_and_head_of_line_waits():
    clock = FakeClock()
    be = FakeBackend(clock)
    jobs = make_jobs(8, nbytes=40)
    server = Server(be, hbm_budget=100, chunk_steps=16, clock=clock, sleep=clock.sleep)
    st = server.run(jobs)
    assert st["done"] == 8
    assert st["peak_hbm_bytes"] <= 100
    assert max(len(b) for b in be.batches) <= 2        # only two 40-byte jobs fit
    admitted = sorted(jobs, key=lambda j: j.admitted_at)
    assert [j.id for j in admitted] == list(range(8))  # first come, first served
    assert server.used == 0


def test_oversized_job_is_rejected_others_complete():
    clock = FakeClock()
    be = FakeBackend(clock)
    jobs = make_jobs(4)
    jobs[1].spec = spec(10 ** 6)
    st = Server(be, hbm_budget=1000, clock=clock, sleep=clock.sleep).run(jobs)
    assert jobs[1].state == "rejected" and "exceeds" in jobs[1].error
    assert st["done"] == 3 and st["rejected"] == 1


def test_cancellation_before_admission_and_while_running():
    clock = FakeClock()
    be = FakeBackend(clock)
    jobs = make_jobs(5, steps=400)
    server = Server(be, hbm_budget=1000, chunk_steps=50, clock=clock, sleep=clock.sleep)
    server.cancel(4)                                   # never admitted
    orig_step = be.step

    def step_and_cancel(batch, n):
        orig_step(batch, n)
        if be.chunk == 2:
            server.cancel(0)                           # running: dropped at the next boundary
    be.step = step_and_cancel
    st = server.run(jobs)
    assert jobs[4].state == "cancelled" and jobs[4].admitted_at is None
    assert jobs[0].state == "cancelled" and 0 in be.freed
    assert st["done"] == 3 and st["cancelled"] == 2 and server.used == 0


def test_injected_backend_failure_fails_the_chunk_and_the_server_carries_on():
    clock = FakeClock()
    be = FakeBackend(clock, fail_chunk=2)
    jobs = make_jobs(3, steps=100, gap=0.0) + [Job(9, spec(10), 50, arrival=5.0)]
    st = Server(be, hbm_budget=1000, chunk_steps=20, clock=clock, sleep=clock.sleep).run(jobs)
    assert all(j.state == "failed" and "injected" in j.error for j in jobs[:3])
    assert jobs[3].state == "done" and jobs[3].result["steps"] == 50
    assert st["failed"] == 3 and st["done"] == 1


def test_member_error_fails_only_that_job():
    """A lattice that latches an error on the device (non-finite sums) fails
    alone: the other members of its batch keep the chunk and finish."""
    clock = FakeClock()
    be = FakeBackend(clock)
    jobs = make_jobs(4, steps=100, gap=0.0)
    orig_step = be.step

    def step_and_poison(batch, n):
        orig_step(batch, n)
        if be.chunk == 2:
            next(h for h in batch if h["id"] == 2)["status"] = -5
    be.step = step_and_poison
    st = Server(be, hbm_budget=1000, chunk_steps=20, clock=clock, sleep=clock.sleep).run(jobs)
    assert jobs[2].state == "failed" and "member error -5" in jobs[2].error
    for j in (jobs[0], jobs[1], jobs[3]):
        assert j.state == "done" and j.result["steps"] == j.steps
    assert st["failed"] == 1 and st["done"] == 3
    assert sorted(be.freed) == [0, 1, 2, 3]


def test_failed_admission_does_not_leak_budget():
    clock = FakeClock()
    be = FakeBackend(clock)
    jobs = make_jobs(3)
    jobs[0].spec = spec(10, fail_create=True)
    server = Server(be, hbm_budget=1000, clock=clock, sleep=clock.sleep)
    st = server.run(jobs)
    assert jobs[0].state == "failed" and st["done"] == 2 and server.used == 0


def test_percentile_and_fifo_baseline():
    assert percentile([], 50) is None
    vals = [1.0, 2.0, 3.0, 4.0]
    assert percentile(vals, 50) == 2.0 and percentile(vals, 99) == 4.0 and percentile(vals, 100) == 4.0
    jobs = [Job(0, spec(1), 10, 0.0), Job(1, spec(1), 10, 1.0), Job(2, spec(1), 10, 10.0)]
    r = fifo_sequential_latencies(jobs, [3.0, 3.0, 1.0])
    # job0: 0 -> 3 (3), job1: 3 -> 6 (5), job2: 10 -> 11 (1)
    assert r["p50_latency_s"] == 3.0 and r["p99_latency_s"] == 5.0 and r["span_s"] == 11.0
