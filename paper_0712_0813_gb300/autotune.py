"""Autotuner for the 3D z-sweep step kernel's launch plan.

The kernel is compiled in several variants (tile rows x TMA pipeline stages)
and splits each tile column into z-chunks; which combination streams HBM best
depends on the lattice size, the number of fields and the precision.  The
autotuner times each candidate on the caller's own lattice through the public
C ABI (one handle, ce_replan between candidates, ce_step timed with CUDA
events) and returns the fastest.  Results are cached per
(N, nfields, precision, expansion) for the process; `save`/`load` persist them.
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass, field

from . import capi

VARIANTS = ((8, 4), (8, 5), (16, 3), (16, 4), (4, 4), (4, 5))
_cache: dict = {}


@dataclass
class TuneResult:
    tile_rows: int
    stages: int
    zchunks: int
    ms_per_step: float
    table: list = field(default_factory=list)   # (tile_rows, stages, zchunks, ms_per_step)

    def hints(self) -> dict:
        return {"tile_rows": self.tile_rows, "stages": self.stages, "zchunks": self.zchunks}


def _key(N, nfields, precision, expansion):
    return f"N{N}_nf{nfields}_{precision}_{'exp' if expansion else 'flat'}"


def zchunk_candidates(N: int) -> list:
    if N >= 512:       # the grid is already many waves deep; a few short columns suffice
        base = [0, 1, 2, 4, 8, 16]
    else:
        base = [0, 4, 6, 8, 10, 12, 14, 16, 19, 24, 32, 38]
    return [z for z in base if z == 0 or z <= N // 2]


def tune_handle(sim, stream, N: int, *, steps: int = 40, warmup: int = 8, repeats: int = 2, zchunks=None,
                variants=VARIANTS) -> list:
    """Time every applicable (tile_rows, stages, zchunks) on an existing
    z-sweep handle (its state advances by the timed steps); returns the table
    (tile_rows, stages, zchunks, ms_per_step).  The handle is left on the
    last candidate: replan it to the chosen plan."""
    import torch
    table, seen = [], set()
    for rows, stages in variants:
        for zc in (zchunks if zchunks is not None else zchunk_candidates(N)):
            try:
                sim.replan(rows, stages, zc)
            except capi.CeError as e:
                if e.code == capi.CE_EINVAL:
                    continue          # this variant does not apply to the lattice
                raise
            plan = sim.sweep_plan
            if plan in seen:          # "automatic" may coincide with an explicit count
                continue
            seen.add(plan)
            sim.step(warmup)
            best = float("inf")
            for _ in range(repeats):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                sim.step(steps)
                e1.record(stream)
                e1.synchronize()
                best = min(best, e0.elapsed_time(e1) / steps)
            sim.synchronize()
            table.append((plan[0], plan[1], plan[2], best))
    if not table:
        raise capi.CeError(capi.CE_EINVAL, "no z-sweep variant applies to this lattice")
    return table


def autotune_sweep(f0, u0, *, N: int, L: float, dt: float, nfields: int, q, expansion: bool,
                   precision: str = "f32", phi0: float = 1.0, steps: int = 40, warmup: int = 8,
                   repeats: int = 2, zchunks=None, variants=VARIANTS, use_cache: bool = True) -> TuneResult:
    """Time every applicable (tile_rows, stages, zchunks) on the given 3D state.

    One handle holds the state; `ce_replan` switches its launch plan between
    candidates, so large lattices are uploaded once."""
    import torch
    key = _key(N, nfields, precision, expansion)
    if use_cache and key in _cache:
        return _cache[key]
    stream = torch.cuda.Stream()
    with capi.Simulation(dims=3, N=N, L=L, dt=dt, nfields=nfields, q=q, expansion=expansion, phi0=phi0,
                         precision=precision, kernel="sweep", stream=stream.cuda_stream) as sim:
        sim.set_fields(f0, u0)
        table = tune_handle(sim, stream, N, steps=steps, warmup=warmup, repeats=repeats, zchunks=zchunks,
                            variants=variants)
    r, s_, z, ms = min(table, key=lambda t: t[3])
    res = TuneResult(r, s_, z, ms, table)
    _cache[key] = res
    return res


def save(path: str):
    with open(path, "w") as fh:
        json.dump({k: {"tile_rows": v.tile_rows, "stages": v.stages, "zchunks": v.zchunks,
                       "ms_per_step": v.ms_per_step} for k, v in _cache.items()}, fh, indent=1)


def load(path: str):
    if not os.path.exists(path):
        return
    with open(path) as fh:
        for k, v in json.load(fh).items():
            _cache[k] = TuneResult(v["tile_rows"], v["stages"], v["zchunks"], v["ms_per_step"])


def autotune_batch(sims, *, candidates=(32, 64, 128, 256), occupancies=(0,), steps: int = 20,
                   warmup: int = 4, stream=None) -> dict:
    """Pick the batched kernel's item length (sites per item along the sweep
    axis) and, optionally, a cap on resident CTAs per SM for a set of handles:
    each candidate batch is timed for `steps` steps with CUDA events (the
    members' states advance; callers tune on a scratch copy or accept the
    extra steps)."""
    import torch
    st = torch.cuda.Stream() if stream is None else stream
    table = []
    for occ in occupancies:
        for L in candidates:
            with capi.Batch(sims, sweep_len=L, stream=st.cuda_stream, ctas_per_sm=occ) as b:
                b.step(warmup)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(st)
                b.step(steps)
                e1.record(st)
                e1.synchronize()
                b.synchronize()
                table.append((L, occ, e0.elapsed_time(e1) / steps))
    best = min(table, key=lambda t: t[2])
    return {"sweep_len": best[0], "ctas_per_sm": best[1], "ms_per_step": best[2], "table": table}
