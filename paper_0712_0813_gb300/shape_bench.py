"""Per-shape timings of the batched kernel and of the single-lattice kernels.

``python -m paper_0712_0813_gb300.shape_bench`` prints one JSON line per case:

* ``mix_class``: the 96-lattice mixed batch (``workloads.mixed_batch_specs``)
  and its 1D, 2D and 3D parts alone, one ``k_step_batched`` launch per step;
* ``batch_3d``: homogeneous batches of about 100 M sites of one 3D side;
* ``single``: one lattice stepped by ``ce_step`` with the generic kernel and
  with the row kernel (``CE_KERNEL_ROWS``, the automatic FP32 choice for 2D
  sides >= 512 and 3D sides >= 64 outside the z-sweep kernel; in FP64 the
  automatic choice is the generic kernel, which runs two passes in 2D/3D).

Times are CUDA events on the library's stream around ``steps`` steps after
``warmup`` steps (graphs of 32 launches); ``frac`` is the algorithmic 16 B per
field and site of FP32 storage divided by the time and the measured HBM
bandwidth.  2 fields, FP32 storage, expansion on for the synthetic cases.
"""
from __future__ import annotations

import argparse
import json
import os

from . import capi, workloads
from .icgen import courant_dt, lattice_ics


def _peak_gbs() -> float:
    here = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    try:
        with open(os.path.join(here, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


def _timed(torch, stream, fn_step, steps: int, warmup: int) -> float:
    fn_step(warmup)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fn_step(steps)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / steps * 1e3        # us per step


def _batch_row(torch, stream, sims, sites, item_lengths, steps, warmup, peak):
    out = {}
    for L in item_lengths:
        with capi.Batch(sims, sweep_len=L, stream=stream.cuda_stream) as b:
            us = _timed(torch, stream, b.step, steps, warmup)
            items = b.info["items"]
            b.synchronize()
        out[f"L{L}"] = {"us": us, "gsite_per_s": sites / us / 1e3, "frac": 32.0 * sites / us / 1e3 / peak,
                        "items": items}
    return out


def run(steps: int = 100, warmup: int = 20, item_lengths=(64, 128)) -> list:
    import torch
    peak = _peak_gbs()
    stream = torch.cuda.Stream()
    rows = []
    specs = workloads.mixed_batch_specs()
    ics = [workloads.make_ics(sp) for sp in specs]
    groups = {"1d": [k for k, s in enumerate(specs) if s["dims"] == 1],
              "2d": [k for k, s in enumerate(specs) if s["dims"] == 2],
              "3d": [k for k, s in enumerate(specs) if s["dims"] == 3],
              "all": list(range(len(specs)))}
    for name, idx in groups.items():
        sims = []
        for k in idx:
            s = capi.Simulation(**workloads.sim_kwargs(specs[k], "f32"), kernel="generic")
            s.set_fields(*ics[k])
            sims.append(s)
        sites = sum(workloads.sites(specs[k]) for k in idx)
        row = {"case": "mix_class", "class": name, "lattices": len(idx), "sites": sites}
        row.update(_batch_row(torch, stream, sims, sites, item_lengths, steps, warmup, peak))
        rows.append(row)
        print(json.dumps(row), flush=True)
        for s in sims:
            s.close()
    for N, count in ((64, 384), (96, 113), (128, 48), (160, 24), (192, 14)):
        f0, u0 = lattice_ics(3, N, 20.0, 2, q=(1.2,), seed=3, amp=1e-2,
                             backend="torch" if N ** 3 >= 1 << 22 else "numpy")
        dt = courant_dt(3, N, 20.0, 1.0, (1.2,))
        sims = []
        for _ in range(count):
            s = capi.Simulation(dims=3, N=N, L=20.0, dt=dt, nfields=2, q=(1.2,), expansion=True,
                                precision="f32", kernel="generic")
            s.set_fields(f0, u0)
            sims.append(s)
        sites = count * N ** 3
        row = {"case": "batch_3d", "N": N, "lattices": count, "sites": sites}
        row.update(_batch_row(torch, stream, sims, sites, item_lengths, steps, warmup, peak))
        rows.append(row)
        print(json.dumps(row), flush=True)
        for s in sims:
            s.close()
    for dims, N in ((1, 65536), (2, 1024), (2, 6000), (3, 64), (3, 96), (3, 160), (3, 192), (3, 288), (3, 448)):
        big = N ** dims >= 1 << 22
        f0, u0 = lattice_ics(dims, N, 20.0, 2, q=(1.2,), seed=3, amp=1e-2, backend="torch" if big else "numpy")
        dt = courant_dt(dims, N, 20.0, 1.0, (1.2,))
        row = {"case": "single", "dims": dims, "N": N}
        for prec in ("f32", "f64"):
            for kern in ("generic", "rows"):
                with capi.Simulation(dims=dims, N=N, L=20.0, dt=dt, nfields=2, q=(1.2,), expansion=True,
                                     precision=prec, kernel=kern, stream=stream.cuda_stream) as s:
                    s.set_fields(f0, u0)
                    n = max(10, min(2 * steps, int(2e9 / (N ** dims * 8 * (4 if prec == "f32" else 8)))))
                    row[f"{prec}_{kern}_us"] = _timed(torch, stream, s.step, n, min(2 * warmup, n))
        rows.append(row)
        print(json.dumps(row), flush=True)
    return rows


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=20)
    args = ap.parse_args(argv)
    run(args.steps, args.warmup)


if __name__ == "__main__":
    main()
