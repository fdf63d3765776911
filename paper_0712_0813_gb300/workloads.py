"""Seeded synthetic workload mixes (lattice specifications, no evolution arithmetic).

`mixed_batch_specs` is the mixed-size batch: 32 1D lattices of N = 65536, 32 2D
lattices of 1024^2 and 32 3D lattices with side drawn uniformly from
{64, 96, 128, 160, 192}; each lattice draws q log-uniform in [0.5, 200] and
phi0 uniform in [0.5, 2], takes dt from its own Courant limit
(`icgen.courant_dt` with the masses at 4 phi0: with q up to 200 and 2000-20000
steps, phi reaches about 3.4 phi0 locally and a step sized at phi0 lets the
leapfrog go unstable at the largest fluctuation), has expansion on for even
indices, box L = 20, two fields.
`serving_job_specs` draws jobs for the serving loop from the same mix plus 5%
3D 512^3 lattices (round(5% of the jobs), at least one from 10 jobs up, at
seeded positions), with 2000-20000 steps each.
"""
from __future__ import annotations

import math

import numpy as np

from .icgen import courant_dt, lattice_ics

L_BOX = 20.0
AMP_MARGIN = 4.0   # largest local |phi| / phi0 the Courant rule allows for


def _spec(rng, dims: int, N: int, index: int, seed: int) -> dict:
    q = float(math.exp(rng.uniform(math.log(0.5), math.log(200.0))))
    phi0 = float(rng.uniform(0.5, 2.0))
    return {"dims": dims, "N": N, "L": L_BOX, "nf": 2, "q": (q,), "phi0": phi0,
            "dt": courant_dt(dims, N, L_BOX, phi0, (q,), amp=AMP_MARGIN), "expansion": index % 2 == 0,
            "seed": seed * 1000 + index}


def mixed_batch_specs(seed: int = 3, n_per_kind: int = 32, sides=(64, 96, 128, 160, 192)) -> list:
    rng = np.random.default_rng(seed)
    specs = []
    for k in range(3 * n_per_kind):
        kind = k // n_per_kind
        if kind == 0:
            dims, N = 1, 65536
        elif kind == 1:
            dims, N = 2, 1024
        else:
            dims, N = 3, int(rng.choice(sides))
        specs.append(_spec(rng, dims, N, k, seed))
    return specs


def serving_job_specs(n_jobs: int, seed: int = 4, big_fraction: float = 0.05,
                      steps_range=(2000, 20000), big_side: int = 512) -> list:
    rng = np.random.default_rng(seed)
    base = mixed_batch_specs(seed=seed)
    n_big = int(round(big_fraction * n_jobs))
    if n_jobs >= 10:
        n_big = max(1, n_big)
    big = set(rng.choice(n_jobs, size=n_big, replace=False).tolist()) if n_big else set()
    jobs = []
    for j in range(n_jobs):
        if j in big:
            spec = _spec(rng, 3, big_side, j, seed + 100)
        else:
            spec = dict(base[int(rng.integers(len(base)))])
            spec["seed"] = seed * 100000 + j
        spec["steps"] = int(rng.integers(steps_range[0], steps_range[1] + 1))
        jobs.append(spec)
    return jobs


def sites(spec: dict) -> int:
    return spec["N"] ** spec["dims"]


def state_bytes(spec: dict, precision: str = "f32") -> int:
    """Device bytes of one lattice's state: f and the velocity state, ping-ponged."""
    es = 4 if precision == "f32" else 8
    return 4 * spec["nf"] * sites(spec) * es


def make_ics(spec: dict):
    big = sites(spec) >= 1 << 24
    return lattice_ics(spec["dims"], spec["N"], spec["L"], spec["nf"], phi0=spec["phi0"], q=spec["q"],
                       seed=spec["seed"], backend="torch" if big else "numpy")


def sim_kwargs(spec: dict, precision: str = "f32") -> dict:
    return dict(dims=spec["dims"], N=spec["N"], L=spec["L"], dt=spec["dt"], nfields=spec["nf"], q=spec["q"],
                expansion=spec["expansion"], phi0=spec["phi0"], precision=precision)
