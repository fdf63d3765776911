"""Parity at the full benchmark sizes, on sampled sites.

The lattices of the benchmark workloads are too large to download and step on
the host (1024^3 x 2 fields is 17 GB per FP64 array, and the oracle needs about
a hundred seconds per step there), so one GPU step is checked site by site:

* the staggered state (f(t), v(t+dt/2)) is sampled on the GPU
  (`ce_sample_fields`) at a few thousand sites -- random ones plus every
  combination of tile edges, lattice edges and z-chunk boundaries of the launch
  plan -- and at their nearest neighbours;
* the GPU takes one step, and the new state is sampled at the sites;
* the oracle's per-site restatement of one step (`oracle/local.py`, pinned
  equal to `orc_step` on whole lattices) computes the new state from the first
  sample.  The step's global sums G and V (they enter only the scale factor)
  come from the oracle too: `local.drifted_sums` (pinned equal to the C
  oracle's sums) streams the whole lattice's state before the step, a slab of
  z-planes at a time, and sums the gradient and potential energy of the
  drifted fields f + dt v in FP64.  No oracle input comes from a GPU output
  other than the sampled state being checked.

Workloads and launch plans are the ones the benchmark times: 3D 256^3, 2
fields, dt = 0.02 (plan 8 rows / 4 stages / 4 z-chunks); 3D 512^3, 4 fields,
q = (0.8, 5, 40) (plan 8 / 5 / 8); 3D 1024^3, 2 fields (the automatic plan,
then 16 / 4 / 8 on the same state); all FP32 storage with expansion; and the
96-lattice mixed batch (FP32, batched kernel, the item length the bench's
autotuner picks); and the odd sides 511^3 (column kernel) and 16001^2 (line-sweep
kernel) on the automatic choice.  Tolerances: f and v
within an error bound of one FP32 step derived from the arithmetic
(`check_one_step`; on the finest lattices the Laplacian's 1/dx^2 weights make
the FP32 rounding of g the dominant term), a(t) to 1e-12, and a', a'' to 1e-5
of the source term Q (FP32 partial sums of the fused kernel against FP64
sums).
"""
import gc

import numpy as np
import pytest

from paper_0712_0813_gb300.icgen import courant_dt, lattice_ics
from step_bounds import EPS64, check_one_step

pytestmark = pytest.mark.gpu

KAPPA2 = 8.0 * np.pi / 3.0 * 0.342 ** 2


def relmax(a, b):
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / (den if den > 0 else 1.0))


def plan_sites(N, tx, ty, zchunks, n_random=3000, seed=11):
    """Random sites plus every combination of tile, lattice and z-chunk edges."""
    xs = sorted({0, 1, tx - 1, tx, tx + 1, N // 2, N - tx, N - 2, N - 1})
    ys = sorted({0, 1, ty - 1, ty, N // 2, N - ty, N - 1})
    zb = {0, 1, N - 2, N - 1}
    for j in range(1, zchunks):
        z = j * N // zchunks
        zb |= {z - 1, z, z + 1}
    xx, yy, zz = np.meshgrid(np.array(xs), np.array(ys), np.array(sorted(zb)), indexing="ij")
    edges = (xx + N * yy + N * N * zz).reshape(-1)
    rng = np.random.default_rng(seed)
    rand = rng.integers(0, N ** 3, size=n_random)
    return np.unique(np.concatenate([edges, rand]).astype(np.int64))


def oracle_sums(local, p, sim):
    """G and V of the drifted fields f + dt v over the whole lattice, computed
    by the oracle (`local.drifted_sums`) from the lattice's current staggered
    state, read a slab of hyperplanes of the slowest axis (about 16 M sites)
    at a time."""
    plane = p.N ** (p.dims - 1)
    slab = max(1, (1 << 24) // plane)
    rest = (p.N,) * (p.dims - 1)

    def read(k0, k1):
        f, v, _ = sim.sample_fields(np.arange(k0 * plane, k1 * plane, dtype=np.int64))
        return f.reshape((p.nf, k1 - k0) + rest), v.reshape((p.nf, k1 - k0) + rest)

    G, V, _ = local.drifted_sums(p, read, slab=max(1, min(slab, p.N)))
    return G, V


SINGLE = [
    # name, N, nf, q, dt (None: Courant rule), plans (rows, stages, zchunks; 0 = automatic)
    ("256cube", 256, 2, (1.2,), 0.02, [(8, 4, 4)]),
    ("512cube_4field", 512, 4, (0.8, 5.0, 40.0), None, [(8, 5, 8)]),
    ("1024cube", 1024, 2, (1.2,), None, [(0, 0, 0), (16, 4, 8)]),
]


@pytest.mark.parametrize("name,N,nf,q,dt,plans", SINGLE, ids=[c[0] for c in SINGLE])
def test_full_size_sampled_step(gpu_capi, orc, name, N, nf, q, dt, plans):
    import torch
    from oracle import local
    capi = gpu_capi
    L = 20.0
    if dt is None:
        dt = courant_dt(3, N, L, 1.0, q)
    p = orc.Params(dims=3, N=N, L=L, dt=dt, nf=nf, q=q, expansion=True)
    f0, u0 = lattice_ics(3, N, L, nf, q=q, seed=1, backend="torch" if N >= 512 else "numpy")
    torch.cuda.empty_cache()
    rows, stages, zchunks = plans[0]
    with capi.Simulation(dims=3, N=N, L=L, dt=dt, nfields=nf, q=q, expansion=True, precision="f32",
                         kernel="sweep", tile_rows=rows, stages=stages, zchunks=zchunks) as sim:
        sim.set_fields(f0, u0)
        del f0, u0
        gc.collect()
        sim.step(3)
        for k, plan in enumerate(plans):
            if k:
                sim.replan(*plan)
            used = sim.sweep_plan
            assert all(want in (0, got) for want, got in zip(plan, used))
            sites = plan_sites(N, 128, used[0], used[2])
            stencil = local.stencil_sites(3, N, sites)
            before = sim.sample_fields(stencil)
            G, V = oracle_sums(local, p, sim)
            sim.step(1)
            after = sim.sample_fields(sites)
            check_one_step(orc, local, p, before, after, sites, stencil, G, V)
            assert after[2].step == 4 + k


# The column kernel (3D) and the line-sweep kernel (2D) at the largest odd sides
# timed in the profiles, on the automatic choice: 30-site strips in x, 6-row
# groups in 3D, chunks along the sweep axis (z in 3D, y in 2D) of the length the
# wave model picks on GB300 (511^3: 73 planes; 16001^2: 471 rows), FP32 storage
# with expansion.
ODD = [("511cube", 3, 511, 73), ("16001sq", 2, 16001, 471)]


def odd_sites(dims, N, chunk, n_random=20000, seed=12):
    """Random sites plus every combination of strip edges, row-group edges,
    chunk boundaries along the sweep axis and lattice edges."""
    last = 30 * ((N - 1) // 30)
    xs = {0, 1, 29, 30, 31, 59, 60, N // 2, last - 1, last, last + 1, N - 2, N - 1}
    sweep = {0, 1, N // 2, N - 2, N - 1}
    for k in range(1, (N + chunk - 1) // chunk):
        sweep |= {k * chunk - 1, k * chunk, k * chunk + 1}
    if dims == 3:
        ys = {0, 1, 5, 6, 7, 11, 12, N // 2, N - 7, N - 6, N - 2, N - 1}
        axes = [sorted(x for x in xs if x < N), sorted(y for y in ys if y < N), sorted(z for z in sweep if z < N)]
    else:
        axes = [sorted(x for x in xs if x < N), sorted(y for y in sweep if y < N)]
    grid = np.meshgrid(*[np.array(a, dtype=np.int64) for a in axes], indexing="ij")
    edges = sum(g * N ** d for d, g in enumerate(grid)).reshape(-1)
    rng = np.random.default_rng(seed)
    rand = rng.integers(0, N ** dims, size=n_random)
    return np.unique(np.concatenate([edges, rand]).astype(np.int64))


@pytest.mark.parametrize("precision", ["f32", "f64"])
@pytest.mark.parametrize("name,dims,N,chunk", ODD, ids=[c[0] for c in ODD])
def test_full_size_odd_side_sampled_step(gpu_capi, orc, name, dims, N, chunk, precision):
    """FP32: the column / line-sweep kernel (the automatic choice); FP64: the
    automatic FP64 choice on the same lattice (the generic kernel's two passes),
    within FP64 bounds of one step and a'' to 1e-10 of its source term."""
    import torch
    from oracle import local
    capi = gpu_capi
    L, nf, q = 20.0, 2, (1.2,)
    dt = courant_dt(dims, N, L, 1.0, q)
    p = orc.Params(dims=dims, N=N, L=L, dt=dt, nf=nf, q=q, expansion=True)
    f0, u0 = lattice_ics(dims, N, L, nf, q=q, seed=1, backend="torch")
    torch.cuda.empty_cache()
    with capi.Simulation(dims=dims, N=N, L=L, dt=dt, nfields=nf, q=q, expansion=True, precision=precision) as sim:
        assert sim.kernel == (capi.CE_KERNEL_PLANES if precision == "f32" else capi.CE_KERNEL_GENERIC)
        sim.set_fields(f0, u0)
        del f0, u0
        gc.collect()
        sim.step(3)
        sites = odd_sites(dims, N, chunk)
        stencil = local.stencil_sites(dims, N, sites)
        before = sim.sample_fields(stencil)
        G, V = oracle_sums(local, p, sim)
        sim.step(1)
        after = sim.sample_fields(sites)
        if precision == "f32":
            check_one_step(orc, local, p, before, after, sites, stencil, G, V)
        else:
            check_one_step(orc, local, p, before, after, sites, stencil, G, V, eps=EPS64, sums_rel=1e-10)
        assert after[2].step == 4


def test_mixed_batch_sampled_step(gpu_capi, orc):
    """The 96-lattice mix of the batched benchmark leg, one batched launch per
    step at the autotuned item length: every member checked on sampled sites."""
    import torch
    from oracle import local
    from paper_0712_0813_gb300 import autotune, workloads
    capi = gpu_capi
    specs = workloads.mixed_batch_specs()
    sims = []
    for sp in specs:
        s = capi.Simulation(**workloads.sim_kwargs(sp, "f32"), kernel="generic")
        s.set_fields(*workloads.make_ics(sp))
        sims.append(s)
    stream = torch.cuda.Stream()
    tune = autotune.autotune_batch(sims, stream=stream, steps=4, warmup=1)
    rng = np.random.default_rng(17)
    picks, befores, sums = [], [], []
    with capi.Batch(sims, sweep_len=tune["sweep_len"], stream=stream.cuda_stream) as b:
        b.step(2)
        b.synchronize()
        for sp, s in zip(specs, sims):
            S = workloads.sites(sp)
            n = min(S, 400)
            edge = np.array([0, 1, sp["N"] - 1, S - 1, S // 2], dtype=np.int64)
            sites = np.unique(np.concatenate([edge, rng.integers(0, S, size=n)]))
            stencil = local.stencil_sites(sp["dims"], sp["N"], sites)
            picks.append((sites, stencil))
            befores.append(s.sample_fields(stencil))
            p = orc.Params(dims=sp["dims"], N=sp["N"], L=sp["L"], dt=sp["dt"], nf=sp["nf"], q=sp["q"],
                           expansion=sp["expansion"])
            sums.append(oracle_sums(local, p, s))
        b.step(1)
        b.synchronize()
    for sp, s, (sites, stencil), before, (G, V) in zip(specs, sims, picks, befores, sums):
        after = s.sample_fields(sites)
        p = orc.Params(dims=sp["dims"], N=sp["N"], L=sp["L"], dt=sp["dt"], nf=sp["nf"], q=sp["q"],
                       expansion=sp["expansion"])
        check_one_step(orc, local, p, before, after, sites, stencil, G, V)
        s.close()


def test_full_size_1024cube_fp64_sampled_step(gpu_capi, orc):
    """The bench's FP64 leg: 3D 1024^3, 2 fields, expansion, FP64 storage (68.7 GB)
    on the automatic FP64 choice (the generic kernel's two passes), one step
    checked at sampled sites against the oracle's per-site step, with the G and
    V of the drifted fields summed by the oracle over the whole lattice; bounds
    of one step in FP64 (EPS64), a'' to 1e-10 of its source term."""
    import torch
    from oracle import local
    capi = gpu_capi
    N, nf, q, L = 1024, 2, (1.2,), 20.0
    dt = courant_dt(3, N, L, 1.0, q)
    p = orc.Params(dims=3, N=N, L=L, dt=dt, nf=nf, q=q, expansion=True)
    f0, u0 = lattice_ics(3, N, L, nf, q=q, seed=1, backend="torch")
    torch.cuda.empty_cache()
    with capi.Simulation(dims=3, N=N, L=L, dt=dt, nfields=nf, q=q, expansion=True, precision="f64") as sim:
        assert sim.kernel == capi.CE_KERNEL_GENERIC
        sim.set_fields(f0, u0)
        del f0, u0
        gc.collect()
        sim.step(3)
        sites = plan_sites(N, 64, 8, 4)
        stencil = local.stencil_sites(3, N, sites)
        before = sim.sample_fields(stencil)
        G, V = oracle_sums(local, p, sim)
        sim.step(1)
        after = sim.sample_fields(sites)
    check_one_step(orc, local, p, before, after, sites, stencil, G, V, eps=EPS64, sums_rel=1e-10)
    assert after[2].step == 4
