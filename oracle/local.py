"""One oracle step evaluated at chosen sites (TEST INFRASTRUCTURE ONLY).

Restates, site by site and in the same order of operations, what ``orc_step``
(``clusterlat_oracle.c``; arXiv:0712.0813 Sec. III staggered leapfrog, readings
c-1..c-4) does to a state (f(t), v(t+dt/2), a(t), a'(t+dt/2)):

* drift  f <- f + dt v;
* scale  a <- a + dt a', then a' and a'' from the closed form of the implicit
  midpoint update with Q = kappa2 (2 G + 3 V) / a, where G and V are the mean
  gradient and potential energies of the new f (inputs here: a lattice of 10^9
  sites is not summed on the host; the caller supplies them);
* kick   v <- v + dt (lap f - dV/df + (a''/a) f).

The drift and the kick at a site read only the site and its 2 d nearest
neighbours, so one step at a set of sites needs the state at those sites and
their neighbours (``stencil_sites``).  Plain numpy in float64; numpy does not
contract a*b+c, so every product and sum is rounded as written, like the C
oracle built with -ffp-contract=off.  Pinned against ``orc_step`` on whole
small lattices (tests/test_oracle_pins.py), where both give identical numbers.
Used only by tests; shares nothing with the CUDA library.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def coords(dims: int, N: int, sites) -> list:
    """Coordinates (x, y, z)[:dims] of linear indices x + N y + N^2 z."""
    s = np.asarray(sites, dtype=np.int64)
    out = []
    for _ in range(dims):
        out.append(s % N)
        s = s // N
    return out


def linear(N: int, cs) -> np.ndarray:
    idx = np.zeros_like(cs[0])
    stride = 1
    for c in cs:
        idx = idx + c * stride
        stride *= N
    return idx


def neighbour(dims: int, N: int, sites, d: int, direction: int) -> np.ndarray:
    """Index of the neighbour one step along axis d in direction +1/-1 (periodic)."""
    cs = coords(dims, N, sites)
    cs[d] = (cs[d] + direction) % N
    return linear(N, cs)


def stencil_sites(dims: int, N: int, sites) -> np.ndarray:
    """Sorted unique indices of the sites and all their nearest neighbours."""
    s = np.asarray(sites, dtype=np.int64).reshape(-1)
    parts = [s]
    for d in range(dims):
        parts.append(neighbour(dims, N, s, d, +1))
        parts.append(neighbour(dims, N, s, d, -1))
    return np.unique(np.concatenate(parts))


@dataclass
class SampledStep:
    f: np.ndarray        # (nf, m) f(t+dt) at the sites
    v: np.ndarray        # (nf, m) v(t+3dt/2) at the sites
    a: float             # a(t+dt)
    ap: float            # a'(t+3dt/2)
    app: float           # a''(t+dt)


def scale_update(expansion: bool, kappa2: float, dt: float, a: float, ap: float, G: float, V: float):
    """orc_step's scale-factor update: returns (a_new, ap_new, app_new, s = app/a)."""
    if not expansion:
        return a, ap, 0.0, 0.0
    a1 = a + dt * ap
    Q = kappa2 * (2.0 * G + 3.0 * V) / a1
    c = 2.0 * ap + dt * Q
    disc = 1.0 + dt * c / a1
    if not disc >= 0.0:
        raise ValueError("no real a' root")
    u = 2.0 * c / (1.0 + math.sqrt(disc))
    app = (u - 2.0 * ap) / dt
    return a1, u - ap, app, app / a1


def step_at(p, sites, stencil, f_st, v_st, a: float, ap: float, G: float, V: float) -> SampledStep:
    """One step at ``sites`` from the state sampled at ``stencil`` (sorted,
    containing every site and its neighbours): f_st, v_st of shape (nf, M).
    p: oracle.Params (dims, N, L, dt, nf, q, expansion, kappa2)."""
    sites = np.asarray(sites, dtype=np.int64).reshape(-1)
    stencil = np.asarray(stencil, dtype=np.int64)
    f_st = np.asarray(f_st, dtype=np.float64).reshape(p.nf, -1)
    v_st = np.asarray(v_st, dtype=np.float64).reshape(p.nf, -1)

    def pos(idx):
        k = np.searchsorted(stencil, idx)
        if np.any(k >= stencil.size) or np.any(stencil[np.minimum(k, stencil.size - 1)] != idx):
            raise ValueError("a neighbour of a site is missing from the stencil")
        return k

    dt = p.dt
    f1 = f_st + dt * v_st                                 # drift
    a1, ap1, app1, s = scale_update(p.expansion, p.kappa2, dt, a, ap, G, V)
    dx = p.L / p.N
    inv_dx2 = 1.0 / (dx * dx)
    k0 = pos(sites)
    lap = np.zeros((p.nf, sites.size))
    for d in range(p.dims):
        kp = pos(neighbour(p.dims, p.N, sites, d, +1))
        km = pos(neighbour(p.dims, p.N, sites, d, -1))
        lap = lap + (f1[:, kp] + f1[:, km] - 2.0 * f1[:, k0])
    lap = lap * inv_dx2
    fs = f1[:, k0]
    q = list(p.q) + [0.0] * 3
    phi = fs[0]
    coupling = np.zeros_like(phi)
    for i in range(1, p.nf):
        coupling = coupling + q[i - 1] * fs[i] * fs[i]
    dv = np.empty_like(fs)
    dv[0] = phi * phi * phi + phi * coupling
    for i in range(1, p.nf):
        dv[i] = q[i - 1] * phi * phi * fs[i]
    F = lap - dv + s * fs
    v1 = v_st[:, k0] + dt * F                             # kick
    return SampledStep(fs, v1, a1, ap1, app1)


def drifted_sums(p, read, slab: int = 16):
    """The step's global sums (row A5 of the step; reading c-4 for G): the mean
    gradient energy G = (1/S) sum_x sum_i sum_d 1/2 ((g_i(x+e_d) - g_i(x))/dx)^2
    and the mean potential V = (1/S) sum_x V(g(x)) of the drifted fields
    g = f + dt v, over the whole lattice, without holding it in memory.

    read(k0, k1) returns (f, v): float64 arrays of shape (nf, k1 - k0, *rest)
    holding f(t) and v(t+dt/2) on the hyperplanes k0 .. k1-1 of the slowest
    axis (z in 3D, y in 2D, x in 1D), x fastest.  Slabs of `slab` hyperplanes
    are read in order, each with the next hyperplane (the first one again at
    the end: the periodic wrap) for the forward difference along the slowest
    axis; within a hyperplane the forward differences wrap with np.roll.  The
    drift f + dt v is the same single rounding as orc_step's; the sums add in
    a different order than orc_gradient_mean / orc_potential_mean (per slab,
    then across slabs), so they agree with those to rounding.
    Returns (G, V, G_per_field)."""
    n = p.N
    dx = p.L / p.N
    q = list(p.q) + [0.0] * 3
    G = np.zeros(p.nf)
    Vsum = 0.0
    first = None
    for k0 in range(0, n, slab):
        k1 = min(n, k0 + slab)
        f, v = read(k0, min(n, k1 + 1))
        g = np.asarray(f, dtype=np.float64) + p.dt * np.asarray(v, dtype=np.float64)
        if k0 == 0:
            first = g[:, :1].copy()
        if k1 == n:
            g = np.concatenate([g, first], axis=1)
        m = k1 - k0
        body = g[:, :m]
        for i in range(p.nf):
            acc = 0.0
            # slowest axis: hyperplane k+1 minus hyperplane k
            dz = (g[i, 1:m + 1] - body[i]) / dx
            acc += float(np.sum(0.5 * dz * dz))
            # the faster axes, periodic within each hyperplane
            for ax in range(1, p.dims):
                d = (np.roll(body[i], -1, axis=ax) - body[i]) / dx
                acc += float(np.sum(0.5 * d * d))
            G[i] += acc
        phi = body[0]
        pot = 0.25 * phi * phi * phi * phi
        for i in range(1, p.nf):
            pot = pot + 0.5 * q[i - 1] * phi * phi * body[i] * body[i]
        Vsum += float(np.sum(pot))
    S = float(p.N) ** p.dims
    G = G / S
    return float(np.sum(G)), Vsum / S, G
