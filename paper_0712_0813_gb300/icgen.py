"""Seeded synthetic initial conditions for lattice runs.

This module is the one input generator shared by the CUDA library's callers and
by the CPU oracle's tests.  It draws random numbers and builds arrays; it holds
none of the evolution's arithmetic (no Laplacian, force, leapfrog or scale-factor
update), so the two implementations it feeds stay independent.

Recipe (a convention: arXiv:0712.0813 leaves initial conditions to the
LATTICEEASY documentation; "parity unpinned" for the recipe itself):
  for each field i, with integer modes n in Z_N^d and k = 2 pi |n| / L,
    omega_k = sqrt(k^2 + m_i^2),  m_phi^2 = 3 phi0^2,  m_chi_i^2 = q_i phi0^2,
    c_n = sqrt(1 / (2 omega_k)) exp(i theta_n),  theta_n uniform in [0, 2 pi),
    c_0 = 0 and c_n = 0 for |n| > N/4 (the cut-off),
    delta f = amp sqrt(S) irfft(c),  delta u = amp sqrt(S) irfft(omega_k c),
  phi = phi0 + delta phi, chi_i = delta chi_i; the velocities are the
  synchronised u = f' - (a'/a) f.  Real output comes from numpy's inverse real
  FFT, which keeps the Hermitian half of the spectrum.
"""
from __future__ import annotations

import math

import numpy as np


def mode_grid(dims: int, N: int) -> np.ndarray:
    """|n|^2 on the half-spectrum grid of numpy's real FFT (last axis = x)."""
    full = np.fft.fftfreq(N, d=1.0 / N)
    half = np.fft.rfftfreq(N, d=1.0 / N)
    axes = [full] * (dims - 1) + [half]
    grids = np.meshgrid(*axes, indexing="ij")
    n2 = np.zeros(grids[0].shape)
    for g in grids:
        n2 += g * g
    return n2


def lattice_ics(dims: int, N: int, L: float, nf: int, phi0: float = 1.0,
                q=(1.2,), amp: float = 1e-4, seed: int = 1,
                kcut_frac: float = 0.25, backend: str = "numpy", pinned: bool = False):
    """Return (f, u) as float64 arrays of shape (nf, N**dims), layout [field][z][y][x].

    backend "numpy" transforms on the host; "torch" draws the same phases and
    runs the inverse FFT with torch (on the GPU when one is present), which is
    what large lattices (512^3 and up) need.  pinned (torch backend with a GPU):
    the arrays live in page-locked host memory, so host<->device copies from and
    into them need no staging."""
    if backend == "torch":
        return _lattice_ics_torch(dims, N, L, nf, phi0, q, amp, seed, kcut_frac, pinned)
    shape = (N,) * dims
    S = N ** dims
    n2 = mode_grid(dims, N)
    k = 2.0 * math.pi * np.sqrt(n2) / L
    keep = (n2 > 0) & (np.sqrt(n2) <= kcut_frac * N)
    f = np.empty((nf, S))
    u = np.empty((nf, S))
    qs = list(q) + [0.0] * 4
    for i in range(nf):
        m2 = 3.0 * phi0 * phi0 if i == 0 else qs[i - 1] * phi0 * phi0
        omega = np.sqrt(k * k + m2)
        rng = np.random.default_rng([seed, i])
        theta = rng.uniform(0.0, 2.0 * math.pi, size=n2.shape)
        c = np.zeros(n2.shape, dtype=np.complex128)
        c[keep] = np.sqrt(1.0 / (2.0 * omega[keep])) * np.exp(1j * theta[keep])
        scale = amp * math.sqrt(S)
        df = np.fft.irfftn(c, s=shape, axes=tuple(range(dims))) * scale
        du = np.fft.irfftn(omega * c, s=shape, axes=tuple(range(dims))) * scale
        f[i] = (phi0 if i == 0 else 0.0) + df.reshape(-1)
        u[i] = du.reshape(-1)
    return f, u


def _lattice_ics_torch(dims, N, L, nf, phi0, q, amp, seed, kcut_frac, pinned=False):
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    shape = (N,) * dims
    S = N ** dims
    n2 = torch.as_tensor(mode_grid(dims, N), device=dev)
    k = 2.0 * math.pi * torch.sqrt(n2) / L
    keep = (n2 > 0) & (torch.sqrt(n2) <= kcut_frac * N)
    if pinned and dev == "cuda":
        f = torch.empty((nf, S), dtype=torch.float64, pin_memory=True).numpy()
        u = torch.empty((nf, S), dtype=torch.float64, pin_memory=True).numpy()
    else:
        f = np.empty((nf, S))
        u = np.empty((nf, S))
    qs = list(q) + [0.0] * 4
    scale = amp * math.sqrt(S)
    for i in range(nf):
        m2 = 3.0 * phi0 * phi0 if i == 0 else qs[i - 1] * phi0 * phi0
        omega = torch.sqrt(k * k + m2)
        rng = np.random.default_rng([seed, i])
        theta = torch.as_tensor(rng.uniform(0.0, 2.0 * math.pi, size=tuple(n2.shape)), device=dev)
        amp_k = torch.where(keep, torch.sqrt(1.0 / (2.0 * omega)), torch.zeros_like(omega))
        c = torch.polar(amp_k, theta)
        axes = tuple(range(dims))
        df = torch.fft.irfftn(c, s=shape, dim=axes) * scale
        du = torch.fft.irfftn(omega * c, s=shape, dim=axes) * scale
        f[i] = (phi0 if i == 0 else 0.0) + df.reshape(-1).cpu().numpy()
        u[i] = du.reshape(-1).cpu().numpy()
        del c, df, du, theta, amp_k, omega
    return f, u


def courant_dt(dims: int, N: int, L: float, phi0: float, q, cap: float = 0.05, amp: float = 1.0) -> float:
    """Time step for configurations that ask for "the Courant limit".

    Convention: omega_max^2 = 4 d / dx^2 + max(3 phi_m^2, max_i q_i phi_m^2) and
    dt = min(cap, 0.9 / omega_max), i.e. 45% of the leapfrog bound 2/omega_max,
    with the masses taken at phi_m = amp * phi0.  amp = 1 is the start-up value.
    Strongly coupled lattices (q phi0^2 comparable to 4 d / dx^2) need amp > 1:
    once the resonance has grown, phi fluctuates locally to several phi0, chi's
    local mass q phi^2 grows with it, and a step taken at amp = 1 turns the
    leapfrog unstable at the largest fluctuation.
    """
    dx = L / N
    pm = amp * phi0
    m2 = max([3.0 * pm * pm] + [qq * pm * pm for qq in q])
    w = math.sqrt(4.0 * dims / (dx * dx) + m2)
    return min(cap, 0.9 / w)
