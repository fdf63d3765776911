"""CPU oracle for the staggered-leapfrog lattice evolution (arXiv:0712.0813, Sec. III).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only users.  The oracle is plain serial
FP64 C (``clusterlat_oracle.c``), compiled with ``-O2 -ffp-contract=off``; this
module only compiles it and marshals numpy arrays through ctypes.  It shares no
code with the CUDA library and never imports it.

Parity status per function (what pins it is in ``tests/test_oracle_pins.py``):
  orc_laplacian          pinned: plane-wave eigenvalue, Kronecker-sum matrix on N=3
  orc_dvdf/orc_potential pinned: finite-difference gradient of V, closed form
  orc_step/orc_init      pinned: free-mode exact discrete solution, homogeneous
                         limit against a cosmic-time RK4 of the physical
                         Klein-Gordon + Friedmann system, energy and Friedmann
                         constraint drift O(dt^2), time reversibility
  orc_energy/orc_means_variances pinned: numpy definitions
  spectrum (numpy FFT + binning) pinned: Parseval, plane-wave and constant fields
  local.step_at (one step at chosen sites, numpy; ``oracle/local.py``) pinned:
                         bit-identical to orc_step on whole small lattices
  local.drifted_sums (G and V of f + dt v, streamed over slabs) pinned: equal
                         to orc_gradient_mean / orc_potential_mean to rounding
  omp_init/omp_step (``clusterlat_oracle_omp.c``, the same loops with OpenMP
                         threads; timing only) checked equal to orc_init /
                         orc_step to rounding
  start-up conventions (a(0)=1, u-velocity, kappa default), the IC recipe and the
  Courant rule are conventions the paper leaves open: parity unpinned there.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "clusterlat_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_OMP_SRC = os.path.join(_HERE, "clusterlat_oracle_omp.c")
_OMP_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle_omp.so")
_lib = None
_omp_lib = None


def _compile(src: str, out: str, extra: list, force: bool):
    stale = (not os.path.exists(out)
             or os.path.getmtime(out) < os.path.getmtime(src)
             or os.path.getmtime(out) < os.path.getmtime(_SRC[:-2] + ".h"))
    if force or stale:
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-Wall", *extra, "-o", tmp, src, "-lm"])
        os.replace(tmp, out)


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` and its OpenMP
    timing copy into ``oracle/_build/liboracle_omp.so`` (gcc, no GPU)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    _compile(_SRC, _LIB_PATH, [], force)
    _compile(_OMP_SRC, _OMP_LIB_PATH, ["-fopenmp"], force)
    return _LIB_PATH


class Model(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int), ("N", ctypes.c_longlong), ("L", ctypes.c_double),
                ("dt", ctypes.c_double), ("nf", ctypes.c_int), ("q", ctypes.c_double * 3),
                ("expansion", ctypes.c_int), ("kappa2", ctypes.c_double)]


class Scale(ctypes.Structure):
    _fields_ = [("a", ctypes.c_double), ("ap", ctypes.c_double), ("app", ctypes.c_double),
                ("t", ctypes.c_double), ("step", ctypes.c_longlong)]


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        d = ctypes.c_double
        pd = P(d)
        pm = P(Model)
        ps = P(Scale)
        sig = {
            "orc_sites": (ctypes.c_longlong, [pm]),
            "orc_laplacian": (None, [pm, pd, pd]),
            "orc_dvdf": (None, [pm, pd, pd]),
            "orc_potential": (d, [pm, pd]),
            "orc_force": (None, [pm, pd, d, pd]),
            "orc_gradient_mean": (d, [pm, pd, pd]),
            "orc_potential_mean": (d, [pm, pd]),
            "orc_init": (ctypes.c_int, [pm, pd, pd, ps]),
            "orc_step": (ctypes.c_int, [pm, pd, pd, ps, ctypes.c_longlong]),
            "orc_sync_velocity": (None, [pm, pd, pd, ps, pd]),
            "orc_sync_u": (None, [pm, pd, pd, ps, pd]),
            "orc_energy": (None, [pm, pd, pd, ps, pd]),
            "orc_means_variances": (None, [pm, pd, pd, pd]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass
class Params:
    """Lattice and model parameters in program units (mirrors ``orc_model``)."""
    dims: int
    N: int
    L: float
    dt: float
    nf: int = 2
    q: tuple = (1.2, 0.0, 0.0)
    expansion: bool = False
    kappa2: float = 8.0 * np.pi / 3.0 * 0.342 ** 2

    def model(self) -> Model:
        q = list(self.q) + [0.0] * (3 - len(self.q))
        return Model(self.dims, self.N, self.L, self.dt, self.nf,
                     (ctypes.c_double * 3)(*q[:3]), int(self.expansion), self.kappa2)

    @property
    def S(self) -> int:
        return self.N ** self.dims


def laplacian(p: Params, f: np.ndarray) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
    out = np.empty_like(f)
    _load().orc_laplacian(ctypes.byref(p.model()), _ptr(f), _ptr(out))
    return out


def dvdf(p: Params, fsite) -> np.ndarray:
    fs = np.ascontiguousarray(fsite, dtype=np.float64)
    out = np.empty(p.nf)
    _load().orc_dvdf(ctypes.byref(p.model()), _ptr(fs), _ptr(out))
    return out


def potential(p: Params, fsite) -> float:
    fs = np.ascontiguousarray(fsite, dtype=np.float64)
    return _load().orc_potential(ctypes.byref(p.model()), _ptr(fs))


def force(p: Params, f: np.ndarray, s: float = 0.0) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
    out = np.empty_like(f)
    _load().orc_force(ctypes.byref(p.model()), _ptr(f), s, _ptr(out))
    return out


def gradient_mean(p: Params, f: np.ndarray):
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
    per = np.zeros(4)
    tot = _load().orc_gradient_mean(ctypes.byref(p.model()), _ptr(f), _ptr(per))
    return tot, per[:p.nf].copy()


def potential_mean(p: Params, f: np.ndarray) -> float:
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
    return _load().orc_potential_mean(ctypes.byref(p.model()), _ptr(f))


@dataclass
class State:
    """f(t), v(t+dt/2) and the scale factor, as the oracle evolves them."""
    p: Params
    f: np.ndarray
    v: np.ndarray
    scale: Scale = field(default_factory=Scale)

    def copy(self) -> "State":
        sc = Scale(self.scale.a, self.scale.ap, self.scale.app, self.scale.t, self.scale.step)
        return State(self.p, self.f.copy(), self.v.copy(), sc)


def init(p: Params, f0: np.ndarray, u0: np.ndarray) -> State:
    """Start-up from f(0) and synchronised u(0) (see ``orc_init``)."""
    f = np.array(f0, dtype=np.float64).reshape(-1).copy()
    v = np.array(u0, dtype=np.float64).reshape(-1).copy()
    assert f.size == p.nf * p.S and v.size == f.size
    sc = Scale()
    rc = _load().orc_init(ctypes.byref(p.model()), _ptr(f), _ptr(v), ctypes.byref(sc))
    if rc != 0:
        raise RuntimeError(f"orc_init failed ({rc})")
    return State(p, f, v, sc)


def step(st: State, n: int) -> State:
    rc = _load().orc_step(ctypes.byref(st.p.model()), _ptr(st.f), _ptr(st.v),
                          ctypes.byref(st.scale), int(n))
    if rc != 0:
        raise RuntimeError(f"orc_step failed ({rc})")
    return st


def _load_omp():
    """The OpenMP copy of the oracle's loops (``clusterlat_oracle_omp.c``), used
    only to time the CPU baseline on all host cores."""
    global _omp_lib
    if _omp_lib is None:
        build()
        lib = ctypes.CDLL(_OMP_LIB_PATH)
        P = ctypes.POINTER
        pd = P(ctypes.c_double)
        lib.orcp_threads.restype = ctypes.c_int
        lib.orcp_threads.argtypes = []
        lib.orcp_set_threads.restype = None
        lib.orcp_set_threads.argtypes = [ctypes.c_int]
        lib.orcp_init.restype = ctypes.c_int
        lib.orcp_init.argtypes = [P(Model), pd, pd, P(Scale)]
        lib.orcp_step.restype = ctypes.c_int
        lib.orcp_step.argtypes = [P(Model), pd, pd, P(Scale), ctypes.c_longlong]
        _omp_lib = lib
    return _omp_lib


def omp_threads(n: int | None = None) -> int:
    """Set (n > 0) and return the number of OpenMP threads of the timing copy."""
    lib = _load_omp()
    if n:
        lib.orcp_set_threads(int(n))
    return lib.orcp_threads()


def omp_init(p: Params, f0: np.ndarray, u0: np.ndarray) -> State:
    """``init`` through the OpenMP timing copy (same result to rounding)."""
    f = np.array(f0, dtype=np.float64).reshape(-1).copy()
    v = np.array(u0, dtype=np.float64).reshape(-1).copy()
    assert f.size == p.nf * p.S and v.size == f.size
    sc = Scale()
    rc = _load_omp().orcp_init(ctypes.byref(p.model()), _ptr(f), _ptr(v), ctypes.byref(sc))
    if rc != 0:
        raise RuntimeError(f"orcp_init failed ({rc})")
    return State(p, f, v, sc)


def omp_step(st: State, n: int) -> State:
    """``step`` through the OpenMP timing copy (same result to rounding)."""
    rc = _load_omp().orcp_step(ctypes.byref(st.p.model()), _ptr(st.f), _ptr(st.v),
                               ctypes.byref(st.scale), int(n))
    if rc != 0:
        raise RuntimeError(f"orcp_step failed ({rc})")
    return st


def sync_velocity(st: State) -> np.ndarray:
    out = np.empty_like(st.v)
    _load().orc_sync_velocity(ctypes.byref(st.p.model()), _ptr(st.f), _ptr(st.v),
                              ctypes.byref(st.scale), _ptr(out))
    return out


def sync_u(st: State) -> np.ndarray:
    out = np.empty_like(st.v)
    _load().orc_sync_u(ctypes.byref(st.p.model()), _ptr(st.f), _ptr(st.v),
                       ctypes.byref(st.scale), _ptr(out))
    return out


ENERGY_KEYS = ("K", "G", "V", "E", "a", "ap", "t", "friedmann_resid")


def energy(st: State) -> dict:
    out = np.zeros(16)
    _load().orc_energy(ctypes.byref(st.p.model()), _ptr(st.f), _ptr(st.v),
                       ctypes.byref(st.scale), _ptr(out))
    nf = st.p.nf
    return {"K": out[0:nf].copy(), "G": out[4:4 + nf].copy(), "V": out[8], "E": out[9],
            "a": out[10], "ap": out[11], "t": out[12], "friedmann_resid": out[13]}


def means_variances(p: Params, f: np.ndarray):
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
    mean = np.zeros(p.nf)
    var = np.zeros(p.nf)
    _load().orc_means_variances(ctypes.byref(p.model()), _ptr(f), _ptr(mean), _ptr(var))
    return mean, var


def spectrum(p: Params, f_field: np.ndarray, nbins: int):
    """Binned power spectrum of one field (the library's output definition):
    fhat(n) = sum_x f(x) exp(-2 pi i n.x / N) (unnormalised DFT, numpy's FFT as
    the transform), bin b = floor(|n| + 1/2) over the integer modes n with
    components in (-N/2, N/2]; power[b] = mean |fhat|^2 over the bin,
    count[b] = number of modes, k[b] = 2 pi b / L.  Parity pinned by Parseval and
    plane waves (tests); the binning convention itself is not from the paper."""
    shape = (p.N,) * p.dims
    F = np.fft.fftn(np.asarray(f_field, dtype=np.float64).reshape(shape))
    freqs = np.meshgrid(*([np.fft.fftfreq(p.N, 1.0 / p.N)] * p.dims), indexing="ij")
    nabs = np.sqrt(sum(g * g for g in freqs))
    bins = np.floor(nabs + 0.5).astype(np.int64).reshape(-1)
    pw = (np.abs(F) ** 2).reshape(-1)
    power = np.zeros(nbins)
    count = np.zeros(nbins)
    for b, w in zip(bins, pw):
        if b < nbins:
            power[b] += w
            count[b] += 1
    mean = np.where(count > 0, power / np.maximum(count, 1), 0.0)
    return 2 * np.pi * np.arange(nbins) / p.L, mean, count
