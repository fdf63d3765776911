"""Python binding of libclusterlat's C ABI (include/clusterlat.h), same names.

Argument marshalling only: every step of the evolution runs in the library's
CUDA kernels.  Loading fails loudly if the library is missing or was built for
another machine; there is no CPU fallback.  PyTorch is optional plumbing: a
CUDA stream handle (``torch.cuda.Stream().cuda_stream``) may be passed as
``stream``, and ``torch_allocator=True`` routes the handle's device
allocations through PyTorch's caching allocator.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

CE_OK, CE_EINVAL, CE_ENOMEM, CE_ECUDA, CE_ETIMEOUT, CE_ENONFINITE, CE_ESTATE = 0, -1, -2, -3, -4, -5, -6
CE_F64, CE_F32 = 0, 1
CE_VEL_SYNC, CE_VEL_STAGGERED = 0, 1
CE_KERNEL_AUTO, CE_KERNEL_GENERIC, CE_KERNEL_SWEEP, CE_KERNEL_ROWS, CE_KERNEL_PLANES = 0, 1, 2, 3, 4
CE_FLAG_ALLOW_UNSTABLE_DT = 1
CE_FLAG_TEST_TMA_STALL = 2

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
RELEASE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class ce_config(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int), ("N", ctypes.c_int64), ("L", ctypes.c_double),
                ("dt", ctypes.c_double), ("nfields", ctypes.c_int), ("q", ctypes.c_double * 3),
                ("expansion", ctypes.c_int), ("phi0_over_mpl", ctypes.c_double),
                ("phi0", ctypes.c_double), ("precision", ctypes.c_int), ("kernel", ctypes.c_int),
                ("flags", ctypes.c_int), ("tile_rows", ctypes.c_int), ("stages", ctypes.c_int),
                ("zchunks", ctypes.c_int), ("stream", ctypes.c_void_p), ("alloc", ALLOC_FN),
                ("release", RELEASE_FN), ("alloc_ctx", ctypes.c_void_p)]


class ce_scalars_t(ctypes.Structure):
    _fields_ = [("a", ctypes.c_double), ("ap_half", ctypes.c_double), ("app", ctypes.c_double),
                ("t", ctypes.c_double), ("step", ctypes.c_int64)]


class ce_energy_t(ctypes.Structure):
    _fields_ = [("K", ctypes.c_double * 4), ("G", ctypes.c_double * 4), ("V", ctypes.c_double),
                ("E", ctypes.c_double), ("a", ctypes.c_double), ("ap", ctypes.c_double),
                ("t", ctypes.c_double), ("friedmann_resid", ctypes.c_double), ("step", ctypes.c_int64)]


class CeError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


_lib = None
_keepalive: dict = {}   # handle -> (config, ctypes callbacks, allocation table)

# Every symbol the public header declares (checked by the test-suite).
EXPORTS = ("ce_create", "ce_set_fields", "ce_step", "ce_synchronize", "ce_means_variances",
           "ce_energy", "ce_get_fields", "ce_free", "ce_last_error", "ce_device_bytes",
           "ce_kernel_in_use", "ce_sweep_plan", "ce_replan", "ce_version", "ce_moments_noalloc",
           "ce_spectrum", "ce_save", "ce_load",
           "ce_sample_fields", "ce_batch_create", "ce_batch_step", "ce_batch_synchronize", "ce_batch_status", "ce_batch_info",
           "ce_batch_free")


def lib_path() -> str:
    return _build.LIB


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libclusterlat (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = _build.build()
    if not os.path.exists(path):
        raise CeError(CE_ECUDA, f"libclusterlat not found at {path}")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    pd = P(ctypes.c_double)
    vp = ctypes.c_void_p
    sigs = {
        "ce_create": (ctypes.c_int, [P(ce_config), P(vp)]),
        "ce_set_fields": (ctypes.c_int, [vp, pd, pd, ctypes.c_int, P(ce_scalars_t)]),
        "ce_step": (ctypes.c_int, [vp, ctypes.c_int64]),
        "ce_synchronize": (ctypes.c_int, [vp]),
        "ce_means_variances": (ctypes.c_int, [vp, pd, pd]),
        "ce_energy": (ctypes.c_int, [vp, P(ce_energy_t)]),
        "ce_get_fields": (ctypes.c_int, [vp, pd, pd, ctypes.c_int, P(ce_scalars_t)]),
        "ce_free": (None, [vp]),
        "ce_last_error": (ctypes.c_char_p, []),
        "ce_device_bytes": (ctypes.c_int64, [vp]),
        "ce_kernel_in_use": (ctypes.c_int, [vp]),
        "ce_sweep_plan": (ctypes.c_int, [vp, P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_int)]),
        "ce_replan": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
        "ce_spectrum": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, pd, pd, pd]),
        "ce_save": (ctypes.c_int, [vp, ctypes.c_char_p]),
        "ce_load": (ctypes.c_int, [vp, ctypes.c_char_p]),
        "ce_version": (ctypes.c_int, []),
        "ce_moments_noalloc": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int64, ctypes.c_int, vp, vp, vp]),
        "ce_batch_create": (ctypes.c_int, [P(vp), ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, P(vp)]),
        "ce_batch_step": (ctypes.c_int, [vp, ctypes.c_int64]),
        "ce_sample_fields": (ctypes.c_int, [vp, P(ctypes.c_int64), ctypes.c_int64, P(ctypes.c_double),
                                            P(ctypes.c_double), P(ce_scalars_t)]),
        "ce_batch_synchronize": (ctypes.c_int, [vp]),
        "ce_batch_status": (ctypes.c_int, [vp, P(ctypes.c_int), ctypes.c_int]),
        "ce_batch_info": (ctypes.c_int, [vp, P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_int),
                                         P(ctypes.c_int64)]),
        "ce_batch_free": (None, [vp]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def ce_last_error() -> str:
    return load().ce_last_error().decode()


def _check(rc: int):
    if rc != CE_OK:
        raise CeError(rc, ce_last_error())


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _as_f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))


def _torch_hooks(table: dict):
    import torch

    def _alloc(nbytes, stream, ctx):
        ptr = torch.cuda.caching_allocator_alloc(int(nbytes), stream=torch.cuda.current_stream())
        table[ptr] = nbytes
        return ptr

    def _release(ptr, nbytes, stream, ctx):
        table.pop(ptr, None)
        torch.cuda.caching_allocator_delete(ptr)

    return ALLOC_FN(_alloc), RELEASE_FN(_release)


def ce_create(dims: int, N: int, L: float, dt: float, nfields: int = 2, q=(1.2,),
              expansion: bool = False, phi0_over_mpl: float = 0.342, phi0: float = 1.0,
              precision: str | int = "f64", kernel: str | int = "auto",
              allow_unstable_dt: bool = False, stream=None, torch_allocator: bool = False,
              tile_rows: int = 0, stages: int = 0, zchunks: int = 0, flags: int = 0):
    """Create a simulation handle (see ce_create in clusterlat.h)."""
    lib = load()
    cfg = ce_config()
    cfg.dims, cfg.N, cfg.L, cfg.dt, cfg.nfields = int(dims), int(N), float(L), float(dt), int(nfields)
    qq = list(q) + [0.0] * 3
    cfg.q = (ctypes.c_double * 3)(*[float(x) for x in qq[:3]])
    cfg.expansion = int(bool(expansion))
    cfg.phi0_over_mpl = float(phi0_over_mpl)
    cfg.phi0 = float(phi0)
    cfg.precision = {"f64": CE_F64, "f32": CE_F32}.get(precision, precision)
    cfg.kernel = {"auto": CE_KERNEL_AUTO, "generic": CE_KERNEL_GENERIC, "sweep": CE_KERNEL_SWEEP,
                  "rows": CE_KERNEL_ROWS, "planes": CE_KERNEL_PLANES}.get(kernel, kernel)
    cfg.flags = (CE_FLAG_ALLOW_UNSTABLE_DT if allow_unstable_dt else 0) | int(flags)
    cfg.tile_rows, cfg.stages, cfg.zchunks = int(tile_rows), int(stages), int(zchunks)
    if stream is not None:
        cfg.stream = ctypes.c_void_p(int(stream))
    keep = [cfg]
    if torch_allocator:
        table: dict = {}
        a, r = _torch_hooks(table)
        cfg.alloc, cfg.release = a, r
        keep += [a, r, table]
    h = ctypes.c_void_p()
    _check(lib.ce_create(ctypes.byref(cfg), ctypes.byref(h)))
    _keepalive[h.value] = keep
    return h


def ce_set_fields(sim, f, v, mode: int = CE_VEL_SYNC, scalars: ce_scalars_t | None = None):
    f = _as_f64(f)
    v = _as_f64(v)
    _check(load().ce_set_fields(sim, _dptr(f), _dptr(v), int(mode),
                                ctypes.byref(scalars) if scalars is not None else None))


def ce_step(sim, n: int):
    _check(load().ce_step(sim, int(n)))


def ce_synchronize(sim):
    _check(load().ce_synchronize(sim))


def ce_means_variances(sim, nfields: int | None = None):
    mean = np.zeros(4)
    var = np.zeros(4)
    _check(load().ce_means_variances(sim, _dptr(mean), _dptr(var)))
    n = 4 if nfields is None else nfields
    return mean[:n], var[:n]


def ce_energy(sim) -> dict:
    e = ce_energy_t()
    _check(load().ce_energy(sim, ctypes.byref(e)))
    return {"K": np.array(e.K[:]), "G": np.array(e.G[:]), "V": e.V, "E": e.E, "a": e.a, "ap": e.ap,
            "t": e.t, "friedmann_resid": e.friedmann_resid, "step": e.step}


def ce_get_fields(sim, nfields: int, sites: int, mode: int = CE_VEL_SYNC, out=None):
    """Return (f, v, scalars); f and v are float64 arrays of nfields * sites."""
    if out is None:
        f = np.empty(nfields * sites)
        v = np.empty(nfields * sites)
    else:
        f, v = out
    sc = ce_scalars_t()
    _check(load().ce_get_fields(sim, _dptr(f), _dptr(v), int(mode), ctypes.byref(sc)))
    return f, v, sc


def ce_sample_fields(sim, nfields: int, sites):
    """Staggered state at the given linear site indices: (f, v, scalars), f and v
    float64 arrays of shape (nfields, len(sites))."""
    idx = np.ascontiguousarray(sites, dtype=np.int64).reshape(-1)
    n = idx.size
    f = np.empty((nfields, n))
    v = np.empty((nfields, n))
    sc = ce_scalars_t()
    _check(load().ce_sample_fields(sim, idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), n,
                                   _dptr(f), _dptr(v), ctypes.byref(sc)))
    return f, v, sc


def ce_free(sim):
    if sim is None or not getattr(sim, "value", None):
        return
    load().ce_free(sim)
    _keepalive.pop(sim.value, None)


def ce_device_bytes(sim) -> int:
    return load().ce_device_bytes(sim)


def ce_kernel_in_use(sim) -> int:
    return load().ce_kernel_in_use(sim)


def ce_sweep_plan(sim):
    """(rows, stages, zchunks) of the z-sweep plan; zeros when the generic kernel runs."""
    r, st, z = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().ce_sweep_plan(sim, ctypes.byref(r), ctypes.byref(st), ctypes.byref(z)))
    return r.value, st.value, z.value


def ce_spectrum(sim, field: int, nbins: int):
    """(k, power, count) arrays of the binned power spectrum of one field."""
    k, p, n = np.zeros(nbins), np.zeros(nbins), np.zeros(nbins)
    _check(load().ce_spectrum(sim, int(field), int(nbins), _dptr(k), _dptr(p), _dptr(n)))
    return k, p, n


def ce_save(sim, path: str):
    _check(load().ce_save(sim, os.fsencode(path)))


def ce_load(sim, path: str):
    _check(load().ce_load(sim, os.fsencode(path)))


def ce_replan(sim, rows: int = 0, stages: int = 0, zchunks: int = 0):
    _check(load().ce_replan(sim, int(rows), int(stages), int(zchunks)))


def ce_version() -> int:
    return load().ce_version()


def ce_moments_noalloc(f_ptr: int, precision: int, n: int, nfields: int, stream: int | None,
                       mean_ptr: int, var_ptr: int):
    """Allocation-free moments of caller-owned device arrays (see clusterlat.h).

    All pointers are device addresses (e.g. ``tensor.data_ptr()``); the call is
    asynchronous on ``stream`` and allocates nothing on the device."""
    _check(load().ce_moments_noalloc(ctypes.c_void_p(int(f_ptr)), int(precision), int(n), int(nfields),
                                     ctypes.c_void_p(int(stream) if stream else 0),
                                     ctypes.c_void_p(int(mean_ptr)), ctypes.c_void_p(int(var_ptr))))


def ce_batch_create(sims, sweep_len: int = 0, stream=None, ctas_per_sm: int = 0):
    """Group handles (ctypes handles or Simulation objects) into a batch."""
    hs = [x.handle if isinstance(x, Simulation) else x for x in sims]
    arr = (ctypes.c_void_p * len(hs))(*[h.value for h in hs])
    b = ctypes.c_void_p()
    _check(load().ce_batch_create(arr, len(hs), int(sweep_len), int(ctas_per_sm),
                                  ctypes.c_void_p(int(stream) if stream else 0), ctypes.byref(b)))
    return b


def ce_batch_step(b, n: int):
    _check(load().ce_batch_step(b, int(n)))


def ce_batch_synchronize(b):
    _check(load().ce_batch_synchronize(b))


def ce_batch_status(b, n: int) -> list:
    """Per-member latched status codes (CE_OK = 0) after waiting for the batch."""
    st = (ctypes.c_int * max(n, 1))()
    _check(load().ce_batch_status(b, st, int(n)))
    return [int(st[k]) for k in range(n)]


def ce_batch_info(b) -> dict:
    m, it, bl, st = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
    _check(load().ce_batch_info(b, ctypes.byref(m), ctypes.byref(it), ctypes.byref(bl), ctypes.byref(st)))
    return {"members": m.value, "items": it.value, "blocks": bl.value, "sites": st.value}


def ce_batch_free(b):
    if b is not None and getattr(b, "value", None):
        load().ce_batch_free(b)


class Batch:
    """Owning wrapper around a batch: ``with Batch(sims) as b: b.step(n)``."""

    def __init__(self, sims, sweep_len: int = 0, stream=None, ctas_per_sm: int = 0):
        self.sims = list(sims)
        self.handle = ce_batch_create(self.sims, sweep_len, stream, ctas_per_sm)

    def step(self, n):
        ce_batch_step(self.handle, n)

    def synchronize(self):
        ce_batch_synchronize(self.handle)

    def member_status(self) -> list:
        return ce_batch_status(self.handle, len(self.sims))

    @property
    def info(self):
        return ce_batch_info(self.handle)

    def close(self):
        if self.handle is not None:
            ce_batch_free(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Simulation:
    """Owning wrapper around one handle: ``with Simulation(...) as sim: ...``."""

    def __init__(self, **cfg):
        self.nfields = int(cfg.get("nfields", 2))
        self.sites = int(cfg["N"]) ** int(cfg["dims"])
        self.handle = ce_create(**cfg)

    def set_fields(self, f, v, mode=CE_VEL_SYNC, scalars=None):
        ce_set_fields(self.handle, f, v, mode, scalars)

    def step(self, n):
        ce_step(self.handle, n)

    def synchronize(self):
        ce_synchronize(self.handle)

    def means_variances(self):
        return ce_means_variances(self.handle, self.nfields)

    def energy(self):
        e = ce_energy(self.handle)
        e["K"] = e["K"][:self.nfields]
        e["G"] = e["G"][:self.nfields]
        return e

    def get_fields(self, mode=CE_VEL_SYNC):
        return ce_get_fields(self.handle, self.nfields, self.sites, mode)

    def sample_fields(self, sites):
        return ce_sample_fields(self.handle, self.nfields, sites)

    @property
    def kernel(self):
        return ce_kernel_in_use(self.handle)

    @property
    def sweep_plan(self):
        return ce_sweep_plan(self.handle)

    def replan(self, rows: int = 0, stages: int = 0, zchunks: int = 0):
        ce_replan(self.handle, rows, stages, zchunks)

    def spectrum(self, field: int, nbins: int):
        return ce_spectrum(self.handle, field, nbins)

    def save(self, path: str):
        ce_save(self.handle, path)

    def load(self, path: str):
        ce_load(self.handle, path)

    def close(self):
        if self.handle is not None:
            ce_free(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
