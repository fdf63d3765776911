"""Host-side checks of the C ABI that need no GPU: the library builds and loads,
exports every symbol include/clusterlat.h declares, and rejects bad
arguments before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    syms = set()
    for name in os.listdir(os.path.join(ROOT, "include")):
        if name.endswith(".h"):
            text = open(os.path.join(ROOT, "include", name)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            text = re.sub(r"//[^\n]*", "", text)
            for m in re.finditer(r"\b(ce_[A-Za-z0-9_]+)\s*\(", text):
                syms.add(m.group(1))
    return syms


def test_header_declares_the_boundary():
    syms = _declared_symbols()
    for required in ("ce_create", "ce_set_fields", "ce_step", "ce_means_variances", "ce_energy",
                     "ce_get_fields", "ce_free", "ce_last_error"):
        assert required in syms


def test_library_exports_every_declared_symbol(capi):
    lib = ctypes.CDLL(capi.lib_path())
    missing = [s for s in sorted(_declared_symbols()) if not hasattr(lib, s)]
    assert not missing, missing
    assert set(capi.EXPORTS) == _declared_symbols()


def test_version_and_null_safety(capi):
    lib = capi.load()
    assert lib.ce_version() >= 10000
    lib.ce_free(None)  # NULL-safe
    assert lib.ce_step(None, 1) == capi.CE_EINVAL
    assert "NULL" in capi.ce_last_error()
    assert lib.ce_synchronize(None) == capi.CE_EINVAL
    assert lib.ce_device_bytes(None) == 0


BAD = [
    (dict(dims=4), "dims"),
    (dict(dims=0), "dims"),
    (dict(N=2), "N must be"),
    (dict(L=0.0), "L must"),
    (dict(L=float("nan")), "L must"),
    (dict(dt=-0.1), "dt must"),
    (dict(dt=1.0), "stability"),
    (dict(nfields=5), "nfields"),
    (dict(nfields=0), "nfields"),
    (dict(q=(-1.0,)), "q_i"),
    (dict(precision=7), "precision"),
    (dict(kernel=9), "kernel"),
    (dict(dims=3, N=1 << 12), "2^34"),
    (dict(dims=2, N=100, kernel="sweep"), "z-sweep"),
    (dict(N=18, precision="f32", kernel="rows"), "row kernel"),
    (dict(dims=1, N=64, dt=0.004, kernel="planes"), "line-sweep"),
    (dict(tile_rows=12), "tile_rows"),
    (dict(tile_rows=2), "tile_rows"),
    (dict(stages=9), "stages"),
    (dict(zchunks=-1), "zchunks"),
    (dict(N=16, zchunks=9), "zchunks"),
]


@pytest.mark.parametrize("kw,msg", BAD, ids=[m for _, m in BAD])
def test_create_rejects_bad_config(capi, kw, msg):
    cfg = dict(dims=3, N=16, L=20.0, dt=0.05, nfields=2, q=(1.2,))
    cfg.update(kw)
    with pytest.raises(capi.CeError) as ei:
        capi.ce_create(**cfg)
    assert ei.value.code == capi.CE_EINVAL
    assert msg in str(ei.value)


def test_unstable_dt_allowed_with_flag_reaches_device_check(capi):
    import torch
    if torch.cuda.is_available():
        pytest.skip("host-only check")
    with pytest.raises(capi.CeError) as ei:
        capi.ce_create(dims=3, N=16, L=20.0, dt=1.0, allow_unstable_dt=True)
    assert ei.value.code == capi.CE_ECUDA  # got past validation; no device here


def test_create_without_device_fails_cleanly(capi):
    import torch
    if torch.cuda.is_available():
        pytest.skip("host-only check")
    with pytest.raises(capi.CeError) as ei:
        capi.ce_create(dims=3, N=16, L=20.0, dt=0.05)
    assert ei.value.code == capi.CE_ECUDA
    assert "no CUDA device" in str(ei.value)


def test_struct_layouts_match_header(capi):
    # ce_config: 5 ints + int64 + 3+1+1+1 doubles ... checked by size/offsets of key fields
    assert ctypes.sizeof(capi.ce_scalars_t) == 40
    assert ctypes.sizeof(capi.ce_energy_t) == 8 * 15
    assert capi.ce_config.stream.offset % 8 == 0


def test_batch_rejects_bad_arguments_without_device(capi):
    lib = capi.load()
    import ctypes
    out = ctypes.c_void_p()
    assert lib.ce_batch_create(None, 0, 0, 0, None, ctypes.byref(out)) == capi.CE_EINVAL
    assert lib.ce_batch_step(None, 1) == capi.CE_EINVAL
    lib.ce_batch_free(None)


def test_replan_and_plan_reject_null(capi):
    lib = capi.load()
    assert lib.ce_replan(None, 0, 0, 0) == capi.CE_EINVAL
    import ctypes
    r = ctypes.c_int()
    assert lib.ce_sweep_plan(None, ctypes.byref(r), ctypes.byref(r), ctypes.byref(r)) == capi.CE_EINVAL
