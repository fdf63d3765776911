"""Outputs: the binned power spectrum against the oracle's definition, and the
grid-image file round trip (save, load into a fresh handle, continue)."""
import os

import numpy as np
import pytest

from paper_0712_0813_gb300.icgen import lattice_ics

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims,N,precision,tol", [
    (3, 32, "f64", 1e-10), (2, 64, "f64", 1e-10), (1, 256, "f64", 1e-10),
    (3, 128, "f32", 2e-5), (2, 96, "f32", 2e-5)])
def test_spectrum_matches_oracle(gpu_capi, orc, dims, N, precision, tol):
    capi = gpu_capi
    f0, u0 = lattice_ics(dims, N, 20.0, 2, q=(1.2,), seed=17, amp=1e-2)
    nb = int(np.ceil(np.sqrt(dims) * N / 2)) + 2
    with capi.Simulation(dims=dims, N=N, L=20.0, dt=0.01, nfields=2, q=(1.2,), expansion=True,
                         precision=precision) as sim:
        sim.set_fields(f0, u0)
        sim.step(7)
        f, _, _ = sim.get_fields(capi.CE_VEL_STAGGERED)
        for field in (0, 1):
            k, power, count = sim.spectrum(field, nb)
            p = orc.Params(dims=dims, N=N, L=20.0, dt=0.01, nf=2)
            kr, pr, cr = orc.spectrum(p, f.reshape(2, -1)[field], nb)
            np.testing.assert_array_equal(count, cr)
            np.testing.assert_allclose(k, kr, rtol=1e-15)
            # relative to the largest bin (the fluctuation bins are small beside bin 0 of phi)
            scale = np.abs(pr[1:]).max() if field == 0 else np.abs(pr).max()
            np.testing.assert_allclose(power, pr, rtol=tol, atol=tol * scale)


def test_grid_image_round_trip_continues_bit_identically(gpu_capi, tmp_path):
    capi = gpu_capi
    cfg = dict(dims=3, N=24, L=20.0, dt=0.05, nfields=2, q=(1.2,), expansion=True, precision="f32")
    f0, u0 = lattice_ics(3, 24, 20.0, 2, q=(1.2,), seed=9)
    path = os.path.join(str(tmp_path), "state.cegrid")
    with capi.Simulation(**cfg) as a:
        a.set_fields(f0, u0)
        a.step(19)
        a.save(path)
        a.step(17)
        fa, va, sa = a.get_fields(capi.CE_VEL_STAGGERED)
    with capi.Simulation(**cfg) as b:
        b.load(path)
        b.step(17)
        fb, vb, sb = b.get_fields(capi.CE_VEL_STAGGERED)
    assert np.array_equal(fa, fb) and np.array_equal(va, vb)
    assert (sa.a, sa.ap_half, sa.t, sa.step) == (sb.a, sb.ap_half, sb.t, sb.step) and sb.step == 36
    other = dict(cfg, N=32)
    with capi.Simulation(**other) as c:
        with pytest.raises(capi.CeError) as ei:
            c.load(path)
        assert ei.value.code == capi.CE_EINVAL


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_sample_fields_equals_full_download(gpu_capi, precision):
    """ce_sample_fields returns exactly the values ce_get_fields(CE_VEL_STAGGERED)
    returns at the same sites, in chunks when the sites outnumber the staging
    buffer; bad indices and a handle without fields are errors."""
    capi = gpu_capi
    N, nf = 24, 3
    f0, u0 = lattice_ics(3, N, 20.0, nf, q=(0.8, 5.0), seed=4, amp=1e-2)
    with capi.Simulation(dims=3, N=N, L=20.0, dt=0.02, nfields=nf, q=(0.8, 5.0), expansion=True,
                         precision=precision) as sim:
        with pytest.raises(capi.CeError) as ei:
            sim.sample_fields([0])
        assert ei.value.code == capi.CE_ESTATE
        sim.set_fields(f0, u0)
        sim.step(7)
        f, v, sc = sim.get_fields(capi.CE_VEL_STAGGERED)
        rng = np.random.default_rng(2)
        sites = rng.integers(0, N ** 3, size=5 * N ** 3)          # repeats, several staging passes
        fs, vs, ss = sim.sample_fields(sites)
        assert np.array_equal(fs, f.reshape(nf, -1)[:, sites])
        assert np.array_equal(vs, v.reshape(nf, -1)[:, sites])
        assert (ss.a, ss.ap_half, ss.app, ss.step) == (sc.a, sc.ap_half, sc.app, sc.step)
        empty = sim.sample_fields(np.zeros(0, dtype=np.int64))
        assert empty[0].shape == (nf, 0)
        for bad in ([-1], [N ** 3]):
            with pytest.raises(capi.CeError) as ei:
                sim.sample_fields(bad)
            assert ei.value.code == capi.CE_EINVAL
