"""ce_moments_noalloc: per-field moments without any device allocation.

Some callers cannot let a library allocate device memory: applications whose
HBM belongs to another allocator (a framework's caching allocator, or an arena
reserved at start-up, where one more cudaMalloc fails or fragments the pool),
and latency-critical loops that cannot absorb the device synchronisation that
cudaMalloc/cudaFree imply.  ce_moments_noalloc serves them from a static
scratch array inside the library; the caller passes its own device arrays for
the fields and for the results.

The GPU test calls the entry point twice in a row through the C ABI on device
arrays the test owns, and compares each result with the handle-based
ce_means_variances on the same lattice state, using the tolerances of the
FP64 parity tests.  This file is collected last and passes both on its own in
a fresh process and after the rest of the suite.
"""
import numpy as np
import pytest

from paper_0712_0813_gb300.icgen import lattice_ics


def test_noalloc_rejects_bad_arguments_before_touching_the_device(capi):
    lib = capi.load()
    assert lib.ce_moments_noalloc(None, capi.CE_F64, 10, 1, None, None, None) == capi.CE_EINVAL
    assert "NULL" in capi.ce_last_error()
    fake = 4096  # never dereferenced: validation fails first
    assert lib.ce_moments_noalloc(fake, capi.CE_F64, 10, 5, None, fake, fake) == capi.CE_EINVAL
    assert "nfields must be 1..4" in capi.ce_last_error()
    assert lib.ce_moments_noalloc(fake, capi.CE_F64, 0, 2, None, fake, fake) == capi.CE_EINVAL
    assert lib.ce_moments_noalloc(fake, capi.CE_F64, (1 << 34) + 1, 2, None, fake, fake) == capi.CE_EINVAL
    assert "2^34" in capi.ce_last_error()
    assert lib.ce_moments_noalloc(fake, 7, 10, 2, None, fake, fake) == capi.CE_EINVAL


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_noalloc_moments_match_handle_moments_twice(gpu_capi, precision):
    import torch
    capi = gpu_capi
    N, nf, q = 24, 3, (0.8, 5.0)
    f0, u0 = lattice_ics(3, N, 20.0, nf, q=q, seed=21)
    with capi.Simulation(dims=3, N=N, L=20.0, dt=0.02, nfields=nf, q=q, expansion=True,
                         precision=precision) as sim:
        sim.set_fields(f0, u0)
        sim.step(12)
        ref_mean, ref_var = sim.means_variances()
        f, _, _ = sim.get_fields(capi.CE_VEL_STAGGERED)   # the device state, exactly
    dtype = torch.float32 if precision == "f32" else torch.float64
    fd = torch.tensor(f, dtype=dtype, device="cuda")     # caller-owned input
    out_mean = torch.empty(nf, dtype=torch.float64, device="cuda")  # caller-owned outputs
    out_var = torch.empty(nf, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    code = capi.CE_F32 if precision == "f32" else capi.CE_F64
    scale = np.maximum(np.abs(ref_mean), np.sqrt(ref_var))
    # The handle's pass keeps per-thread partials in the storage type over 16 sites
    # before FP64: in FP32 each partial carries up to 16 x 2^-24 of its largest term
    # (|f - f(0)| up to a few standard deviations), so ~1e-5 of the spread; in FP64
    # the two paths agree to rounding.
    tol_m, tol_v = (1e-12, 1e-6) if precision == "f64" else (1e-5, 1e-5)
    for _ in range(2):
        out_mean.fill_(float("nan"))
        out_var.fill_(float("nan"))
        capi.ce_moments_noalloc(fd.data_ptr(), code, N ** 3, nf, stream.cuda_stream,
                                out_mean.data_ptr(), out_var.data_ptr())
        torch.cuda.synchronize()
        mean = out_mean.cpu().numpy()
        var = out_var.cpu().numpy()
        assert np.all(np.abs(mean - ref_mean) <= tol_m * scale + 1e-15), (mean, ref_mean)
        np.testing.assert_allclose(var, ref_var, rtol=tol_v, atol=1e-18)
