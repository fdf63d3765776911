"""ce_moments_noalloc: per-field moments without any device allocation.

Some callers cannot let a library allocate device memory: applications whose
HBM belongs to another allocator (a framework's caching allocator, or an arena
reserved at start-up, where one more cudaMalloc fails or fragments the pool),
and latency-critical loops that cannot absorb the device synchronisation that
cudaMalloc/cudaFree imply.  ce_moments_noalloc serves them from a static
scratch array inside the library; the caller passes its own device arrays for
the fields and for the results.

The GPU tests call the entry point twice in a row through the C ABI on device
arrays the test owns, and compare each result with the handle-based
ce_means_variances on the same lattice state and with the oracle's moments of
that state; a lattice of 2^21 sites with 4 fields runs the partial-sum pass
over several grid strides, a single site checks the degenerate n = 1, and
hundreds of calls leave the device's free memory unchanged.  This file is
collected last and passes both on its own in a fresh process and after the
rest of the suite.
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


CASES = [
    # dims, N, nfields, couplings: a small lattice, and 2^21 sites x 4 fields so that
    # the partial-sum pass's grid-stride loop runs several rounds and every block
    # writes a non-trivial partial
    (3, 24, 3, (0.8, 5.0)),
    (3, 128, 4, (0.8, 5.0, 40.0)),
]


def _noalloc_moments(capi, torch, fd, code, n, nf, out_mean, out_var):
    out_mean.fill_(float("nan"))
    out_var.fill_(float("nan"))
    capi.ce_moments_noalloc(fd.data_ptr(), code, n, nf, torch.cuda.current_stream().cuda_stream,
                            out_mean.data_ptr(), out_var.data_ptr())
    torch.cuda.synchronize()
    return out_mean.cpu().numpy(), out_var.cpu().numpy()


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("dims,N,nf,q", CASES, ids=[f"{c[1]}cube_nf{c[2]}" for c in CASES])
def test_noalloc_moments_match_handle_and_oracle_twice(gpu_capi, orc, precision, dims, N, nf, q):
    """Two calls in a row on caller-owned device arrays agree with the handle's
    ce_means_variances on the same state and with the oracle's two-pass FP64
    moments of that state (exported exactly, ce_get_fields), and leave the
    device's free memory unchanged over many calls."""
    import torch
    capi = gpu_capi
    f0, u0 = lattice_ics(dims, N, 20.0, nf, q=q, seed=21)
    with capi.Simulation(dims=dims, N=N, L=20.0, dt=0.02, nfields=nf, q=q, expansion=True,
                         precision=precision) as sim:
        sim.set_fields(f0, u0)
        sim.step(12)
        ref_mean, ref_var = sim.means_variances()
        f, _, _ = sim.get_fields(capi.CE_VEL_STAGGERED)   # the device state, exactly
    p = orc.Params(dims=dims, N=N, L=20.0, dt=0.02, nf=nf, q=q)
    orc_mean, orc_var = orc.means_variances(p, f)
    n = N ** dims
    dtype = torch.float32 if precision == "f32" else torch.float64
    fd = torch.tensor(f, dtype=dtype, device="cuda")     # caller-owned input
    out_mean = torch.empty(nf, dtype=torch.float64, device="cuda")  # caller-owned outputs
    out_var = torch.empty(nf, dtype=torch.float64, device="cuda")
    code = capi.CE_F32 if precision == "f32" else capi.CE_F64
    scale = np.maximum(np.abs(ref_mean), np.sqrt(ref_var))
    # The handle's pass keeps per-thread partials in the storage type over 16 sites
    # before FP64: in FP32 each partial carries up to 16 x 2^-24 of its largest term
    # (|f - f(0)| up to a few standard deviations), so ~1e-5 of the spread.  In FP64
    # both paths, and the oracle, agree to rounding: shifted one-pass sums of
    # (f - f(0)) against the two-pass definition differ by a few ulps of the
    # spread times the number of additions in a partial.
    tol_m, tol_v = (1e-12, 1e-10) if precision == "f64" else (1e-5, 1e-5)
    for _ in range(2):
        mean, var = _noalloc_moments(capi, torch, fd, code, n, nf, out_mean, out_var)
        assert np.all(np.abs(mean - ref_mean) <= tol_m * scale + 1e-15), (mean, ref_mean)
        np.testing.assert_allclose(var, ref_var, rtol=tol_v, atol=1e-18)
        # the input values are the stored ones, so against the oracle only the
        # summation differs: FP64 accumulation on both sides
        assert np.all(np.abs(mean - orc_mean) <= 1e-12 * scale + 1e-15), (mean, orc_mean)
        np.testing.assert_allclose(var, orc_var, rtol=1e-10, atol=1e-18)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(200):
        capi.ce_moments_noalloc(fd.data_ptr(), code, n, nf, torch.cuda.current_stream().cuda_stream,
                                out_mean.data_ptr(), out_var.data_ptr())
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_noalloc_single_site(gpu_capi, precision):
    """n = 1: each field's mean is its one value and its variance is 0."""
    import torch
    capi = gpu_capi
    vals = np.array([1.25, -3.5, 0.0, 7.0])
    dtype = torch.float32 if precision == "f32" else torch.float64
    fd = torch.tensor(vals, dtype=dtype, device="cuda")
    out_mean = torch.empty(4, dtype=torch.float64, device="cuda")
    out_var = torch.empty(4, dtype=torch.float64, device="cuda")
    code = capi.CE_F32 if precision == "f32" else capi.CE_F64
    for _ in range(2):
        mean, var = _noalloc_moments(capi, torch, fd, code, 1, 4, out_mean, out_var)
        assert np.array_equal(mean, vals) and np.array_equal(var, np.zeros(4))
