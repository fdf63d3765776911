"""CUDA path vs CPU oracle, element by element, through the C ABI.

Tolerances (FP64): relative max error max|gpu - ref| / max|ref| per field and
per velocity array, and |d|/|ref| for scalars, <= 1e-11 after 100 steps.  The
two sides round differently (FMA contraction, summation order of the global
sums, the velocity kept as w + c f), each step adding O(1e-16) relative
error that the dynamics carry forward; 1e-11 leaves about three decades of
margin over 100 steps of these runs.
FP32 storage: errors are reported against the FP64 oracle and checked only
against the 1e-3 statistics bound.
"""
import math

import numpy as np
import pytest

from paper_0712_0813_gb300.icgen import courant_dt, lattice_ics
from step_bounds import check_one_step

pytestmark = pytest.mark.gpu

TOL64 = 1e-11


def relmax(a, b):
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / (den if den > 0 else 1.0))


def per_field_err(a, b, nf):
    a = np.asarray(a).reshape(nf, -1)
    b = np.asarray(b).reshape(nf, -1)
    return max(relmax(a[i], b[i]) for i in range(nf))


def run_pair(orc, capi, dims, N, L, dt, nf, q, expansion, steps, precision="f64", kernel="auto",
             seed=1, phi0=1.0, amp=1e-4):
    f0, u0 = lattice_ics(dims, N, L, nf, phi0=phi0, q=q, seed=seed, amp=amp)
    p = orc.Params(dims=dims, N=N, L=L, dt=dt, nf=nf, q=tuple(q) if q else (0.0,), expansion=expansion)
    ref = orc.init(p, f0, u0)
    orc.step(ref, steps)
    sim = capi.Simulation(dims=dims, N=N, L=L, dt=dt, nfields=nf, q=q, expansion=expansion,
                          precision=precision, kernel=kernel, phi0=phi0)
    sim.set_fields(f0, u0)
    sim.step(steps)
    f, v, sc = sim.get_fields(capi.CE_VEL_STAGGERED)
    return ref, sim, f, v, sc


CASES = [
    # dims, N, L, dt, nf, q, expansion
    (3, 32, 20.0, 0.05, 2, (1.2,), False),   # the plain 32^3 FP64 case
    (3, 32, 20.0, 0.05, 2, (1.2,), True),
    (3, 64, 20.0, 0.02, 2, (1.2,), True),
    (1, 4096, 20.0, 0.004, 2, (1.2,), True),
    (1, 4099, 20.0, 0.004, 2, (1.2,), True),  # 1D tail after the last 16-byte group
    (1, 5, 3.0, 0.05, 1, (), True),
    (2, 256, 20.0, 0.02, 2, (1.2,), True),
    (3, 3, 2.0, 0.05, 2, (1.2,), True),      # every neighbour wraps
    (3, 5, 3.0, 0.05, 1, (), True),
    (3, 37, 20.0, 0.05, 3, (0.8, 5.0), True),  # ragged N
    (3, 20, 20.0, 0.03, 4, (0.8, 5.0, 40.0), True),
    (2, 100, 20.0, 0.05, 4, (0.8, 5.0, 40.0), False),
]


@pytest.mark.parametrize("kernel", ["auto", "generic"])
@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}d_N{c[1]}_nf{c[4]}_{'exp' if c[6] else 'flat'}" for c in CASES])
def test_fp64_parity_100_steps(gpu_capi, orc, case, kernel):
    """The automatic kernel choice, and the generic kernel where that choice is
    another kernel, against the oracle."""
    dims, N, L, dt, nf, q, expansion = case
    if kernel == "generic" and auto_kernel(gpu_capi, dims, N, "f64") == gpu_capi.CE_KERNEL_GENERIC:
        pytest.skip("the automatic choice is the generic kernel")
    ref, sim, f, v, sc = run_pair(orc, gpu_capi, dims, N, L, dt, nf, q, expansion, 100, kernel=kernel)
    with sim:
        assert sim.kernel == (auto_kernel(gpu_capi, dims, N, "f64") if kernel == "auto" else gpu_capi.CE_KERNEL_GENERIC)
        assert per_field_err(f, ref.f, nf) <= TOL64
        assert per_field_err(v, ref.v, nf) <= TOL64
        assert sc.step == 100 and sc.t == ref.scale.t
        if expansion:
            assert abs(sc.a - ref.scale.a) / ref.scale.a <= TOL64
            assert abs(sc.ap_half - ref.scale.ap) / abs(ref.scale.ap) <= TOL64
            assert abs(sc.app - ref.scale.app) / abs(ref.scale.app) <= 1e-9
        else:
            assert sc.a == 1.0 and sc.ap_half == 0.0
        en_ref = orc.energy(ref)
        en = sim.energy()
        for key in ("V", "E", "a", "ap"):
            assert en[key] == pytest.approx(en_ref[key], rel=1e-10, abs=1e-14), key
        np.testing.assert_allclose(en["K"], en_ref["K"], rtol=1e-8, atol=1e-15)
        np.testing.assert_allclose(en["G"], en_ref["G"], rtol=1e-8, atol=1e-15)
        if expansion:
            assert en["friedmann_resid"] == pytest.approx(en_ref["friedmann_resid"], rel=1e-6, abs=1e-12)
        mean, var = sim.means_variances()
        mref, vref = orc.means_variances(ref.p, ref.f)
        np.testing.assert_allclose(mean, mref, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(var, vref, rtol=1e-6, atol=1e-18)
        fs, us, _ = sim.get_fields(gpu_capi.CE_VEL_SYNC)
        assert per_field_err(us, orc.sync_u(ref), nf) <= TOL64


def test_startup_roundtrip_returns_input_velocity(gpu_capi, orc):
    f0, u0 = lattice_ics(3, 16, 20.0, 2, q=(1.2,), seed=5)
    with gpu_capi.Simulation(dims=3, N=16, L=20.0, dt=0.05, nfields=2, q=(1.2,), expansion=True) as sim:
        sim.set_fields(f0, u0)
        f, u, sc = sim.get_fields(gpu_capi.CE_VEL_SYNC)
        assert np.array_equal(f, f0.reshape(-1))
        assert relmax(u, u0) <= 1e-12
        assert sc.step == 0 and sc.t == 0.0 and sc.a == 1.0


def test_checkpoint_roundtrip_is_bit_exact(gpu_capi):
    for precision in ("f64", "f32"):
        cfg = dict(dims=3, N=24, L=20.0, dt=0.05, nfields=2, q=(1.2,), expansion=True, precision=precision)
        f0, u0 = lattice_ics(3, 24, 20.0, 2, q=(1.2,), seed=9)
        with gpu_capi.Simulation(**cfg) as a, gpu_capi.Simulation(**cfg) as b:
            a.set_fields(f0, u0)
            a.step(37)
            fs, vs, sc = a.get_fields(gpu_capi.CE_VEL_STAGGERED)
            b.set_fields(fs, vs, gpu_capi.CE_VEL_STAGGERED, sc)
            a.step(25)
            b.step(25)
            fa, va, sa = a.get_fields(gpu_capi.CE_VEL_STAGGERED)
            fb, vb, sb = b.get_fields(gpu_capi.CE_VEL_STAGGERED)
            assert np.array_equal(fa, fb) and np.array_equal(va, vb), precision
            assert (sa.a, sa.ap_half, sa.app, sa.t, sa.step) == (sb.a, sb.ap_half, sb.app, sb.t, sb.step)


def test_fp32_storage_error_against_fp64_oracle(gpu_capi, orc):
    """FP32 fields/velocities with FP64 sums and a(t): statistics within 1e-3."""
    dims, N, L, dt, nf, q = 3, 32, 20.0, 0.05, 2, (1.2,)
    ref, sim, f, v, sc = run_pair(orc, gpu_capi, dims, N, L, dt, nf, q, True, 100, precision="f32")
    with sim:
        ef = per_field_err(f, ref.f, nf)
        ev = per_field_err(v, ref.v, nf)
        assert ef < 1e-5 and ev < 1e-3, (ef, ev)
        assert abs(sc.a - ref.scale.a) / ref.scale.a < 1e-6
        en = sim.energy()
        en_ref = orc.energy(ref)
        assert en["E"] == pytest.approx(en_ref["E"], rel=1e-3)
        mean, var = sim.means_variances()
        mref, vref = orc.means_variances(ref.p, ref.f)
        # a zero-mean field (chi) is judged against its spread, not its ~1e-11 mean
        scale = np.maximum(np.abs(mref), np.sqrt(vref))
        assert np.all(np.abs(mean - mref) <= 1e-3 * scale), (mean, mref, vref)
        np.testing.assert_allclose(var, vref, rtol=1e-3)


def test_plain_fp64_case_over_its_full_1000_steps(gpu_capi, orc):
    """The plain method in FP64 (3D 32^3, 2 fields, q = 1.2, L = 20, dt = 0.05, no
    expansion, amplitude 1e-4) for the full 1000 steps against the oracle: fields,
    velocities and the energy."""
    dims, N, L, dt, nf, q = 3, 32, 20.0, 0.05, 2, (1.2,)
    ref, sim, f, v, sc = run_pair(orc, gpu_capi, dims, N, L, dt, nf, q, False, 1000)
    with sim:
        assert per_field_err(f, ref.f, nf) <= 1e-10
        assert per_field_err(v, ref.v, nf) <= 1e-10
        assert sc.step == 1000 and sc.a == 1.0
        en, en_ref = sim.energy(), orc.energy(ref)
        assert en["E"] == pytest.approx(en_ref["E"], rel=1e-12)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_long_nonlinear_run_statistics_against_oracle(gpu_capi, orc, precision):
    """A long run in the nonlinear regime (3D 32^3, 2 fields, expansion on,
    amplitude 1e-2, 2000 steps): where the evolution is chaotic, runs are compared
    through means, variances, total energy and a(t), each within 1e-3."""
    dims, N, L, dt, nf, q = 3, 32, 20.0, 0.05, 2, (1.2,)
    ref, sim, f, v, sc = run_pair(orc, gpu_capi, dims, N, L, dt, nf, q, True, 2000, precision=precision,
                                  amp=1e-2)
    with sim:
        assert sc.step == 2000
        assert abs(sc.a - ref.scale.a) <= 1e-3 * ref.scale.a
        en, en_ref = sim.energy(), orc.energy(ref)
        assert en["E"] == pytest.approx(en_ref["E"], rel=1e-3)
        mean, var = sim.means_variances()
        mref, vref = orc.means_variances(ref.p, ref.f)
        scale = np.maximum(np.abs(mref), np.sqrt(vref))
        assert np.all(np.abs(mean - mref) <= 1e-3 * scale), (mean, mref)
        np.testing.assert_allclose(var, vref, rtol=1e-3)


def test_nonfinite_state_is_reported_not_faulted(gpu_capi):
    """A state whose potential overflows makes the global sums non-finite: the
    device latches CE_ENONFINITE and the next synchronising call returns it."""
    N = 8
    f0 = np.zeros((2, N ** 3))
    f0[0] = 1e200
    u0 = np.zeros_like(f0)
    with gpu_capi.Simulation(dims=3, N=N, L=20.0, dt=0.05, nfields=2, q=(1.2,), expansion=True) as sim:
        with pytest.raises(gpu_capi.CeError) as ei:
            sim.set_fields(f0, u0)
        assert ei.value.code == gpu_capi.CE_ENONFINITE


def test_step_before_set_fields_is_a_state_error(gpu_capi):
    with gpu_capi.Simulation(dims=3, N=8, L=20.0, dt=0.05) as sim:
        with pytest.raises(gpu_capi.CeError) as ei:
            sim.step(1)
        assert ei.value.code == gpu_capi.CE_ESTATE


def test_zero_steps_and_torch_stream_and_allocator(gpu_capi, orc):
    import torch
    s = torch.cuda.Stream()
    f0, u0 = lattice_ics(3, 16, 20.0, 2, q=(1.2,), seed=3)
    with gpu_capi.Simulation(dims=3, N=16, L=20.0, dt=0.05, nfields=2, q=(1.2,), expansion=True,
                             stream=s.cuda_stream, torch_allocator=True) as sim:
        sim.set_fields(f0, u0)
        sim.step(0)
        sim.step(10)
        f, v, sc = sim.get_fields(gpu_capi.CE_VEL_STAGGERED)
    p = orc.Params(dims=3, N=16, L=20.0, dt=0.05, nf=2, q=(1.2,), expansion=True)
    ref = orc.step(orc.init(p, f0, u0), 10)
    assert per_field_err(f, ref.f, 2) <= TOL64


# ---------------------------------------------------------------- z-sweep kernel

@pytest.mark.parametrize("nf,q", [(1, ()), (2, (1.2,)), (3, (0.8, 5.0)), (4, (0.8, 5.0, 40.0))])
def test_sweep_kernel_matches_generic_fp64(gpu_capi, nf, q):
    """Decomposition invariance: the tiled z-sweep and the one-thread-per-site
    kernel agree to rounding (their global sums are added in different orders)."""
    N, dt = 64, 0.02
    f0, u0 = lattice_ics(3, N, 20.0, nf, q=q, seed=4, amp=1e-2)
    out = {}
    for kernel in ("generic", "sweep"):
        with gpu_capi.Simulation(dims=3, N=N, L=20.0, dt=dt, nfields=nf, q=q, expansion=True,
                                 kernel=kernel) as sim:
            assert sim.kernel == {"generic": 1, "sweep": 2}[kernel]
            sim.set_fields(f0, u0)
            sim.step(60)
            out[kernel] = sim.get_fields(gpu_capi.CE_VEL_STAGGERED)
    fg, vg, sg = out["generic"]
    fs, vs, ss = out["sweep"]
    assert per_field_err(fs, fg, nf) <= 1e-12
    assert per_field_err(vs, vg, nf) <= 1e-12
    assert abs(ss.a - sg.a) <= 1e-13 * sg.a


def test_sweep_kernel_matches_generic_fp32(gpu_capi):
    N, nf, q = 128, 2, (1.2,)
    f0, u0 = lattice_ics(3, N, 20.0, nf, q=q, seed=6)
    out = {}
    for kernel in ("generic", "sweep"):
        with gpu_capi.Simulation(dims=3, N=N, L=20.0, dt=0.02, nfields=nf, q=q, expansion=True,
                                 precision="f32", kernel=kernel) as sim:
            sim.set_fields(f0, u0)
            sim.step(40)
            out[kernel] = sim.get_fields(gpu_capi.CE_VEL_STAGGERED)
    assert per_field_err(out["sweep"][0], out["generic"][0], nf) <= 1e-6
    assert per_field_err(out["sweep"][1], out["generic"][1], nf) <= 1e-4


@pytest.mark.parametrize("N,steps,nf,q", [(64, 100, 2, (1.2,)), (128, 10, 4, (0.8, 5.0, 40.0))])
def test_sweep_kernel_fp64_vs_oracle(gpu_capi, orc, N, steps, nf, q):
    dt = 0.02 if nf == 2 else 0.01
    ref, sim, f, v, sc = run_pair(orc, gpu_capi, 3, N, 20.0, dt, nf, q, True, steps, kernel="sweep")
    with sim:
        assert sim.kernel == gpu_capi.CE_KERNEL_SWEEP
        assert per_field_err(f, ref.f, nf) <= TOL64
        assert per_field_err(v, ref.v, nf) <= TOL64
        assert abs(sc.a - ref.scale.a) / ref.scale.a <= TOL64


@pytest.mark.parametrize("precision,tol_f,tol_v", [("f32", 2e-6, 2e-5), ("f64", 1e-13, 1e-12)])
def test_full_size_256cube_one_step_against_oracle(gpu_capi, orc, precision, tol_f, tol_v):
    """The bench workload (3D 256^3, 2 fields, expansion, dt = 0.02) in the
    launch configuration the bench times: after 20 GPU steps the exported
    state is stepped once by the oracle (FP64) and once by the GPU, and every
    site is compared."""
    N, nf, q, dt, L = 256, 2, (1.2,), 0.02, 20.0
    f0, u0 = lattice_ics(3, N, L, nf, q=q, seed=1)
    with gpu_capi.Simulation(dims=3, N=N, L=L, dt=dt, nfields=nf, q=q, expansion=True,
                             precision=precision, kernel="sweep") as sim:
        assert sim.kernel == gpu_capi.CE_KERNEL_SWEEP
        sim.set_fields(f0, u0)
        sim.step(20)
        fs, vs, sc = sim.get_fields(gpu_capi.CE_VEL_STAGGERED)
        sim.step(1)
        f1, v1, sc1 = sim.get_fields(gpu_capi.CE_VEL_STAGGERED)
    p = orc.Params(dims=3, N=N, L=L, dt=dt, nf=nf, q=q, expansion=True)
    st = orc.State(p, fs.copy(), vs.copy(), orc.Scale(sc.a, sc.ap_half, sc.app, sc.t, sc.step))
    orc.step(st, 1)
    assert per_field_err(f1, st.f, nf) <= tol_f
    assert per_field_err(v1, st.v, nf) <= tol_v
    assert abs(sc1.a - st.scale.a) <= 1e-12 * st.scale.a
    if precision == "f64":
        assert abs(sc1.ap_half - st.scale.ap) <= 1e-9 * abs(st.scale.ap)
    else:
        # G and V come from FP32 per-thread partial sums (folded into FP64 per
        # block): a'' is good to ~1e-5 of its source term Q, |Q| <= |a''| + a'^2/a,
        # so one step moves a' by at most 1e-5 dt of that (the full-size tests' bound)
        scale = abs(st.scale.app) + st.scale.ap ** 2 / st.scale.a
        assert abs(sc1.ap_half - st.scale.ap) <= 1e-5 * dt * scale + 1e-12 * abs(st.scale.ap)


VARIANTS = [(8, 4), (8, 5), (16, 3), (16, 4), (4, 4), (4, 5)]


@pytest.mark.parametrize("rows,stages", VARIANTS)
@pytest.mark.parametrize("zchunks", [1, 3, 8])
def test_sweep_variants_and_directions_match_generic_fp64(gpu_capi, rows, stages, zchunks):
    """Every compiled (rows, stages) variant, with odd and even numbers of
    z-chunks (neighbouring chunks sweep in opposite directions), agrees with
    the one-thread-per-site kernel."""
    N, nf, q = 64, 2, (1.2,)
    f0, u0 = lattice_ics(3, N, 20.0, nf, q=q, seed=12, amp=1e-2)
    out = {}
    for kernel in ("generic", "sweep"):
        kw = dict(tile_rows=rows, stages=stages, zchunks=zchunks) if kernel == "sweep" else {}
        with gpu_capi.Simulation(dims=3, N=N, L=20.0, dt=0.02, nfields=nf, q=q, expansion=True,
                                 kernel=kernel, **kw) as sim:
            if kernel == "sweep":
                assert sim.sweep_plan == (rows, stages, zchunks)
            sim.set_fields(f0, u0)
            sim.step(33)
            out[kernel] = sim.get_fields(gpu_capi.CE_VEL_STAGGERED)
    assert per_field_err(out["sweep"][0], out["generic"][0], nf) <= 1e-12
    assert per_field_err(out["sweep"][1], out["generic"][1], nf) <= 1e-12
    assert abs(out["sweep"][2].a - out["generic"][2].a) <= 1e-13 * out["generic"][2].a


def test_automatic_choice_in_fp64_and_plan_hints(gpu_capi):
    """FP64 2D/3D lattices run the generic kernel's two-pass form (measured faster
    than the z-sweep and row kernels there); z-sweep plan hints select the z-sweep
    kernel."""
    kw = dict(dims=3, N=128, L=20.0, dt=0.02, nfields=2, q=(1.2,), expansion=True, precision="f64")
    with gpu_capi.Simulation(**kw) as sim:
        assert sim.kernel == gpu_capi.CE_KERNEL_GENERIC
        assert sim.sweep_plan == (0, 0, 0)
    with gpu_capi.Simulation(**kw, tile_rows=8) as sim:
        assert sim.kernel == gpu_capi.CE_KERNEL_SWEEP
        assert sim.sweep_plan[0] == 8
    with gpu_capi.Simulation(**dict(kw, dims=2, N=1024, dt=courant_dt(2, 1024, 20.0, 1.0, (1.2,)))) as sim:
        assert sim.kernel == gpu_capi.CE_KERNEL_GENERIC


def test_automatic_plan_of_the_256cube_lattice(gpu_capi):
    """Without hints the bench lattice (3D 256^3, 2 fields, FP32) gets the plan the
    autotuner measures fastest on a GB300 (152 SMs): 8 rows, 4 stages, 4
    z-chunks, 0.84 of a wave of 304 CTAs, which the launch model prefers to the
    14 chunks that would fill whole waves (101.6 against 93.3 us per step)."""
    with gpu_capi.Simulation(dims=3, N=256, L=20.0, dt=0.02, nfields=2, q=(1.2,), expansion=True,
                             precision="f32") as sim:
        assert sim.kernel == gpu_capi.CE_KERNEL_SWEEP
        assert sim.sweep_plan == (8, 4, 4)


@pytest.mark.parametrize("rows,stages", VARIANTS)
def test_sweep_variants_fp32_vs_oracle(gpu_capi, orc, rows, stages):
    N, nf, q, dt = 128, 2, (1.2,), 0.02
    f0, u0 = lattice_ics(3, N, 20.0, nf, q=q, seed=13)
    p = orc.Params(dims=3, N=N, L=20.0, dt=dt, nf=nf, q=q, expansion=True)
    ref = orc.step(orc.init(p, f0, u0), 5)
    with gpu_capi.Simulation(dims=3, N=N, L=20.0, dt=dt, nfields=nf, q=q, expansion=True, precision="f32",
                             kernel="sweep", tile_rows=rows, stages=stages, zchunks=5) as sim:
        sim.set_fields(f0, u0)
        sim.step(5)
        f, v, sc = sim.get_fields(gpu_capi.CE_VEL_STAGGERED)
    assert per_field_err(f, ref.f, nf) <= 2e-6
    assert per_field_err(v, ref.v, nf) <= 2e-5


@pytest.mark.parametrize("N,nf,precision", [(4096, 1, "f64"), (4096, 4, "f64"), (1001, 2, "f64"), (8, 3, "f64"),
                                          (65536, 2, "f64"), (4, 2, "f32"), (4096, 2, "f32"), (65536, 2, "f32")])
def test_1d_kernel_vs_oracle(gpu_capi, orc, N, nf, precision):
    """1D lattices on the generic path: sides that are multiples of the 16-byte
    vector take the vectorised 1D kernel (down to a single vector of sites, whose
    two neighbours wrap onto itself), other sides the one-thread-per-site kernel.
    FP64: 40 steps against the oracle.  FP32: after 20 steps, one step from the
    exported state at every site within the derived FP32 one-step bound (over
    many steps FP32 storage drifts from the FP64 oracle whatever the kernel: on
    the 65536-site lattice the Laplacian's 1/dx^2 ~ 1e7 weight makes that ~1e-3
    of v in 40 steps)."""
    from oracle import local
    q = (0.8, 5.0, 40.0)[: nf - 1]
    L = 20.0
    dt = courant_dt(1, N, L, 1.0, q)
    f0, u0 = lattice_ics(1, N, L, nf, q=q, seed=1, amp=1e-2)
    p = orc.Params(dims=1, N=N, L=L, dt=dt, nf=nf, q=q, expansion=True)
    with gpu_capi.Simulation(dims=1, N=N, L=L, dt=dt, nfields=nf, q=q, expansion=True, precision=precision,
                             kernel="generic") as sim:
        assert sim.kernel == gpu_capi.CE_KERNEL_GENERIC
        sim.set_fields(f0, u0)
        if precision == "f64":
            ref = orc.step(orc.init(p, f0, u0), 40)
            sim.step(40)
            f, v, sc = sim.get_fields(gpu_capi.CE_VEL_STAGGERED)
            assert per_field_err(f, ref.f, nf) <= TOL64
            assert per_field_err(v, ref.v, nf) <= TOL64
            assert abs(sc.a - ref.scale.a) <= 1e-12 * ref.scale.a
        else:
            sim.step(20)
            sites = np.arange(N, dtype=np.int64)
            stencil = local.stencil_sites(1, N, sites)
            before = sim.sample_fields(stencil)
            sim.step(1)
            after = sim.sample_fields(sites)
            en = sim.energy()
            check_one_step(orc, local, p, before, after, sites, stencil, float(np.sum(en["G"])), en["V"])


def auto_kernel(capi, dims, N, precision):
    """The kernel ce_create picks by itself (no plan hints).  FP32: the z-sweep
    kernel for 3D sides that are multiples of its tile, the row kernel for other
    2D/3D lattices it takes with sides >= 256 (3D) or 512 (2D), the column
    kernel (CE_KERNEL_PLANES) for the other 3D lattices and the line-sweep kernel
    (the same id) for the other 2D sides >= 320, the generic kernel for the rest.
    FP64: the generic kernel (its two-pass form in 2D/3D)."""
    if precision == "f64":
        return capi.CE_KERNEL_GENERIC
    if dims == 3 and N % 128 == 0:
        return capi.CE_KERNEL_SWEEP
    if dims >= 2 and N % 4 == 0 and N >= (256 if dims == 3 else 512):
        return capi.CE_KERNEL_ROWS
    if dims == 3 or (dims == 2 and N >= 320):
        return capi.CE_KERNEL_PLANES
    return capi.CE_KERNEL_GENERIC


@pytest.mark.parametrize("dims,N,precision", [(3, 96, "f64"), (2, 130, "f64"), (1, 2048, "f64"), (3, 40, "f32"),
                                              (3, 68, "f32"), (2, 520, "f32")])
def test_row_kernel_single_lattice(gpu_capi, orc, dims, N, precision):
    """ce_step through the batched row-sweep kernel on one lattice (CE_KERNEL_ROWS,
    an explicit choice) against the oracle; the item length along the sweep axis
    is the one ce_create's launch model picks for the lattice."""
    q, nf = (1.2,), 2
    dt = 0.02 if dims > 1 else 0.004
    ref, sim, f, v, sc = run_pair(orc, gpu_capi, dims, N, 20.0, dt, nf, q, True, 40, precision=precision,
                                  kernel="rows", amp=1e-2)
    with sim:
        assert sim.kernel == gpu_capi.CE_KERNEL_ROWS
        tol_f, tol_v = (TOL64, TOL64) if precision == "f64" else (2e-6, 2e-4)
        assert per_field_err(f, ref.f, nf) <= tol_f
        assert per_field_err(v, ref.v, nf) <= tol_v
    with gpu_capi.Simulation(dims=dims, N=N, L=20.0, dt=dt, nfields=nf, q=q, precision=precision) as auto:
        assert auto.kernel == auto_kernel(gpu_capi, dims, N, precision)


# N, nf, q, dt, steps for the column kernel (strips of 30 x-sites; FP64 row
# groups of 4 rows for one field, 2 for more): every neighbour wraps (3, 5), a
# 1-site-wide last strip with a 3-row last row group (31), a 3-site last strip
# with a 1-row last group (33), ragged strips, groups and z-chunks (37, 45,
# 195: a 15-site last strip, a 1-row last group)
PLANES_CASES = [(3, 2, (1.2,), 0.05, 100), (5, 1, (), 0.05, 100), (31, 1, (), 0.05, 100), (33, 2, (1.2,), 0.05, 100),
                (37, 3, (0.8, 5.0), 0.05, 100), (45, 4, (0.8, 5.0, 40.0), 0.02, 100), (195, 2, (1.2,), 0.02, 6)]


@pytest.mark.parametrize("N,nf,q,dt,steps", PLANES_CASES, ids=[f"N{c[0]}_nf{c[1]}" for c in PLANES_CASES])
def test_planes_kernel_fp64_vs_oracle(gpu_capi, orc, N, nf, q, dt, steps):
    """The 3D column kernel (CE_KERNEL_PLANES: plain loads, any N) against the oracle with
    expansion, FP64 (100 steps; 6 on the 195^3 lattice, which the oracle
    steps in about a second each)."""
    L = 20.0 if N > 5 else 3.0
    ref, sim, f, v, sc = run_pair(orc, gpu_capi, 3, N, L, dt, nf, q, True, steps, kernel="planes", amp=1e-2)
    with sim:
        assert sim.kernel == gpu_capi.CE_KERNEL_PLANES
        assert per_field_err(f, ref.f, nf) <= TOL64
        assert per_field_err(v, ref.v, nf) <= TOL64
        assert abs(sc.a - ref.scale.a) / ref.scale.a <= TOL64
        assert abs(sc.ap_half - ref.scale.ap) / abs(ref.scale.ap) <= TOL64


# FP32 column kernel, 2 fields: row groups of 4 rows below side 160, 6 from it;
# 1-site last strips (61, 31 + 30), 1-row last groups (33, 37, 61, 101), a 5-row
# (197) and a 3-row (225) last group
@pytest.mark.parametrize("N", [3, 33, 37, 61, 101, 197, 225])
def test_planes_kernel_fields_equal_generic_fp32(gpu_capi, N):
    """Per site the column kernel does the generic kernel's arithmetic:
    without expansion (no global sums feed back) the FP32 fields agree bit for
    bit over many steps.  With expansion, after one step f agrees bit for bit;
    the staggered velocity w + c f takes c = dt a''/a of the next step, whose
    a'' comes from the step's FP32 partial sums, added in another order by each
    kernel, so v agrees to the rounding of those sums.  The automatic FP32
    choice for these sides is the column kernel."""
    nf, q = 2, (1.2,)
    f0, u0 = lattice_ics(3, N, 20.0, nf, q=q, seed=4, amp=1e-2)
    for expansion, steps in ((False, 20), (True, 1)):
        out = []
        for kernel in ("auto", "generic"):
            with gpu_capi.Simulation(dims=3, N=N, L=20.0, dt=0.02, nfields=nf, q=q, expansion=expansion,
                                     precision="f32", kernel=kernel) as sim:
                assert sim.kernel == (gpu_capi.CE_KERNEL_PLANES if kernel == "auto" else gpu_capi.CE_KERNEL_GENERIC)
                sim.set_fields(f0, u0)
                sim.step(steps)
                out.append(sim.get_fields(gpu_capi.CE_VEL_STAGGERED))
        (fa, va, sa), (fb, vb, sb) = out
        assert np.array_equal(fa, fb), (N, expansion)
        if expansion:
            assert np.max(np.abs(va - vb)) <= 1e-6 * (np.max(np.abs(vb)) + np.max(np.abs(fb))), N
        else:
            assert np.array_equal(va, vb), N
        assert abs(sa.a - sb.a) <= 1e-15 * sb.a


# 2D line-sweep kernel (strips of 30 x-sites): N, nf, q: every neighbour wraps
# (3), a 1-site-wide last strip (31, 61: its right halo on lane 2), a 3-site
# last strip (33), ragged (37, 65, 101), a side that is a multiple of the strip (90)
LINES_CASES = [(3, 2, (1.2,)), (31, 1, ()), (33, 2, (1.2,)), (37, 3, (0.8, 5.0)), (61, 2, (1.2,)), (65, 1, ()),
               (90, 4, (0.8, 5.0, 40.0)), (101, 2, (1.2,))]


@pytest.mark.parametrize("N,nf,q", LINES_CASES, ids=[f"N{c[0]}_nf{c[1]}" for c in LINES_CASES])
def test_lines_kernel_fp64_vs_oracle(gpu_capi, orc, N, nf, q):
    """The 2D line-sweep kernel (CE_KERNEL_PLANES in 2D) against the oracle over
    100 steps with expansion, FP64."""
    L = 20.0 if N > 5 else 3.0
    ref, sim, f, v, sc = run_pair(orc, gpu_capi, 2, N, L, 0.02, nf, q, True, 100, kernel="planes", amp=1e-2)
    with sim:
        assert sim.kernel == gpu_capi.CE_KERNEL_PLANES
        assert per_field_err(f, ref.f, nf) <= TOL64
        assert per_field_err(v, ref.v, nf) <= TOL64
        assert abs(sc.a - ref.scale.a) / ref.scale.a <= TOL64
        assert abs(sc.ap_half - ref.scale.ap) / abs(ref.scale.ap) <= TOL64


@pytest.mark.parametrize("N", [3, 31, 33, 37, 61, 101, 1001])
def test_lines_kernel_fields_equal_generic_fp32(gpu_capi, N):
    """Per site the 2D line-sweep kernel does the generic kernel's arithmetic:
    FP32 fields bit-identical over many steps without expansion; with it, f
    bit-identical after one step and the staggered velocity equal to the
    rounding of the step's sums (see the column-kernel test)."""
    nf, q = 2, (1.2,)
    f0, u0 = lattice_ics(2, N, 20.0, nf, q=q, seed=4, amp=1e-2)
    dt = courant_dt(2, N, 20.0, 1.0, q)
    for expansion, steps in ((False, 20), (True, 1)):
        out = []
        for kernel in ("planes", "generic"):
            with gpu_capi.Simulation(dims=2, N=N, L=20.0, dt=dt, nfields=nf, q=q, expansion=expansion,
                                     precision="f32", kernel=kernel) as sim:
                assert sim.kernel == (gpu_capi.CE_KERNEL_PLANES if kernel == "planes" else gpu_capi.CE_KERNEL_GENERIC)
                sim.set_fields(f0, u0)
                sim.step(steps)
                out.append(sim.get_fields(gpu_capi.CE_VEL_STAGGERED))
        (fa, va, sa), (fb, vb, sb) = out
        assert np.array_equal(fa, fb), (N, expansion)
        if expansion:
            assert np.max(np.abs(va - vb)) <= 1e-6 * (np.max(np.abs(vb)) + np.max(np.abs(fb))), N
        else:
            assert np.array_equal(va, vb), N
        assert abs(sa.a - sb.a) <= 1e-15 * sb.a


@pytest.mark.parametrize("N,expected", [(1001, "planes"), (6001, "planes"), (385, "planes"), (257, "generic"),
                                        (1024, "rows")])
def test_automatic_choice_2d_fp32(gpu_capi, N, expected):
    """FP32 2D: the row kernel for sides >= 512 that are multiples of 4, the
    line-sweep kernel for the other sides >= 320, the generic kernel below."""
    ids = {"planes": gpu_capi.CE_KERNEL_PLANES, "generic": gpu_capi.CE_KERNEL_GENERIC, "rows": gpu_capi.CE_KERNEL_ROWS}
    with gpu_capi.Simulation(dims=2, N=N, L=20.0, dt=courant_dt(2, N, 20.0, 1.0, (1.2,)), nfields=2, q=(1.2,),
                             precision="f32") as sim:
        assert sim.kernel == ids[expected] == auto_kernel(gpu_capi, 2, N, "f32")


@pytest.mark.parametrize("precision", ["f32", "f64"])
@pytest.mark.parametrize("N", [3, 5, 7, 4097, 4099])
def test_1d_ragged_shift_invariance(gpu_capi, N, precision):
    """1D sides that are not a multiple of the 16-byte group (4 sites in FP32,
    2 in FP64): the sites after the last whole group take the one-site path,
    the others the grouped one, with the same per-site arithmetic.  Without
    expansion (no global sums feed back) a periodic shift of the initial state
    then shifts the result bit for bit after 20 steps, whichever sites fall in
    the tail (sides below one group are all tail)."""
    L, q = 3.0 if N < 10 else 20.0, (1.2,)
    f0, u0 = lattice_ics(1, N, L, 2, q=q, seed=6, amp=1e-2)
    f0, u0 = np.asarray(f0).reshape(2, N), np.asarray(u0).reshape(2, N)
    dt = courant_dt(1, N, L, 1.0, q)
    out = []
    for shift in (0, 1):
        with gpu_capi.Simulation(dims=1, N=N, L=L, dt=dt, nfields=2, q=q, expansion=False,
                                 precision=precision) as sim:
            sim.set_fields(np.roll(f0, shift, axis=-1), np.roll(u0, shift, axis=-1))
            sim.step(20)
            f, v, _ = sim.get_fields(gpu_capi.CE_VEL_STAGGERED)
            out.append((np.asarray(f).reshape(2, N), np.asarray(v).reshape(2, N)))
    (f, v), (fs, vs) = out
    assert np.array_equal(np.roll(f, 1, axis=-1), fs) and np.array_equal(np.roll(v, 1, axis=-1), vs), N
