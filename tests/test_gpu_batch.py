"""Batched persistent kernel (ce_batch_*): many lattices, one launch per step.

* Each member of a mixed 1D/2D/3D batch matches the FP64 oracle (<= 1e-11
  relative max error after 30 steps), including ragged row segments (N not a
  multiple of the segment), every 3D segment width (32, 16 and 8 lanes per
  row), partial row groups, 1D lattices over several blocks of the 1D launch
  with a partial last block, and lattices with and without expansion in the
  same launch; a batch of 1D lattices only (no persistent launch) as well.
* "The same alone and in the mix": a lattice advanced in a batch of one and
  inside the mix is bit-identical (its items and their summation order do not
  depend on the other members), in FP32 and FP64.
"""
import numpy as np
import pytest

from paper_0712_0813_gb300.icgen import lattice_ics

pytestmark = pytest.mark.gpu

# dims, N, nf, q, expansion, dt
MIX = [
    (3, 32, 2, (1.2,), True, 0.05),
    (3, 48, 2, (1.2,), True, 0.05),     # 12 valid lanes (FP32), 24 (FP64)
    (3, 20, 2, (1.2,), False, 0.05),    # partial 8-row group
    (2, 100, 2, (1.2,), True, 0.05),
    (2, 256, 2, (5.0,), True, 0.02),
    (1, 4096, 2, (1.2,), True, 0.004),
    (1, 2600, 2, (3.0,), True, 0.004),  # full blocks + a partial last block
    (1, 36, 2, (40.0,), False, 0.02),
]


def relmax(a, b):
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def make_sim(capi, case, precision, seed):
    dims, N, nf, q, expansion, dt = case
    f0, u0 = lattice_ics(dims, N, 20.0, nf, q=q, seed=seed, amp=1e-2)
    sim = capi.Simulation(dims=dims, N=N, L=20.0, dt=dt, nfields=nf, q=q, expansion=expansion,
                          precision=precision, kernel="generic")
    sim.set_fields(f0, u0)
    return sim, f0, u0


def test_batch_members_match_oracle_fp64(gpu_capi, orc):
    capi = gpu_capi
    sims, inputs = [], []
    for k, case in enumerate(MIX):
        sim, f0, u0 = make_sim(capi, case, "f64", 100 + k)
        sims.append(sim)
        inputs.append((f0, u0))
    with capi.Batch(sims) as b:
        info = b.info
        assert info["members"] == len(MIX) and info["items"] >= len(MIX)
        b.step(30)
        b.synchronize()
    for k, (case, sim) in enumerate(zip(MIX, sims)):
        dims, N, nf, q, expansion, dt = case
        p = orc.Params(dims=dims, N=N, L=20.0, dt=dt, nf=nf, q=q, expansion=expansion)
        ref = orc.step(orc.init(p, *inputs[k]), 30)
        f, v, sc = sim.get_fields(capi.CE_VEL_STAGGERED)
        assert sc.step == 30 and sc.t == pytest.approx(30 * dt)
        assert relmax(f, ref.f) <= 1e-11, case
        assert relmax(v, ref.v) <= 1e-11, case
        if expansion:
            assert abs(sc.a - ref.scale.a) <= 1e-11 * ref.scale.a
        en, en_ref = sim.energy(), orc.energy(ref)
        assert en["E"] == pytest.approx(en_ref["E"], rel=1e-10)
        sim.close()


def test_batch_of_1d_lattices_only_matches_oracle_fp64(gpu_capi, orc):
    """A batch without 2D/3D members runs the 1D launch alone."""
    capi = gpu_capi
    cases = [c for c in MIX if c[0] == 1]
    sims, inputs = [], []
    for k, case in enumerate(cases):
        sim, f0, u0 = make_sim(capi, case, "f64", 300 + k)
        sims.append(sim)
        inputs.append((f0, u0))
    with capi.Batch(sims) as b:
        b.step(40)
        b.synchronize()
    for k, (case, sim) in enumerate(zip(cases, sims)):
        dims, N, nf, q, expansion, dt = case
        p = orc.Params(dims=dims, N=N, L=20.0, dt=dt, nf=nf, q=q, expansion=expansion)
        ref = orc.step(orc.init(p, *inputs[k]), 40)
        f, v, sc = sim.get_fields(capi.CE_VEL_STAGGERED)
        assert relmax(f, ref.f) <= 1e-11 and relmax(v, ref.v) <= 1e-11, case
        if expansion:
            assert abs(sc.a - ref.scale.a) <= 1e-11 * ref.scale.a
        sim.close()


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_batch_alone_and_in_mix_bit_identical(gpu_capi, precision):
    capi = gpu_capi
    mix = [make_sim(capi, case, precision, 200 + k)[0] for k, case in enumerate(MIX)]
    with capi.Batch(mix) as b:
        b.step(45)   # one graph of 32 + 13 single launches
    for k, case in enumerate(MIX):
        alone, _, _ = make_sim(capi, case, precision, 200 + k)
        with capi.Batch([alone]) as b1:
            b1.step(45)
        fa, va, sa = alone.get_fields(capi.CE_VEL_STAGGERED)
        fm, vm, sm = mix[k].get_fields(capi.CE_VEL_STAGGERED)
        assert np.array_equal(fa, fm) and np.array_equal(va, vm), case
        assert (sa.a, sa.ap_half, sa.step) == (sm.a, sm.ap_half, sm.step)
        alone.close()
    for s in mix:
        s.close()


def test_batch_matches_single_lattice_path_fp32(gpu_capi):
    """Batch vs ce_step (z-sweep kernel) on the same 3D lattice: agreement to FP32 rounding."""
    capi = gpu_capi
    N, nf, q = 128, 2, (1.2,)
    f0, u0 = lattice_ics(3, N, 20.0, nf, q=q, seed=7)
    cfg = dict(dims=3, N=N, L=20.0, dt=0.02, nfields=nf, q=q, expansion=True, precision="f32")
    with capi.Simulation(**cfg) as a, capi.Simulation(**cfg) as m:
        a.set_fields(f0, u0)
        m.set_fields(f0, u0)
        a.step(20)
        with capi.Batch([m]) as b:
            b.step(20)
        fa, va, sa = a.get_fields(capi.CE_VEL_STAGGERED)
        fm, vm, sm = m.get_fields(capi.CE_VEL_STAGGERED)
    assert relmax(fm, fa) <= 1e-6 and relmax(vm, va) <= 1e-4
    assert abs(sm.a - sa.a) <= 1e-7 * sa.a


def test_batch_membership_rules(gpu_capi):
    capi = gpu_capi
    s1, _, _ = make_sim(capi, MIX[0], "f32", 1)
    s2, _, _ = make_sim(capi, MIX[3], "f64", 2)
    with pytest.raises(capi.CeError) as ei:
        capi.Batch([s1, s2])                      # mixed precision
    assert ei.value.code == capi.CE_EINVAL
    odd = capi.Simulation(dims=3, N=37, L=20.0, dt=0.05, precision="f32")
    odd.set_fields(*lattice_ics(3, 37, 20.0, 2, q=(1.2,)))
    with pytest.raises(capi.CeError):
        capi.Batch([odd])                         # N not a multiple of 4
    with capi.Batch([s1]) as b:
        with pytest.raises(capi.CeError) as ei:
            s1.step(1)                            # members are stepped by the batch
        assert ei.value.code == capi.CE_ESTATE
        with pytest.raises(capi.CeError) as ei:
            capi.Batch([s1])                      # already in a batch
        assert ei.value.code == capi.CE_ESTATE
        b.step(3)
        assert s1.energy()["step"] == 3           # read-outs wait for the batch
    s1.step(2)                                    # usable alone again after the batch is freed
    assert s1.energy()["step"] == 5
    s3, _, _ = make_sim(capi, MIX[1], "f32", 3)
    b2 = capi.Batch([s3, s1])
    s3.close()                                    # freeing a member invalidates the batch
    with pytest.raises(capi.CeError) as ei:
        b2.step(1)
    assert ei.value.code == capi.CE_ESTATE
    b2.close()
    for s in (s1, s2, odd):
        s.close()


def test_member_error_is_reported_per_member_and_isolated(gpu_capi):
    """A member stepped far beyond the leapfrog stability bound grows until its
    FP32 sums overflow and latches CE_ENONFINITE; ce_batch_status names it, and
    the healthy member of the same batch is bit-identical to running alone."""
    capi = gpu_capi
    healthy_case = MIX[3]
    f0, u0 = lattice_ics(1, 64, 20.0, 2, q=(1.2,), seed=5, amp=1e-2)
    bad = capi.Simulation(dims=1, N=64, L=20.0, dt=1.0, nfields=2, q=(1.2,), expansion=True, precision="f32",
                          kernel="generic", flags=capi.CE_FLAG_ALLOW_UNSTABLE_DT)
    bad.set_fields(f0, u0)
    good, _, _ = make_sim(capi, healthy_case, "f32", 31)
    with capi.Batch([good, bad]) as b:
        b.step(64)
        with pytest.raises(capi.CeError) as ei:
            b.synchronize()
        assert ei.value.code == capi.CE_ENONFINITE
        assert b.member_status() == [capi.CE_OK, capi.CE_ENONFINITE]
    alone, _, _ = make_sim(capi, healthy_case, "f32", 31)
    with capi.Batch([alone]) as b1:
        b1.step(64)
        assert b1.member_status() == [capi.CE_OK]
    fa, va, sa = alone.get_fields(capi.CE_VEL_STAGGERED)
    fg, vg, sg = good.get_fields(capi.CE_VEL_STAGGERED)
    assert np.array_equal(fa, fg) and np.array_equal(va, vg)
    assert (sa.a, sa.step) == (sg.a, sg.step)
    for s in (bad, good, alone):
        s.close()
