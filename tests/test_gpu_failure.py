"""Failure detection on the GPU without a GPU fault.

With CE_FLAG_TEST_TMA_STALL every plane the z-sweep kernel loads announces 16
bytes that never arrive, so the kernel's bounded mbarrier waits run out: each
launch latches CE_ETIMEOUT in the handle's status word and completes.  The
host reads the code at the next synchronising call and the CUDA context stays
usable (a second handle on the same device runs normally)."""
import numpy as np
import pytest

from paper_0712_0813_gb300.icgen import lattice_ics

pytestmark = pytest.mark.gpu


def test_bounded_wait_expiry_is_reported_and_context_survives(gpu_capi):
    capi = gpu_capi
    N = 128
    f0, u0 = lattice_ics(3, N, 20.0, 2, q=(1.2,), seed=2)
    cfg = dict(dims=3, N=N, L=20.0, dt=0.02, nfields=2, q=(1.2,), expansion=True, precision="f32",
               kernel="sweep")
    with capi.Simulation(**cfg, flags=capi.CE_FLAG_TEST_TMA_STALL) as bad:
        with pytest.raises(capi.CeError) as ei:
            bad.set_fields(f0, u0)          # the start-up half kick is a z-sweep launch: it
        assert ei.value.code == capi.CE_ETIMEOUT   # completes and reports the expired wait
        with pytest.raises(capi.CeError) as ei:
            bad.step(1)                     # a failed start-up leaves no state to step
        assert ei.value.code == capi.CE_ESTATE
        with pytest.raises(capi.CeError) as ei:
            bad.synchronize()               # the code stays latched
        assert ei.value.code == capi.CE_ETIMEOUT
    with capi.Simulation(**cfg) as good:   # the context is intact
        good.set_fields(f0, u0)
        good.step(5)
        good.synchronize()
        assert good.energy()["step"] == 5


def test_replan_keeps_the_state_fp64(gpu_capi):
    capi = gpu_capi
    N = 64
    f0, u0 = lattice_ics(3, N, 20.0, 2, q=(1.2,), seed=8, amp=1e-2)
    cfg = dict(dims=3, N=N, L=20.0, dt=0.02, nfields=2, q=(1.2,), expansion=True, kernel="sweep")
    with capi.Simulation(**cfg) as a, capi.Simulation(**cfg) as b:
        a.set_fields(f0, u0)
        b.set_fields(f0, u0)
        a.step(40)
        b.step(13)
        b.replan(16, 3, 3)
        assert b.sweep_plan == (16, 3, 3)
        b.step(27)
        fa, va, sa = a.get_fields(capi.CE_VEL_STAGGERED)
        fb, vb, sb = b.get_fields(capi.CE_VEL_STAGGERED)
    assert np.abs(fa - fb).max() <= 1e-12 * np.abs(fa).max()
    assert np.abs(va - vb).max() <= 1e-12 * np.abs(va).max()
    assert sa.step == sb.step == 40
