"""Pins of the CPU oracle against facts that do not come from the oracle itself.

arXiv:0712.0813 prints no equations and no worked example, so every pin here is
a closed form, an identity of the discrete operators, an independent
integration of the continuum equations, or a library routine:

  * Laplacian (reading c-1): plane-wave eigenvalues; a Kronecker-sum matrix
    built from 1D circulant second differences on N=3 and N=4.
  * Model (V = phi^4/4 + q/2 phi^2 chi^2): hand-evaluated values, and dV/df
    against central differences of V.
  * Leapfrog + start-up (Sec. III): a free massless mode, whose leapfrog
    solution is known exactly (cos(n Omega dt), sin(Omega dt/2) = dt/2 sqrt(lambda)).
  * Rescaled field equation + scale-factor equation (readings c-2..c-4): the
    homogeneous limit against an RK4 of the physical Klein-Gordon + Friedmann
    system in cosmic variables, with second-order convergence.
  * Whole scheme: energy drift O(dt^2) without expansion, Friedmann-constraint
    drift O(dt^2) with expansion (strong gradients, so the G coefficient
    matters), exact time reversibility.
  * Outputs: numpy mean/var; G = -1/2 <f lap f> (summation by parts).
"""
import math

import numpy as np
import pytest

KAPPA2 = 8.0 * math.pi / 3.0 * 0.342 ** 2


def coords(dims, N, L):
    dx = L / N
    axes = [np.arange(N) * dx] * dims
    grids = np.meshgrid(*axes, indexing="ij")  # grids[0] slowest (z), grids[-1] = x
    return grids[::-1]  # x, y, z


# ---------------------------------------------------------------- Laplacian

@pytest.mark.parametrize("dims,N,L,modes", [
    (1, 16, 7.0, [(1,), (3,), (8,)]),
    (2, 12, 5.0, [(1, 2), (6, 5)]),
    (3, 10, 3.0, [(1, 2, 3), (5, 0, 4)]),
])
def test_laplacian_plane_wave_eigenvalue(orc, dims, N, L, modes):
    p = orc.Params(dims=dims, N=N, L=L, dt=0.01, nf=1)
    dx = L / N
    X = coords(dims, N, L)
    for n in modes:
        k = [2 * math.pi * nd / L for nd in n]
        phase = sum(kd * Xd for kd, Xd in zip(k, X))
        f = np.cos(phase + 0.3).reshape(-1)
        lam = sum(4.0 / dx ** 2 * math.sin(kd * dx / 2) ** 2 for kd in k)
        out = orc.laplacian(p, f)
        np.testing.assert_allclose(out, -lam * f, rtol=0, atol=1e-12 * max(lam, 1.0))


def _circulant_second_difference(N):
    D = -2.0 * np.eye(N)
    for i in range(N):
        D[i, (i + 1) % N] += 1.0
        D[i, (i - 1) % N] += 1.0
    return D


@pytest.mark.parametrize("dims", [1, 2, 3])
@pytest.mark.parametrize("N", [3, 4])
def test_laplacian_kronecker_sum(orc, dims, N):
    """lap = sum over axes of I x .. x D x .. x I; x is the fastest (last) factor."""
    L = 2.5
    dx = L / N
    D = _circulant_second_difference(N) / dx ** 2
    I = np.eye(N)
    A = np.zeros((N ** dims, N ** dims))
    for axis in range(dims):  # axis 0 = x = last Kronecker factor
        factors = [I] * dims
        factors[dims - 1 - axis] = D
        M = factors[0]
        for fct in factors[1:]:
            M = np.kron(M, fct)
        A += M
    rng = np.random.default_rng(7)
    f = rng.standard_normal(N ** dims)
    p = orc.Params(dims=dims, N=N, L=L, dt=0.01, nf=1)
    np.testing.assert_allclose(orc.laplacian(p, f), A @ f, rtol=0, atol=1e-12)


# ---------------------------------------------------------------- model

def test_potential_hand_values(orc):
    p = orc.Params(dims=1, N=4, L=1.0, dt=0.01, nf=2, q=(1.2,))
    # V(2, 1) = 16/4 + 0.6 * 4 * 1
    assert orc.potential(p, [2.0, 1.0]) == pytest.approx(6.4, abs=1e-14)
    # dV/dphi = phi^3 + q phi chi^2 = 8 + 2.4;  dV/dchi = q phi^2 chi = 4.8
    np.testing.assert_allclose(orc.dvdf(p, [2.0, 1.0]), [10.4, 4.8], atol=1e-13)
    p4 = orc.Params(dims=1, N=4, L=1.0, dt=0.01, nf=4, q=(0.8, 5.0, 40.0))
    # V(1, .1, .2, .3) = .25 + (.8*.01 + 5*.04 + 40*.09)/2
    assert orc.potential(p4, [1.0, 0.1, 0.2, 0.3]) == pytest.approx(0.25 + 0.5 * 3.808, abs=1e-14)


@pytest.mark.parametrize("nf,q", [(1, ()), (2, (1.2,)), (4, (0.8, 5.0, 40.0))])
def test_dvdf_is_gradient_of_potential(orc, nf, q):
    p = orc.Params(dims=1, N=4, L=1.0, dt=0.01, nf=nf, q=q)
    rng = np.random.default_rng(nf)
    h = 1e-5
    for _ in range(5):
        fs = rng.uniform(-1.5, 1.5, nf)
        fd = np.empty(nf)
        for i in range(nf):
            e = np.zeros(nf)
            e[i] = h
            fd[i] = (orc.potential(p, fs + e) - orc.potential(p, fs - e)) / (2 * h)
        np.testing.assert_allclose(orc.dvdf(p, fs), fd, rtol=1e-8, atol=1e-8)


# ---------------------------------------------------------------- sums

def test_gradient_mean_plane_wave_and_summation_by_parts(orc):
    dims, N, L = 3, 8, 4.0
    p = orc.Params(dims=dims, N=N, L=L, dt=0.01, nf=1)
    dx = L / N
    X = coords(dims, N, L)
    n = (1, 2, 3)
    k = [2 * math.pi * nd / L for nd in n]
    f = np.cos(sum(kd * Xd for kd, Xd in zip(k, X))).reshape(-1)
    # forward difference of cos: -2 sin(k dx/2) sin(...); mean of sin^2 = 1/2
    expect = sum(math.sin(kd * dx / 2) ** 2 for kd in k) / dx ** 2
    G, per = orc.gradient_mean(p, f)
    assert G == pytest.approx(expect, rel=1e-12)
    # summation by parts on the periodic lattice: G = -1/2 <f lap f>
    rng = np.random.default_rng(3)
    p2 = orc.Params(dims=dims, N=N, L=L, dt=0.01, nf=2)
    f2 = rng.standard_normal(2 * N ** dims)
    G2, per2 = orc.gradient_mean(p2, f2)
    sbp = [-0.5 * np.mean(f2[i * N ** 3:(i + 1) * N ** 3] * orc.laplacian(p, f2[i * N ** 3:(i + 1) * N ** 3]))
           for i in range(2)]
    np.testing.assert_allclose(per2, sbp, rtol=1e-12)
    assert G2 == pytest.approx(sum(sbp), rel=1e-12)


def test_potential_mean_and_moments_match_numpy(orc):
    p = orc.Params(dims=2, N=9, L=3.0, dt=0.01, nf=3, q=(0.7, 2.0))
    rng = np.random.default_rng(11)
    f = rng.standard_normal(3 * 81) * 0.3 + np.repeat([1.0, 0.0, -0.2], 81)
    fr = f.reshape(3, 81)
    V = 0.25 * fr[0] ** 4 + 0.5 * 0.7 * fr[0] ** 2 * fr[1] ** 2 + 0.5 * 2.0 * fr[0] ** 2 * fr[2] ** 2
    assert orc.potential_mean(p, f) == pytest.approx(V.mean(), rel=1e-13)
    mean, var = orc.means_variances(p, f)
    np.testing.assert_allclose(mean, fr.mean(axis=1), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(var, fr.var(axis=1), rtol=1e-12)


# ---------------------------------------------------------------- free mode (exact)

@pytest.mark.parametrize("dims,N,L,nf,n_vecs", [
    (1, 16, 6.0, 2, [(2,)]),
    (2, 12, 5.0, 2, [(1, 3)]),
    (3, 8, 4.0, 2, [(1, 2, 3)]),
    (3, 6, 3.0, 4, [(1, 0, 0), (0, 2, 1), (1, 1, 1)]),
])
def test_free_massless_mode_exact(orc, dims, N, L, nf, n_vecs):
    """phi == 0 makes every chi_i a free massless field.  The leapfrog with the
    half-kick start reproduces chi_n = A cos(k.x) cos(n theta), sin(theta/2) =
    (dt/2) sqrt(lambda_k), exactly; v(t+dt/2) and the synchronised velocity and
    energies follow in closed form as well."""
    dt = 0.05
    p = orc.Params(dims=dims, N=N, L=L, dt=dt, nf=nf, q=(1.2, 3.0, 0.5)[:nf - 1])
    dx = L / N
    X = coords(dims, N, L)
    S = N ** dims
    A = [0.3, 0.2, 0.1]
    f0 = np.zeros((nf, S))
    u0 = np.zeros((nf, S))
    thetas, shapes, lams = [], [], []
    for i, n in enumerate(n_vecs):
        k = [2 * math.pi * nd / L for nd in n]
        shape = np.cos(sum(kd * Xd for kd, Xd in zip(k, X))).reshape(-1)
        lam = sum(4.0 / dx ** 2 * math.sin(kd * dx / 2) ** 2 for kd in k)
        theta = 2.0 * math.asin(dt / 2 * math.sqrt(lam))
        f0[i + 1] = A[i] * shape
        thetas.append(theta)
        shapes.append(shape)
        lams.append(lam)
    st = orc.init(p, f0, u0)
    n_total = 0
    for chunk in (1, 9, 90, 900):
        orc.step(st, chunk)
        n_total += chunk
        f = st.f.reshape(nf, S)
        v = st.v.reshape(nf, S)
        assert np.all(f[0] == 0.0) and np.all(v[0] == 0.0)
        for i, (theta, shape, lam) in enumerate(zip(thetas, shapes, lams)):
            fe = A[i] * shape * math.cos(n_total * theta)
            ve = -(2 * A[i] / dt) * math.sin(theta / 2) * math.sin((n_total + 0.5) * theta) * shape
            np.testing.assert_allclose(f[i + 1], fe, rtol=0, atol=2e-13)
            np.testing.assert_allclose(v[i + 1], ve, rtol=0, atol=2e-12)
        us = orc.sync_u(st).reshape(nf, S)
        en = orc.energy(st)
        for i, (theta, shape, lam) in enumerate(zip(thetas, shapes, lams)):
            vs = -(A[i] / dt) * math.sin(theta) * math.sin(n_total * theta) * shape
            np.testing.assert_allclose(us[i + 1], vs, rtol=0, atol=2e-12)
            amp_v = (A[i] / dt) * math.sin(theta) * math.sin(n_total * theta)
            nonzero_modes = sum(1 for nd in n_vecs[i] if nd % N != 0)
            cos2 = 0.5 if nonzero_modes else 1.0
            assert en["K"][i + 1] == pytest.approx(0.5 * amp_v ** 2 * cos2, abs=1e-13)
            amp_f = A[i] * math.cos(n_total * theta)
            assert en["G"][i + 1] == pytest.approx(0.5 * amp_f ** 2 * lam * cos2, abs=1e-12)
        assert en["V"] == 0.0
    assert st.scale.step == 1000 and st.scale.t == pytest.approx(1000 * dt)


# ---------------------------------------------------------------- homogeneous limit vs cosmic-time RK4

def _rk4_cosmic(phi, chi, psi_phi, psi_chi, q, kappa2, tau_end, h, record_every):
    """Physical variables (lambda = 1, phi0 = 1, so program time tau has dt_cosmic
    = a dtau and kappa2 = 8 pi / (3 M_pl^2)):
        phi_tt + 3 H phi_t + dV/dphi = 0,  H^2 = kappa2 (1/2 phi_t^2 + ... + V),
        V = phi^4/4 + q/2 phi^2 chi^2.
    Returns the program-variable predictions f = a phi, a at each record."""
    def rhs(y):
        ph, ch, pp, pc, a = y
        rho = 0.5 * pp * pp + 0.5 * pc * pc + 0.25 * ph ** 4 + 0.5 * q * ph * ph * ch * ch
        H = math.sqrt(kappa2 * rho)
        return np.array([a * pp, a * pc,
                         a * (-3 * H * pp - (ph ** 3 + q * ph * ch * ch)),
                         a * (-3 * H * pc - q * ph * ph * ch),
                         a * a * H])
    y = np.array([phi, chi, psi_phi, psi_chi, 1.0])
    nsub = int(round(tau_end / h))
    out = []
    for s in range(nsub + 1):
        if s % record_every == 0:
            out.append((y[4] * y[0], y[4] * y[1], y[4]))
        if s == nsub:
            break
        k1 = rhs(y)
        k2 = rhs(y + 0.5 * h * k1)
        k3 = rhs(y + 0.5 * h * k2)
        k4 = rhs(y + h * k3)
        y = y + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    return np.array(out)


def test_homogeneous_limit_matches_cosmic_rk4_second_order(orc):
    q = 1.2
    phi_init, chi_init, u_phi, u_chi = 1.0, 0.3, 0.1, -0.2
    tau_end = 8.0
    errs = []
    for dt in (0.04, 0.02, 0.01):
        p = orc.Params(dims=3, N=3, L=3.0, dt=dt, nf=2, q=(q,), expansion=True, kappa2=KAPPA2)
        S = 27
        f0 = np.concatenate([np.full(S, phi_init), np.full(S, chi_init)])
        u0 = np.concatenate([np.full(S, u_phi), np.full(S, u_chi)])
        st = orc.init(p, f0, u0)
        per = int(round(0.4 / dt))
        nrec = int(round(tau_end / dt)) // per
        sub = 8
        ref = _rk4_cosmic(phi_init, chi_init, u_phi, u_chi, q, KAPPA2, tau_end, dt / sub, per * sub)
        e = 0.0
        for r in range(1, nrec + 1):
            orc.step(st, per)
            fo = st.f.reshape(2, S)
            assert np.ptp(fo[0]) == 0.0 and np.ptp(fo[1]) == 0.0  # stays homogeneous
            e = max(e, abs(fo[0, 0] - ref[r, 0]), abs(fo[1, 0] - ref[r, 1]), abs(st.scale.a - ref[r, 2]))
        errs.append(e)
    assert errs[-1] < 2e-4
    for coarse, fine in zip(errs, errs[1:]):
        assert 3.2 < coarse / fine < 4.8, errs


# ---------------------------------------------------------------- conservation laws

def _strong_ic(dims, N, L, nf=2):
    X = coords(dims, N, L)
    S = N ** dims
    f = np.zeros((nf, S))
    f[0] = (1.0 + 0.3 * np.cos(2 * math.pi * X[0] / L) + 0.1 * np.sin(4 * math.pi * X[-1] / L)).reshape(-1)
    f[1] = (0.4 * np.cos(2 * math.pi * X[min(1, dims - 1)] / L + 0.5)).reshape(-1)
    u = np.zeros((nf, S))
    u[1] = (0.2 * np.sin(2 * math.pi * X[0] / L)).reshape(-1)
    return f, u


def test_energy_drift_second_order_without_expansion(orc):
    drifts = []
    for dt in (0.04, 0.02):
        p = orc.Params(dims=3, N=8, L=6.0, dt=dt, nf=2, q=(1.2,), expansion=False)
        f0, u0 = _strong_ic(3, 8, 6.0)
        st = orc.init(p, f0, u0)
        E0 = orc.energy(st)["E"]
        d = 0.0
        for _ in range(40):
            orc.step(st, int(round(0.2 / dt)))
            d = max(d, abs(orc.energy(st)["E"] - E0) / E0)
        drifts.append(d)
    assert drifts[0] < 5e-3
    assert 3.2 < drifts[0] / drifts[1] < 4.8, drifts


def test_friedmann_constraint_second_order_with_expansion(orc):
    res = []
    for dt in (0.04, 0.02):
        p = orc.Params(dims=3, N=8, L=6.0, dt=dt, nf=2, q=(1.2,), expansion=True, kappa2=KAPPA2)
        f0, u0 = _strong_ic(3, 8, 6.0)
        st = orc.init(p, f0, u0)
        en0 = orc.energy(st)
        assert en0["friedmann_resid"] < 0.01  # O(dt^2) only through the half-step a'
        # gradient energy is a sizeable part of rho here, so its coefficient in a'' matters
        assert sum(en0["G"]) > 0.1 * en0["E"]
        r = 0.0
        for _ in range(30):
            orc.step(st, int(round(0.2 / dt)))
            r = max(r, orc.energy(st)["friedmann_resid"])
        res.append(r)
    assert res[0] < 2e-3
    assert 3.2 < res[0] / res[1] < 4.8, res


def test_time_reversibility(orc):
    dt = 0.03
    p = orc.Params(dims=3, N=8, L=6.0, dt=dt, nf=2, q=(1.2,), expansion=True, kappa2=KAPPA2)
    f0, u0 = _strong_ic(3, 8, 6.0)
    start = orc.init(p, f0, u0)
    st = start.copy()
    orc.step(st, 150)
    # kick back one step, then reverse velocities and a'
    s = st.scale.app / st.scale.a
    v_prev = st.v - dt * orc.force(p, st.f, s)
    ap_prev = st.scale.ap - dt * st.scale.app
    st.v = -v_prev
    st.scale.ap = -ap_prev
    orc.step(st, 150)
    s0 = start.scale.app / start.scale.a
    v_before = start.v - dt * orc.force(p, start.f, s0)
    np.testing.assert_allclose(st.f, start.f, rtol=0, atol=1e-11)
    np.testing.assert_allclose(st.v, -v_before, rtol=0, atol=1e-10)
    assert st.scale.a == pytest.approx(1.0, abs=1e-12)
    assert st.scale.ap == pytest.approx(-(start.scale.ap - dt * start.scale.app), abs=1e-11)


# ---------------------------------------------------------------- power spectrum

@pytest.mark.parametrize("dims,N", [(1, 32), (2, 16), (3, 8)])
def test_spectrum_parseval_and_counts(orc, dims, N):
    rng = np.random.default_rng(dims)
    p = orc.Params(dims=dims, N=N, L=5.0, dt=0.01, nf=1)
    f = rng.standard_normal(N ** dims)
    nb = int(np.ceil(np.sqrt(dims) * N / 2)) + 2
    k, power, count = orc.spectrum(p, f, nb)
    assert count.sum() == N ** dims                       # every mode binned once
    assert (power * count).sum() == pytest.approx(N ** dims * (f * f).sum(), rel=1e-12)   # Parseval
    assert k[1] == pytest.approx(2 * np.pi / 5.0)


def test_spectrum_plane_wave_and_constant(orc):
    dims, N, L, A = 3, 16, 4.0, 0.7
    p = orc.Params(dims=dims, N=N, L=L, dt=0.01, nf=1)
    X = coords(dims, N, L)
    n0 = (3, 0, 4)                                         # |n0| = 5
    f = (A * np.cos(sum(2 * np.pi * nd / L * Xd for nd, Xd in zip(n0, X)))).reshape(-1)
    k, power, count = orc.spectrum(p, f, 12)
    S = N ** dims
    # fhat = A S / 2 at +n0 and -n0, zero elsewhere
    assert power[5] * count[5] == pytest.approx(2 * (A * S / 2) ** 2, rel=1e-12)
    assert np.delete(power * count, 5).max() < 1e-18 * power[5] * count[5]
    k, power, count = orc.spectrum(p, np.full(S, 1.5), 12)
    assert power[0] == pytest.approx((1.5 * S) ** 2) and count[0] == 1


LOCAL_CASES = [
    # dims, N, nf, q, expansion, dt
    (3, 6, 2, (1.2,), True, 0.05),
    (3, 5, 4, (0.8, 5.0, 40.0), True, 0.03),
    (2, 9, 3, (0.8, 5.0), False, 0.05),
    (1, 11, 1, (), True, 0.02),
    (3, 3, 2, (1.2,), True, 0.05),          # every neighbour wraps
]


@pytest.mark.parametrize("dims,N,nf,q,expansion,dt", LOCAL_CASES)
def test_local_step_equals_orc_step(orc, dims, N, nf, q, expansion, dt):
    """The per-site restatement of one step (oracle/local.py), evaluated at
    every site from the whole state and fed the G, V of the drifted fields,
    reproduces orc_step exactly; evaluated at a subset of sites from the state
    at those sites' stencil only, it gives the same numbers there."""
    from oracle import local
    from paper_0712_0813_gb300.icgen import lattice_ics
    L = 20.0 if N > 5 else 3.0
    p = orc.Params(dims=dims, N=N, L=L, dt=dt, nf=nf, q=q if q else (0.0,), expansion=expansion)
    f0, u0 = lattice_ics(dims, N, L, nf, q=q if q else (1.2,), seed=21, amp=3e-2)
    st = orc.init(p, f0, u0)
    S = p.S
    fb, vb = st.f.copy().reshape(nf, S), st.v.copy().reshape(nf, S)
    a, ap = st.scale.a, st.scale.ap
    drifted = (fb + p.dt * vb).reshape(-1)
    G = orc.gradient_mean(p, drifted)[0]
    V = orc.potential_mean(p, drifted)
    orc.step(st, 1)
    everywhere = np.arange(S)
    res = local.step_at(p, everywhere, everywhere, fb, vb, a, ap, G, V)
    assert np.array_equal(res.f, st.f.reshape(nf, S))
    assert np.array_equal(res.v, st.v.reshape(nf, S))
    assert (res.a, res.ap, res.app) == (st.scale.a, st.scale.ap, st.scale.app)
    rng = np.random.default_rng(5)
    some = np.sort(rng.choice(S, size=max(1, S // 3), replace=False))
    sten = local.stencil_sites(dims, N, some)
    part = local.step_at(p, some, sten, fb[:, sten], vb[:, sten], a, ap, G, V)
    assert np.array_equal(part.f, res.f[:, some]) and np.array_equal(part.v, res.v[:, some])
    with pytest.raises(ValueError):
        local.step_at(p, some, some, fb[:, some], vb[:, some], a, ap, G, V)   # neighbours missing


# ------------------------------------------- slab-streamed sums of the drift

SUM_CASES = [(1, 64, 2, 7), (2, 3, 1, 2), (2, 20, 4, 6), (3, 3, 2, 1), (3, 17, 3, 5), (3, 32, 2, 16)]


def _slab_reader(f, v, nf, dims, N):
    sh = (nf,) + (N,) * dims
    F, V = f.reshape(sh), v.reshape(sh)
    return lambda k0, k1: (F[:, k0:k1], V[:, k0:k1])


@pytest.mark.parametrize("dims,N,nf,slab", SUM_CASES)
def test_drifted_sums_equal_whole_lattice_sums(orc, dims, N, nf, slab):
    """local.drifted_sums, read slab by slab (slab sizes that leave a ragged
    last slab, N = 3 where every neighbour wraps), gives the G and V that
    orc_gradient_mean / orc_potential_mean give for the whole drifted array
    f + dt v, to rounding (the two add in different orders)."""
    from oracle import local
    from paper_0712_0813_gb300.icgen import lattice_ics
    q = (1.2, 5.0, 40.0)[:max(nf - 1, 1)]
    p = orc.Params(dims=dims, N=N, L=20.0, dt=0.03, nf=nf, q=q, expansion=True)
    f, _ = lattice_ics(dims, N, 20.0, nf, q=q, seed=3, amp=1e-2)
    v = np.random.default_rng(1).normal(size=f.shape)
    G, V, Gp = local.drifted_sums(p, _slab_reader(f, v, nf, dims, N), slab=slab)
    g = (f + p.dt * v).reshape(-1)
    G0, Gp0 = orc.gradient_mean(p, g)
    V0 = orc.potential_mean(p, g)
    assert abs(G - G0) <= 1e-13 * G0
    assert abs(V - V0) <= 1e-13 * V0
    np.testing.assert_allclose(Gp, Gp0, rtol=1e-13, atol=0)


@pytest.mark.parametrize("dims,N,n", [(1, 24, (5,)), (2, 16, (3, 2)), (3, 12, (1, 4, 2))])
def test_drifted_sums_plane_wave_closed_form(orc, dims, N, n):
    """A plane wave A cos(k.x + theta) as the drifted field (v = 0) has mean
    forward-difference gradient energy A^2 sum_d sin^2(k_d dx/2) / dx^2, and a
    constant phi = c has V = c^4 / 4 (chi = 0)."""
    from oracle import local
    L, A = 7.0, 0.3
    dx = L / N
    p = orc.Params(dims=dims, N=N, L=L, dt=0.01, nf=2, q=(1.2,))
    X = coords(dims, N, L)
    k = [2 * math.pi * nd / L for nd in n]
    chi = A * np.cos(sum(kd * Xd for kd, Xd in zip(k, X)) + 0.4).reshape(-1)
    c = 0.7
    f = np.stack([np.full(N ** dims, c), chi])
    G, V, Gp = local.drifted_sums(p, _slab_reader(f, np.zeros_like(f), 2, dims, N), slab=5)
    expect = A * A * sum(math.sin(kd * dx / 2) ** 2 for kd in k) / dx ** 2
    assert abs(Gp[0]) == 0.0
    assert abs(Gp[1] - expect) <= 1e-13 * expect
    # V = c^4/4 + (q/2) c^2 <chi^2>, <chi^2> = A^2/2
    assert abs(V - (c ** 4 / 4 + 0.6 * c * c * A * A / 2)) <= 1e-14


# ------------------------------------------ OpenMP timing copy of the oracle

def test_omp_copy_matches_serial_oracle(orc):
    """The OpenMP copy of the oracle's loops (timed as the CPU baseline on all
    host cores) reproduces the serial oracle on the expanding 32^3 lattice to
    rounding: only the order of the global sums differs."""
    from paper_0712_0813_gb300.icgen import lattice_ics
    p = orc.Params(dims=3, N=32, L=20.0, dt=0.05, nf=2, q=(1.2,), expansion=True)
    f0, u0 = lattice_ics(3, 32, 20.0, 2, q=(1.2,), seed=1, amp=1e-2)
    orc.omp_threads(4)
    assert orc.omp_threads() == 4
    ser = orc.step(orc.init(p, f0, u0), 20)
    par = orc.omp_step(orc.omp_init(p, f0, u0), 20)
    assert np.abs(par.f - ser.f).max() <= 1e-13 * np.abs(ser.f).max()
    assert np.abs(par.v - ser.v).max() <= 1e-12 * np.abs(ser.v).max()
    assert abs(par.scale.a - ser.scale.a) <= 1e-14 * ser.scale.a
    assert abs(par.scale.ap - ser.scale.ap) <= 1e-13 * abs(ser.scale.ap)
    assert par.scale.step == ser.scale.step == 20
