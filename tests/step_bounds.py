"""Error bound of one step against the FP64 oracle, shared by the GPU parity
tests (imported by the test modules; holds no test itself)."""
import numpy as np

EPS32 = 2.0 ** -24   # unit roundoff of FP32 storage
EPS64 = 2.0 ** -53   # unit roundoff of FP64


def check_one_step(orc, local, p, before, after, sites, stencil, G, V, eps=EPS32, sums_rel=1e-5):
    """before/after: (f, v, scalars) sampled at stencil / sites.

    Error bound of one step in the storage precision (unit roundoff eps:
    EPS32 for FP32 storage, EPS64 for FP64) against FP64 arithmetic on the
    same stored inputs (the oracle starts from the sampled values, so only the
    step's own roundings count): f' = g = f + dt v is one rounding of
    |f| + dt |v|; v' = v + dt (lap g - dV/df(g) + s g) carries the rounding of
    every g it reads multiplied by the Laplacian's weights (sum 4 d / dx^2), of
    dV/df and of the sum, each a few units of eps.  Eight units per term leave
    room for the FMA/non-FMA differences and the final conversions.  The
    scale factor's a'' is compared to sums_rel of its source term: the GPU's
    global sums are added in another order (FP32 per-thread partials in the
    FP32 kernels: 1e-5; FP64 throughout: rounding)."""
    fb, vb, scb = before
    fa, va, sca = after
    ref = local.step_at(p, sites, stencil, fb, vb, scb.a, scb.ap_half, G, V)
    dxinv2 = (p.N / p.L) ** 2
    s = ref.app / ref.a
    q = list(p.q) + [0.0] * 3
    gm = [float(np.abs(ref.f[i]).max()) for i in range(p.nf)]
    # |dV/df_i| bounds: phi^3 + phi sum q chi^2, and q_i phi^2 chi_i
    dvm = [gm[0] ** 3 + gm[0] * sum(q[j - 1] * gm[j] ** 2 for j in range(1, p.nf))]
    dvm += [q[i - 1] * gm[0] ** 2 * gm[i] for i in range(1, p.nf)]
    for i in range(p.nf):
        vmax = float(np.abs(vb[i]).max())
        tol_f = 4.0 * eps * (float(np.abs(fb[i]).max()) + p.dt * vmax)
        tol_v = 8.0 * eps * (vmax + p.dt * ((4 * p.dims + 2) * dxinv2 * gm[i] + dvm[i] + abs(s) * gm[i]))
        assert np.abs(fa[i] - ref.f[i]).max() <= tol_f, (i, np.abs(fa[i] - ref.f[i]).max(), tol_f)
        assert np.abs(va[i] - ref.v[i]).max() <= tol_v, (i, np.abs(va[i] - ref.v[i]).max(), tol_v)
    assert abs(sca.a - ref.a) <= 1e-12 * ref.a
    Q = p.kappa2 * (2.0 * G + 3.0 * V) / ref.a
    scale = abs(Q) + ref.ap ** 2 / ref.a
    assert abs(sca.app - ref.app) <= sums_rel * scale
    assert abs(sca.ap_half - ref.ap) <= sums_rel * p.dt * scale + 1e-12 * abs(ref.ap)
