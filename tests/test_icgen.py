"""The shared input generator: real, seeded, band-limited, and the torch FFT path
agrees with the numpy one."""
import math

import numpy as np
import pytest

from paper_0712_0813_gb300.icgen import courant_dt, lattice_ics


def test_reproducible_and_seed_dependent():
    a = lattice_ics(3, 12, 20.0, 2, seed=5)
    b = lattice_ics(3, 12, 20.0, 2, seed=5)
    c = lattice_ics(3, 12, 20.0, 2, seed=6)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not np.array_equal(a[0], c[0])


@pytest.mark.parametrize("dims,N", [(1, 64), (2, 32), (3, 16)])
def test_band_limit_zero_mode_and_mean(dims, N):
    f, u = lattice_ics(dims, N, 20.0, 2, phi0=1.3, seed=2)
    for i, base in enumerate((1.3, 0.0)):
        d = (f[i] - base).reshape((N,) * dims)
        spec = np.fft.fftn(d)
        freqs = np.meshgrid(*([np.fft.fftfreq(N, 1.0 / N)] * dims), indexing="ij")
        nabs = np.sqrt(sum(g * g for g in freqs))
        assert np.abs(spec[nabs > N / 4 + 1e-9]).max() < 1e-10 * np.abs(spec).max()  # round-off only
        assert abs(d.mean()) < 1e-15                        # zero mode removed
        assert 1e-6 < d.std() < 1e-3                        # amplitude 1e-4 scale


def test_torch_backend_matches_numpy():
    pytest.importorskip("torch")
    a = lattice_ics(3, 16, 20.0, 2, q=(5.0,), seed=9)
    b = lattice_ics(3, 16, 20.0, 2, q=(5.0,), seed=9, backend="torch")
    np.testing.assert_allclose(b[0], a[0], rtol=0, atol=1e-15)
    np.testing.assert_allclose(b[1], a[1], rtol=0, atol=1e-14)


def test_courant_dt():
    dx = 20.0 / 256
    w = math.sqrt(12 / dx ** 2 + 3.0)
    assert courant_dt(3, 256, 20.0, 1.0, (1.2,)) == pytest.approx(0.9 / w)
    assert courant_dt(1, 8, 20.0, 1.0, (1.2,)) == 0.05
    # masses at amp * phi0: a strongly coupled lattice takes a smaller step
    w4 = math.sqrt(12.0 / (20.0 / 96) ** 2 + 72.9 * (4 * 1.98) ** 2)
    assert courant_dt(3, 96, 20.0, 1.98, (72.9,), amp=4.0) == pytest.approx(0.9 / w4)
    assert courant_dt(3, 96, 20.0, 1.98, (72.9,), amp=4.0) < 0.5 * courant_dt(3, 96, 20.0, 1.98, (72.9,))
