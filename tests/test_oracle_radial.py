"""Pins of the radial basis and the polynomial cutoff envelope (closed forms)."""
import math

import numpy as np
from scipy.integrate import quad

from oracle.allegro64 import bessel, envelope, silu, silu_grad


def test_envelope_values_and_smoothness_at_cutoff():
    rc, p = 5.0, 6
    f0, _ = envelope(np.array([1e-12]), rc, p)
    assert abs(f0[0] - 1.0) < 1e-12
    f, df = envelope(np.array([rc - 1e-9, rc, rc + 0.1]), rc, p)
    assert np.all(np.abs(f) < 1e-12) and np.all(np.abs(df) < 1e-12)
    # second derivative vanishes at rc: f ~ c (1 - x)^3 near x = 1
    d1, d2 = 1e-2, 0.5e-2
    fa = envelope(np.array([rc - d1]), rc, p)[0][0]
    fb = envelope(np.array([rc - d2]), rc, p)[0][0]
    assert abs(fa / fb - 8.0) < 0.2


def test_envelope_derivative_fd():
    rc, p = 6.0, 6
    r = np.linspace(0.3, 5.9, 40)
    h = 1e-6
    fd = (envelope(r + h, rc, p)[0] - envelope(r - h, rc, p)[0]) / (2 * h)
    np.testing.assert_allclose(envelope(r, rc, p)[1], fd, atol=1e-8)


def test_bessel_orthonormal():
    rc, nb = 5.0, 8
    for n in range(1, nb + 1):
        for m in range(n, nb + 1):
            val, _ = quad(lambda r: (bessel(np.array([r]), rc, nb)[0][0, n - 1]
                                     * bessel(np.array([r]), rc, nb)[0][0, m - 1] * r * r),
                          0.0, rc, limit=200)
            assert abs(val - (1.0 if n == m else 0.0)) < 1e-9


def test_bessel_derivative_fd_and_closed_form():
    rc, nb = 6.0, 8
    r = np.linspace(0.5, 5.9, 30)
    h = 1e-6
    B, dB = bessel(r, rc, nb)
    fd = (bessel(r + h, rc, nb)[0] - bessel(r - h, rc, nb)[0]) / (2 * h)
    np.testing.assert_allclose(dB, fd, atol=1e-7)
    n = 3
    np.testing.assert_allclose(B[:, n - 1], math.sqrt(2 / rc) * np.sin(n * np.pi * r / rc) / r)


def test_silu_derivative():
    z = np.linspace(-8, 8, 101)
    h = 1e-6
    np.testing.assert_allclose(silu_grad(z), (silu(z + h) - silu(z - h)) / (2 * h), atol=1e-8)
    np.testing.assert_allclose(silu(z), z / (1 + np.exp(-z)))
