"""Pins of the discrete operators of Eqs. 20a and 20b.

Second-order central schemes are exact on polynomials of degree two: the
gradient of a quadratic at the stencil centre and the Laplacian of a quadratic
are reproduced exactly, which fixes every weight and sign of the stencils.
"""
import numpy as np
import pytest

RNG = np.random.default_rng(1710)


def _stencil_values(orc, fn):
    e, _, _ = orc.lattice_vectors()
    return np.array([fn(ex, ey) for ex, ey in e])


@pytest.mark.parametrize("trial", range(10))
def test_gradient_exact_on_quadratics(orc, trial):
    a, b, c, d, ee, f = RNG.normal(size=6)
    x0, y0 = RNG.normal(size=2)
    q = lambda x, y: a + b * x + c * y + d * x * x + ee * y * y + f * x * y
    v = _stencil_values(orc, lambda ex, ey: q(x0 + ex, y0 + ey))
    g = orc.grad9(v)
    exact = np.array([b + 2 * d * x0 + f * y0, c + 2 * ee * y0 + f * x0])
    assert np.allclose(g, exact, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("trial", range(10))
def test_laplacian_exact_on_quadratics(orc, trial):
    a, b, c, d, ee, f = RNG.normal(size=6)
    x0, y0 = RNG.normal(size=2)
    q = lambda x, y: a + b * x + c * y + d * x * x + ee * y * y + f * x * y
    v = _stencil_values(orc, lambda ex, ey: q(x0 + ex, y0 + ey))
    assert np.isclose(orc.lap9(v), 2 * d + 2 * ee, rtol=1e-12, atol=1e-12)


def test_laplacian_fourier_symbol(orc):
    """Isotropic 9-point Laplacian: symbol -2(1 - cos k) for a 1D mode sin(k x)
    and second-order isotropy for oblique modes."""
    for k in (0.1, 0.5, 1.0):
        v = _stencil_values(orc, lambda ex, ey: np.sin(k * ex + 0.3))
        assert np.isclose(orc.lap9(v), -2 * (1 - np.cos(k)) * np.sin(0.3), rtol=1e-12)
    k = 0.05
    for ang in (0.0, 0.4, 0.785):
        kx, ky = k * np.cos(ang), k * np.sin(ang)
        v = _stencil_values(orc, lambda ex, ey: np.cos(kx * ex + ky * ey))
        assert np.isclose(orc.lap9(v), -k * k, rtol=k * k / 6)  # O(k^2) truncation
