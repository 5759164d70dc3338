"""Moment pins of the oracle's equilibria and source terms (Eqs. 2a, 2b, 4, 11a, 11b).

The equilibria and forcing terms of the model are built to have prescribed
velocity moments (the Chapman-Enskog analysis behind Eqs. 16-18 relies on
them).  Each test sums the oracle's per-direction values over the D2Q9 set and
compares with the moment the construction is designed to produce; a dropped
term, a wrong sign or a transposed component breaks at least one of them.
"""
import numpy as np
import pytest

RNG = np.random.default_rng(9534)
CS2 = 1.0 / 3.0


@pytest.fixture(scope="module")
def lat(orc):
    e, w, opp = orc.lattice_vectors()
    return e.astype(float), w


def _rand_u():
    return RNG.uniform(-0.08, 0.08, 2)


@pytest.mark.parametrize("trial", range(10))
def test_order_parameter_equilibrium_moments(orc, lat, trial):
    e, w = lat
    c, mu, eta = RNG.uniform(0, 1), RNG.normal(0, 1e-3), RNG.uniform(0.3, 3)
    u = _rand_u()
    f = np.array([orc.feq(k, c, mu, eta, *u) for k in range(9)])
    assert np.isclose(f.sum(), c, rtol=1e-14, atol=1e-16)                       # Eq. 13a
    assert np.allclose(e.T @ f, c * u, rtol=1e-13, atol=1e-17)                   # advection flux
    assert np.allclose(np.einsum("k,ka,kb->ab", f, e, e), CS2 * eta * mu * np.eye(2),
                       rtol=1e-12, atol=1e-18)                                    # M grad mu flux


@pytest.mark.parametrize("trial", range(10))
def test_hydrodynamic_equilibrium_moments(orc, lat, trial):
    e, w = lat
    p, rho = RNG.normal(0, 1e-3), RNG.uniform(0.5, 10)
    u = _rand_u()
    g = np.array([orc.geq(k, p, rho, *u) for k in range(9)])
    s = np.array([orc.sk(k, *u) for k in range(9)])
    assert abs(s.sum()) < 1e-17
    assert np.allclose(e.T @ s, u, atol=1e-16)
    assert np.allclose(np.einsum("k,ka,kb->ab", s, e, e), np.outer(u, u), atol=1e-16)
    assert abs(g.sum()) < 1e-15
    assert np.allclose(e.T @ g, rho * u, rtol=1e-13, atol=1e-16)
    assert np.allclose(np.einsum("k,ka,kb->ab", g, e, e), p * np.eye(2) + rho * np.outer(u, u),
                       rtol=1e-12, atol=1e-16)


@pytest.mark.parametrize("trial", range(10))
def test_order_parameter_source_moments(orc, lat, trial):
    e, w = lat
    tau = RNG.uniform(0.55, 1.5)
    dcu = RNG.normal(0, 1e-3, 2)
    F = np.array([orc.src_f(k, tau, *dcu) for k in range(9)])
    assert abs(F.sum()) < 1e-18
    assert np.allclose(e.T @ F, (1 - 0.5 / tau) * dcu, rtol=1e-13, atol=1e-19)
    assert np.allclose(np.einsum("k,ka,kb->ab", F, e, e), 0, atol=1e-18)


@pytest.mark.parametrize("trial", range(10))
def test_hydrodynamic_forcing_moments(orc, lat, trial):
    """Zeroth moment (1 - 1/2tau) u.grad rho (the pressure correction of Eq. 13c),
    first moment (1 - 1/2tau)(F_s + G) + F_a (the force of Eq. 17b and Eq. 12)."""
    e, w = lat
    taug = RNG.uniform(0.55, 1.5)
    u = _rand_u()
    gr = RNG.normal(0, 0.1, 2)
    Ft = RNG.normal(0, 1e-4, 2)
    Fa = RNG.normal(0, 1e-5, 2)
    G = np.array([orc.src_g(k, taug, *u, *gr, *Ft, *Fa) for k in range(9)])
    a = 1 - 0.5 / taug
    assert np.isclose(G.sum(), a * (u @ gr), rtol=1e-12, atol=1e-17)
    assert np.allclose(e.T @ G, a * Ft + Fa, rtol=1e-11, atol=1e-17)
