"""Pins of the oracle's MRT option (reading R8: moment-space relaxation with
the BGK update as the equal-rates limit)."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import OracleLattice

RNG = np.random.default_rng(2017)


def test_moment_matrix_rows_are_the_named_moments(orc):
    """Rows: 1, e = -4 + 3|e|^2, eps = 4 - 21/2|e|^2 + 9/2|e|^4, j_x, q_x = (-5 + 3|e|^2)e_x,
    j_y, q_y, p_xx = e_x^2 - e_y^2, p_xy = e_x e_y (Lallemand and Luo's D2Q9 basis)."""
    e, _, _ = orc.lattice_vectors()
    ex, ey = e[:, 0].astype(float), e[:, 1].astype(float)
    e2 = ex * ex + ey * ey
    rows = np.array([np.ones(9), -4 + 3 * e2, 4 - 10.5 * e2 + 4.5 * e2 * e2, ex, (-5 + 3 * e2) * ex,
                     ey, (-5 + 3 * e2) * ey, ex * ex - ey * ey, ex * ey])
    M, Mi = orc.mrt_matrices()
    assert np.array_equal(M, rows)
    assert np.allclose(Mi @ M, np.eye(9), atol=1e-15)
    assert np.allclose(M @ M.T, np.diag(np.diag(M @ M.T)))  # orthogonal rows


def test_equal_rates_give_the_bgk_relaxation(orc):
    for _ in range(5):
        f, feq, src = RNG.normal(size=(3, 9))
        tau = RNG.uniform(0.55, 1.5)
        bgk = f - (f - feq) / tau + (1 - 0.5 / tau) * src
        assert np.allclose(orc.mrt_relax(f, feq, src, np.full(9, 1 / tau)), bgk, rtol=1e-13, atol=1e-14)


def test_each_moment_relaxes_at_its_own_rate(orc):
    """M f' = M f - S (M f - M feq) + (I - S/2) M src, moment by moment."""
    M, _ = orc.mrt_matrices()
    f, feq, src = RNG.normal(size=(3, 9))
    s = RNG.uniform(0.3, 1.9, 9)
    out = orc.mrt_relax(f, feq, src, s)
    m, meq, ms = M @ f, M @ feq, M @ src
    assert np.allclose(M @ out, m - s * (m - meq) + (1 - s / 2) * ms, rtol=1e-12, atol=1e-13)


def _lattice(w, mrt=None):
    prm = dict(w.params)
    if mrt is not None:
        prm.update(collision=1.0, mrt_s_f=mrt[0], mrt_s_g=mrt[1])
    L = OracleLattice(w.nx, w.ny, w.edges, w.mask, prm)
    L.set_fields(w.c1, w.c2, w.ux, w.uy, w.p)
    return L


@pytest.mark.parametrize("edges,lid", [((0, 0, 1, 2), 0.0), ((0, 0, 1, 3), 0.02), ((1, 2, 0, 0), 0.0)])
def test_mrt_with_bgk_rates_reproduces_the_bgk_step(edges, lid):
    w = W.random_lattice(40, 28, 31, edges=edges, solids=("disc", "corner"), lid_u=lid)
    w.params.update(tau1=0.85, tau2=0.85, nu1=0.1, nu2=0.1, nu3=0.1)
    taug = 3 * 0.1 + 0.5
    A = _lattice(w)
    B = _lattice(w, mrt=(1 / 0.85, 1 / taug))
    A.step(60)
    B.step(60)
    assert np.abs(A.state() - B.state()).max() < 1e-13


def test_mrt_conserves_each_component():
    w = W.random_lattice(40, 30, 4, edges=(2, 1, 1, 2), solids=("disc", "pillar"))
    L = _lattice(w, mrt=(1.3, 1.3))
    m0 = L.mass()
    L.step(200)
    assert np.all(np.abs(L.mass() - m0) <= 1e-12 * np.abs(m0).max())


def test_mrt_shear_viscosity_set_by_stress_rows_only():
    """A shear wave decays at nu k^2 with nu = cs^2 (tau_g - 1/2) whatever the
    energy-moment rate s_g."""
    nx, ny, U = 4, 48, 1e-4
    x, y = W.grid(nx, ny)
    k = 2 * math.pi / ny
    for s_g in (1.1, 1.7):
        prm = W.params(nu=(0.08, 0.08, 0.08), mrt=(1.2, s_g))
        L = OracleLattice(nx, ny, (0, 0, 0, 0), None, prm)
        z = np.zeros((ny, nx))
        L.set_fields(z + 0.3, z + 0.2, U * np.sin(k * y), z)

        def amp():
            return 2 * np.mean(L.fields()["ux"] * np.sin(k * y))

        L.step(100)
        a1 = amp()
        L.step(1000)
        rate = -math.log(amp() / a1) / 1000
        assert abs(rate / (0.08 * k * k) - 1) < 3e-3


def test_mrt_mobility_set_by_flux_rows_only():
    """The linearised Cahn-Hilliard decay rate (Eq. 16, M_1 from Eq. 18a)
    holds with the other order-parameter moments relaxing at s_f != 1/tau."""
    nx, ny, c0, eps, lam, D, M = 64, 4, 0.1, 1e-3, 0.01, 4.0, 0.1
    for s_f in (1.0, 1.5):
        prm = W.params(sigma=(lam, lam, lam), mobility=M, D=D, tau=(0.9, 0.9), mrt=(s_f, 1.2))
        x, y = W.grid(nx, ny)
        k = 2 * math.pi / nx
        L = OracleLattice(nx, ny, (0, 0, 0, 0), None, prm)
        z = np.zeros((ny, nx))
        L.set_fields(c0 + eps * np.sin(k * x), z, z, z)

        def amp():
            c = L.fields()["c1"]
            return 2 * np.mean((c - c.mean()) * np.sin(k * x))

        L.step(4000)
        a1 = amp()
        L.step(8000)
        rate = -math.log(amp() / a1) / 8000
        phi_p = 1 - 6 * c0 + 6 * c0 ** 2
        theory = M * k * k * (12 / D * lam * phi_p + 0.75 * D * lam * 2 * (1 - math.cos(k)))
        assert abs(rate / theory - 1) < 0.01


def test_mrt_laplace_pressure_jump():
    n, R, sig = 64, 14.0, 1e-3
    x, y = W.grid(n, n)
    c1 = W.profile(x, y, n / 2, n / 2, R, 4.0, n, n)
    prm = W.params(sigma=(sig, sig, sig), rho=(3.0, 1.0, 1.0), mrt=(1.2, 1.4))
    L = OracleLattice(n, n, (0, 0, 0, 0), None, prm)
    z = np.zeros((n, n))
    L.set_fields(c1, z, z, z)
    L.step(5000)
    f = L.fields()
    dp = f["p"][n // 2, n // 2] - f["p"][0, 0]
    assert abs(dp * R / sig - 1.0) < 0.05
