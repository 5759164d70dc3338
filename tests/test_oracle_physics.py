"""Closed-form physics pins of the oracle (Sec. II and Sec. III of the paper).

Each test runs the full oracle time step on a small lattice and compares
with a result fixed independently of the code: the tanh interface that makes
Eq. 8 vanish, Laplace's law, the linear Couette profile between a bounce-back
wall and the velocity lid of Eqs. 51-53, the linearised Cahn-Hilliard decay
rate of Eq. 16 with the mobility of Eq. 18a, Young/de Gennes equilibrium
shapes (Eq. 47 and theta_n of Sec. III.A), the two-phase reduction, and the
exact uniform-translation solution of Eq. 17b with density contrast (which
depends on the interfacial force F_a of Eq. 12).
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import OracleLattice


def _run(nx, ny, edges, prm, c1, c2, ux=None, uy=None, steps=0, mask=None):
    z = np.zeros((ny, nx))
    L = OracleLattice(nx, ny, edges, mask, prm)
    L.set_fields(c1, c2, z if ux is None else ux, z if uy is None else uy)
    if steps:
        L.step(steps)
    return L


def test_tanh_profile_is_the_equilibrium_of_eq8():
    """c = 1/2 + 1/2 tanh(2x/D) makes the bulk and gradient terms of Eq. 8
    cancel; on the lattice the residual is O(1/D^2) (second-order stencil)."""
    errs = []
    for D in (4.0, 8.0, 16.0):
        nx, ny = int(16 * D), 4
        x, y = W.grid(nx, ny)
        c1 = 0.5 + 0.5 * np.tanh(2 * (x - nx / 4) / D) - 0.5 - 0.5 * np.tanh(2 * (x - 3 * nx / 4) / D) + 0.0
        lam = 1e-3
        prm = W.params(sigma=(lam, lam, lam), D=D)
        L = _run(nx, ny, (0, 0, 0, 0), prm, c1, np.zeros((ny, nx)))
        mu = L.fields()["mu1"]
        scale = 12.0 / D * lam * 0.1  # magnitude of each term of Eq. 8 in the interface
        errs.append(np.abs(mu).max() / scale)
    assert errs[0] < 0.1
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5


@pytest.mark.parametrize("rho1,tol", [(1.0, 0.03), (5.0, 0.05)])
def test_laplace_pressure_jump(rho1, tol):
    """p_in - p_out = sigma_13 / R for a 2D drop of fluid 1 in fluid 3."""
    n, R, sig = 64, 14.0, 1e-3
    x, y = W.grid(n, n)
    c1 = W.profile(x, y, n / 2, n / 2, R, 4.0, n, n)
    prm = W.params(sigma=(sig, sig, sig), rho=(rho1, 1.0, 1.0))
    L = _run(n, n, (0, 0, 0, 0), prm, c1, np.zeros((n, n)), steps=5000)
    f = L.fields()
    dp = f["p"][n // 2, n // 2] - f["p"][0, 0]
    assert abs(dp * R / sig - 1.0) < tol
    assert np.abs(f["ux"]).max() < 1e-5  # spurious currents stay small


def test_couette_flow_between_wall_and_velocity_lid():
    """Single phase between a half-way bounce-back wall at y = -1/2 and the
    Eq. 51 lid row at y = ny-1 moving at U0: the steady profile is linear."""
    nx, ny, U0 = 4, 16, 0.01
    prm = W.params(lid_u=U0, nu=(0.1, 0.1, 0.1))
    z = np.zeros((ny, nx))
    ux = z.copy()
    ux[-1] = U0
    L = _run(nx, ny, (0, 0, 2, 3), prm, z, z, ux=ux, steps=20000)
    f = L.fields()
    y = np.arange(ny)
    exact = U0 * (y + 0.5) / (ny - 1 + 0.5)
    assert np.abs(f["ux"] - exact[:, None]).max() < 1e-10 * U0 * 1e4
    assert np.abs(f["uy"]).max() < 1e-14


def test_linearised_cahn_hilliard_decay_rate():
    """A small sinusoid c1 = c0 + eps sin(kx) (c2 = 0) decays at the rate of the
    linearised Eq. 16: M_1 k^2 [(12/D) lambda phi'(c0) + (3/4) D lambda k_d^2],
    phi(c) = c(1-c)(1-2c), k_d^2 = 2(1 - cos k) the symbol of Eq. 20b, and
    M_1 = eta_1 cs^2 (tau_1 - 1/2) (Eq. 18a)."""
    nx, ny, c0, eps, lam, D, M = 64, 4, 0.1, 1e-3, 0.01, 4.0, 0.1
    prm = W.params(sigma=(lam, lam, lam), mobility=M, D=D, tau=(0.9, 0.9))
    x, y = W.grid(nx, ny)
    k = 2 * math.pi / nx
    L = _run(nx, ny, (0, 0, 0, 0), prm, c0 + eps * np.sin(k * x), np.zeros((ny, nx)))
    L.step(4000)

    def amp():
        c = L.fields()["c1"]
        return 2 * np.mean((c - c.mean()) * np.sin(k * x))

    a1 = amp()
    L.step(8000)
    a2 = amp()
    rate = -math.log(a2 / a1) / 8000
    phi_p = 1 - 6 * c0 + 6 * c0 ** 2
    kd2 = 2 * (1 - math.cos(k))
    theory = M * k * k * (12 / D * lam * phi_p + 0.75 * D * lam * kd2)
    assert abs(rate / theory - 1) < 0.01


def _degennes(theta_deg, R):
    """Eq. 47: equilibrium spreading length and height of a 2D cap of area pi R^2 / 2."""
    th = math.radians(theta_deg)
    f = math.sqrt((math.pi / 2) / (th - math.sin(th) * math.cos(th)))
    return 2 * R * f * math.sin(th), R * f * (1 - math.cos(th))


@pytest.mark.parametrize("theta13", [60.0, 120.0])
def test_equilibrium_contact_angle_on_flat_wall(theta13):
    """A drop of fluid 1 in fluid 3 relaxes to theta_13 (Sec. III.A): theta_n =
    2 atan(2 H_d / L_s) within 3.5 deg and L_s, H_d within 7% of Eq. 47."""
    nx, ny, R, sig = 80, 32, 12.0, 1e-2
    th12 = W.theta12_from(sig, sig, sig, theta13, 90.0)
    prm = W.params(sigma=(sig, sig, sig), theta=(th12, theta13, 90.0), mobility=0.2)
    x, y = W.grid(nx, ny)
    c1 = W.profile(x, y, nx / 2, -0.5, R, 4.0, period_x=nx)
    L = _run(nx, ny, (0, 0, 1, 2), prm, c1, np.zeros((ny, nx)), steps=12000)
    c = L.fields()["c1"]
    (Ls, Hd, _), = oracle.drop_geometry(c)
    theta_n = math.degrees(2 * math.atan(2 * Hd / Ls))
    assert abs(theta_n - theta13) < 3.5
    Ls0, Hd0 = _degennes(theta13, R)
    assert abs(Ls / Ls0 - 1) < 0.07 and abs(Hd / Hd0 - 1) < 0.07


def test_two_phase_reduction_of_wetting():
    """c3 = 0: a drop of fluid 1 in fluid 2 takes theta_12, as in the binary
    model (Eqs. 36, 37 and Eq. 26 with cos theta = cos theta_12), and fluid 3
    stays absent up to the weak compressibility of the flow."""
    nx, ny, R, sig = 80, 32, 12.0, 1e-2
    th12 = 60.0
    th13 = 90.0
    th23 = math.degrees(math.acos(math.cos(math.radians(th13)) - math.cos(math.radians(th12))))
    prm = W.params(sigma=(sig, sig, sig), theta=(th12, th13, th23), mobility=0.2)
    x, y = W.grid(nx, ny)
    c1 = W.profile(x, y, nx / 2, -0.5, R, 4.0, period_x=nx)
    L = _run(nx, ny, (0, 0, 1, 2), prm, c1, 1 - c1, steps=12000)
    f = L.fields()
    theta_n = oracle.contact_angle_deg(f["c1"])[0]
    assert abs(theta_n - th12) < 3.5
    # c1 + c2 is only advected, so c3 follows the lattice compressibility
    # div u = -dp/dt / (rho cs^2): bounded by the pressure scale 3 |p|
    assert np.abs(f["c3"]).max() < 3.0 * np.abs(f["p"]).max()


def _translation_error(s):
    """Layer of fluid 1 (rho 10) in fluid 3 (rho 1), interface twice too thick so
    that mass diffuses, uniform flow U along the layer; returns the slope of
    (u_x - U)/U against the relative density change, at resolution s."""
    U = 0.02
    nx, ny, D = 4, 64 * s, 4.0 * s
    prm = W.params(sigma=(1e-3,) * 3, rho=(10.0, 1.0, 1.0), mobility=1.0 * s, D=D, tau=(1.0, 1.0))
    x, y = W.grid(nx, ny)
    c1 = 0.5 + 0.5 * np.tanh(2 * (16 * s - np.abs(y - 32 * s)) / (2 * D))
    z = np.zeros((ny, nx))
    L = _run(nx, ny, (0, 0, 0, 0), prm, c1, z, ux=U + z)
    r0 = L.fields()["rho"][:, 0]
    L.step(400 * s * s)
    f = L.fields()
    du = f["ux"][:, 0] - U
    dr = (f["rho"][:, 0] - r0) / f["rho"][:, 0]
    return np.polyfit(dr, du, 1)[0] / U


def test_uniform_translation_with_density_contrast_converges():
    """u = U is an exact solution of Eq. 17b for a layer whose density changes
    by diffusion; the lattice error must vanish at second order under
    refinement, which needs F_a (Eq. 12) to carry the momentum of the
    diffusing mass (without it the error stalls near 10% of U)."""
    e2, e4 = _translation_error(2), _translation_error(4)
    assert abs(e4) < 0.04
    assert abs(e2 / e4) > 3.0


def test_translation_pin_covers_fluid_two():
    """The same exact solution with the dense layer made of fluid 2, so that
    the second term of F_a (Eq. 12) is exercised."""
    U, s = 0.02, 4
    nx, ny, D = 4, 64 * s, 4.0 * s
    prm = W.params(sigma=(1e-3,) * 3, rho=(1.0, 10.0, 1.0), mobility=1.0 * s, D=D, tau=(1.0, 1.0))
    x, y = W.grid(nx, ny)
    c2 = 0.5 + 0.5 * np.tanh(2 * (16 * s - np.abs(y - 32 * s)) / (2 * D))
    z = np.zeros((ny, nx))
    L = _run(nx, ny, (0, 0, 0, 0), prm, z, c2, ux=U + z)
    r0 = L.fields()["rho"][:, 0]
    L.step(400 * s * s)
    f = L.fields()
    slope = np.polyfit((f["rho"][:, 0] - r0) / f["rho"][:, 0], f["ux"][:, 0] - U, 1)[0] / U
    assert abs(slope) < 0.04


@pytest.mark.parametrize("comp", [1, 2])
def test_cahn_hilliard_decay_per_component(comp):
    """Eq. 18a with a different tau_i per component: each order parameter
    diffuses with its own M_i = eta_i cs^2 (tau_i - 1/2)."""
    nx, ny, c0, eps, lam, D, M = 64, 4, 0.1, 1e-3, 0.01, 4.0, 0.1
    prm = W.params(sigma=(lam, lam, lam), mobility=M, D=D, tau=(0.9, 0.65))
    x, y = W.grid(nx, ny)
    k = 2 * math.pi / nx
    wave = c0 + eps * np.sin(k * x)
    z = np.zeros((ny, nx))
    L = _run(nx, ny, (0, 0, 0, 0), prm, wave if comp == 1 else z, wave if comp == 2 else z)
    name = f"c{comp}"

    def amp():
        c = L.fields()[name]
        return 2 * np.mean((c - c.mean()) * np.sin(k * x))

    L.step(4000)
    a1 = amp()
    L.step(8000)
    rate = -math.log(amp() / a1) / 8000
    phi_p = 1 - 6 * c0 + 6 * c0 ** 2
    theory = M * k * k * (12 / D * lam * phi_p + 0.75 * D * lam * 2 * (1 - math.cos(k)))
    assert abs(rate / theory - 1) < 0.01


def test_shear_wave_viscosity_of_mixture():
    """A shear wave u_x = U sin(k y) in a uniform mixture decays at nu k^2 with
    nu = c1 nu1 + c2 nu2 + c3 nu3 (Eq. 15) and tau_g = nu / cs^2 + 1/2 (Eq. 18b)."""
    nx, ny, U = 4, 48, 1e-4
    c1v, c2v = 0.3, 0.5
    nus = (0.02, 0.15, 0.07)
    prm = W.params(nu=nus, rho=(1.0, 1.0, 1.0))
    x, y = W.grid(nx, ny)
    k = 2 * math.pi / ny
    L = _run(nx, ny, (0, 0, 0, 0), prm, np.full((ny, nx), c1v), np.full((ny, nx), c2v),
             ux=U * np.sin(k * y))

    def amp():
        return 2 * np.mean(L.fields()["ux"] * np.sin(k * y))

    L.step(100)
    a1 = amp()
    L.step(1000)
    rate = -math.log(amp() / a1) / 1000
    nu = c1v * nus[0] + c2v * nus[1] + (1 - c1v - c2v) * nus[2]
    kd2 = 2 * (1 - math.cos(k))
    assert abs(rate / (nu * k * k) - 1) < 3e-3  # O(k^2) lattice error ~ 1e-3


def test_couette_lid_keeps_a_uniform_mixture_uniform():
    """Eq. 51 rebuilds the lid populations of both order parameters from the
    node below: a uniform mixture sheared by the lid stays uniform and the
    steady profile is linear."""
    nx, ny, U0 = 4, 16, 0.01
    prm = W.params(lid_u=U0, nu=(0.1, 0.1, 0.1), rho=(2.0, 3.0, 1.0))
    z = np.zeros((ny, nx))
    ux = z.copy()
    ux[-1] = U0
    L = _run(nx, ny, (0, 0, 2, 3), prm, z + 0.3, z + 0.2, ux=ux, steps=20000)
    f = L.fields()
    # the lid is not mass-conserving: O(c U0^2)-level drift only
    assert np.abs(f["c1"] - 0.3).max() < 5e-5 and np.abs(f["c2"] - 0.2).max() < 5e-5
    y = np.arange(ny)
    exact = U0 * (y + 0.5) / (ny - 1 + 0.5)
    assert np.abs(f["ux"] - exact[:, None]).max() < 1e-5 * U0


def test_body_force_poiseuille_and_hydrostatics():
    """Body force G = rho g (Eqs. 11b, 13b): a plane Poiseuille flow between
    half-way walls is parabolic (exact for tau_g - 1/2 = sqrt(3/16)), and a
    closed box at rest builds the hydrostatic gradient dp/dy = rho g_y."""
    nx, ny, g = 4, 20, 1e-6
    nu = math.sqrt(3.0) / 12.0
    z = np.zeros((ny, nx))
    L = _run(nx, ny, (0, 0, 2, 2), W.params(nu=(nu,) * 3, g=(g, 0.0)), z, z, steps=30000)
    y = np.arange(ny)
    exact = g / (2 * nu) * (y + 0.5) * (ny - 0.5 - y)
    assert np.abs(L.fields()["ux"][:, 0] - exact).max() < 1e-7 * exact.max()
    L = _run(nx, ny, (0, 0, 2, 2), W.params(nu=(0.1,) * 3, g=(0.0, -1e-5), rho=(1, 1, 2.0)), z, z,
             steps=20000)
    f = L.fields()
    assert np.allclose(np.diff(f["p"][:, 0]), 2.0 * -1e-5, rtol=1e-9)
    assert np.abs(f["uy"]).max() < 1e-15


def test_solid_row_in_mask_equals_wall_edge():
    """A wetting wall given as a solid row of the mask (periodic lattice one
    row taller) and the same wall given as lattice edges produce identical
    fields: the ghost rules (Eqs. 42, 43) and bounce-back (Eq. 44) do not
    depend on how the solid is described."""
    nx, ny = 40, 24
    x, y = W.grid(nx, ny)
    c1 = W.profile(x, y, 14, -0.5, 8, 4.0, period_x=nx)
    c2 = W.profile(x, y, 28, ny - 0.5, 7, 4.0, period_x=nx)
    ux = 0.003 * np.sin(2 * np.pi * x / nx)
    sig = (1.2e-3, 1.0e-3, 0.9e-3)
    prm = W.params(sigma=sig, theta=(W.theta12_from(*sig, 65, 115), 65, 115), rho=(3.0, 2.0, 1.0))
    A = _run(nx, ny, (0, 0, 1, 1), prm, c1, c2, ux=ux)
    mask = np.zeros((ny + 1, nx), np.uint8)
    mask[0] = 1
    pad = lambda a: np.vstack([np.zeros((1, nx)), a])
    B = _run(nx, ny + 1, (0, 0, 0, 0), prm, pad(c1), pad(c2), ux=pad(ux), mask=mask)
    A.step(200)
    B.step(200)
    fa, fb = A.fields(), B.fields()
    for k in ("c1", "c2", "ux", "uy", "p", "mu1", "mu2"):
        assert np.abs(fa[k] - fb[k][1:]).max() <= 1e-14 * max(1.0, np.abs(fa[k]).max()), k


def test_film_thickness_measurement():
    """The film reading: crossing of c = 1/2 above the half-way wall."""
    ny, nx, y_top = 40, 3, 9
    c = np.zeros((ny, nx))
    # a linear ramp 1 -> 0 between rows 20 and 21 crosses 1/2 at 20.5: h = 20.5 - 9.5
    c[10:21, 1] = 1.0
    c[20, 1] = 0.75
    c[21, 1] = 0.25
    assert oracle.film_thickness(c, 1, y_top) == pytest.approx(11.0, abs=1e-15)
    # no liquid on the solid: zero
    assert oracle.film_thickness(c, 0, y_top) == 0.0
    # liquid up to the top row: bounded by it
    c[10:, 2] = 1.0
    assert oracle.film_thickness(c, 2, y_top) == pytest.approx(ny - 1 - (y_top + 0.5))
    # a tanh film of thickness h0 (Eq. 50 profile across a flat interface)
    y = np.arange(ny, dtype=float)
    for h0 in (6.3, 12.8):
        prof = 0.5 + 0.5 * np.tanh(2.0 * (h0 - (y - (y_top + 0.5))) / 4.0)
        prof[: y_top + 1] = 0.0
        col = np.repeat(prof[:, None], 1, axis=1)
        assert abs(oracle.film_thickness(col, 0, y_top) - h0) < 0.02
