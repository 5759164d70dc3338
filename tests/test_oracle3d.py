"""Pins of the D3Q19 form of the oracle (the model of Sec. II.A in three
dimensions): lattice identities, exact stencils, invariants of the whole step
and closed-form physics, each fixed independently of the code.

- D3Q19 moments: sum w = 1, sum w e_a e_b = cs^2 delta_ab, fourth-order
  isotropy, opposite table.
- Eq. 20 on D3Q19: exact gradient of a linear field and Laplacian of a
  quadratic one (cross terms included).
- Whole step: each component's mass conserved to round-off with walls and
  solids; the uniform rest state is a fixed point; a uniform flow stays
  uniform; mirror symmetry in x and symmetry under a cyclic permutation of
  the axes.
- Closed forms: the linearised Cahn-Hilliard decay rate (Eq. 16 with Eq. 8,
  the mobility of Eq. 18a, D3Q19's discrete Laplacian symbol), the shear-wave
  decay at the mixture viscosity (Eqs. 15, 18b), the Laplace jump of a
  spherical drop, p_in - p_out = 2 sigma / R.
- Projection: D3Q19 summed over e_z is D2Q9 (weights 4/9, 1/9, 1/36), and
  the wetting ghost of Eq. 42 is the same on every link, so a state uniform in
  z has the steady states of the D2Q9 model; only the pressure transients
  differ (Eq. 13c counts the z-links as moving populations in 3D and as rest
  in 2D).  Two drops on a wetting wall reach the D2Q9 oracle's contact angles.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import OracleLattice, OracleLattice3D


def run3(w, steps=0):
    O = OracleLattice3D(w.nx, w.ny, w.nz, w.edges, w.mask, w.params)
    O.set_fields(w.c1, w.c2, w.ux, w.uy, w.uz, w.p)
    if steps:
        O.step(steps)
    return O


def test_d3q19_moments_and_opposites():
    e, w, opp = oracle.lattice3_vectors()
    assert abs(w.sum() - 1) < 1e-15
    assert np.allclose(np.einsum("k,ka,kb->ab", w, e, e), np.eye(3) / 3, atol=1e-15)
    assert np.allclose(np.einsum("k,ka->a", w, e), 0, atol=1e-15)
    assert np.allclose(np.einsum("k,ka,kb,kc->abc", w, e, e, e), 0, atol=1e-15)
    d = np.eye(3)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.allclose(np.einsum("k,ka,kb,kc,kd->abcd", w, e, e, e, e), iso, atol=1e-15)
    assert all((e[opp[k]] == -e[k]).all() for k in range(19))
    assert sorted(map(tuple, e.tolist())) == sorted({tuple(v) for v in e.tolist()})  # distinct


def test_stencils_exact_on_linear_and_quadratic_fields():
    e, _, _ = oracle.lattice3_vectors()
    rng = np.random.default_rng(4)
    b = rng.standard_normal(3)
    A = rng.standard_normal((3, 3))
    A = A + A.T
    x0 = rng.standard_normal(3)
    lin = [b @ (x0 + e[k]) for k in range(19)]
    assert np.allclose(oracle.grad3(lin), b, atol=1e-13)
    quad = [(x0 + e[k]) @ A @ (x0 + e[k]) + b @ (x0 + e[k]) for k in range(19)]
    assert abs(oracle.lap3(quad) - 2 * np.trace(A)) < 1e-12
    assert np.allclose(oracle.grad3(quad), 2 * A @ x0 + b, atol=1e-12)


@pytest.mark.parametrize("seed,edges,solids", [
    (1, (0, 0, 1, 2, 0, 0), ("sphere",)),
    (2, (1, 2, 1, 1, 2, 1), ("pillar", "corner")),
    (3, (0, 0, 0, 0, 0, 0), ("sphere", "corner")),
])
def test_mass_of_each_component_is_conserved(seed, edges, solids):
    w = W.random_lattice3(14, 12, 10, seed, edges=edges, solids=solids)
    O = run3(w)
    m0 = O.mass()
    O.step(40)
    m1 = O.mass()
    assert np.allclose(m1[:2], m0[:2], rtol=1e-12, atol=1e-12)


def test_uniform_rest_state_is_a_fixed_point():
    w = W.random_lattice3(8, 7, 6, 5, edges=(0, 0, 1, 2, 1, 2), solids=())
    w.c1[:] = 0.3
    w.c2[:] = 0.25
    for a in (w.ux, w.uy, w.uz):
        a[:] = 0
    # neutral wetting (cos = 0 for every pair) keeps the walls' ghosts symmetric
    w.params.update(gx=0.0, gy=0.0, theta12_deg=90.0, theta13_deg=90.0, theta23_deg=90.0)
    O = run3(w)
    s0 = O.state()
    O.step(20)
    assert np.abs(O.state() - s0).max() < 2e-14  # round-off of the BGK update


def test_uniform_flow_stays_uniform():
    w = W.random_lattice3(8, 7, 6, 6, edges=(0,) * 6, solids=())
    w.c1[:] = 0.4
    w.c2[:] = 0.1
    w.ux[:], w.uy[:], w.uz[:] = 0.01, -0.02, 0.005
    w.params.update(gx=0.0, gy=0.0)
    O = run3(w, steps=10)
    f = O.fields()
    for k, v in (("c1", 0.4), ("c2", 0.1), ("ux", 0.01), ("uy", -0.02), ("uz", 0.005)):
        assert np.abs(f[k] - f[k].mean()).max() < 1e-15, k
        assert abs(f[k].mean() - v) < 1e-12, k


def test_mirror_symmetry_in_x():
    w = W.random_lattice3(12, 10, 8, 7, edges=(1, 1, 1, 2, 0, 0), solids=("sphere",))
    m = W.Workload3(w.name, w.nx, w.ny, w.nz, w.edges, w.mask[:, :, ::-1].copy(), w.params,
                    w.c1[:, :, ::-1].copy(), w.c2[:, :, ::-1].copy(), -w.ux[:, :, ::-1].copy(),
                    w.uy[:, :, ::-1].copy(), w.uz[:, :, ::-1].copy())
    a, b = run3(w, 20).fields(), run3(m, 20).fields()
    for k in ("c1", "c2", "p", "mu1", "uy", "uz"):
        assert np.abs(a[k][:, :, ::-1] - b[k]).max() <= 1e-13 * max(1.0, np.abs(a[k]).max()), k
    assert np.abs(a["ux"][:, :, ::-1] + b["ux"]).max() <= 1e-13


def test_cyclic_permutation_of_the_axes():
    """(x, y, z) -> (y, z, x) on a periodic cube, no body force."""
    n = 9
    w = W.random_lattice3(n, n, n, 8, edges=(0,) * 6, solids=("sphere",))
    w.params.update(gx=0.0, gy=0.0)
    # rotated lattice: x' = y, y' = z, z' = x, so A'[z', y', x'] = A[z, y, x] at x = z', y = x', z = y'
    rot = lambda a: np.transpose(a, (2, 0, 1))  # noqa: E731
    r = W.Workload3(w.name, n, n, n, w.edges, rot(w.mask).copy(), w.params, rot(w.c1).copy(),
                    rot(w.c2).copy(), rot(w.uy).copy(), rot(w.uz).copy(), rot(w.ux).copy())
    a, b = run3(w, 15).fields(), run3(r, 15).fields()
    for k in ("c1", "c2", "p", "mu2"):
        assert np.abs(rot(a[k]) - b[k]).max() <= 1e-13 * max(1.0, np.abs(a[k]).max()), k
    for ka, kb in (("uy", "ux"), ("uz", "uy"), ("ux", "uz")):
        assert np.abs(rot(a[ka]) - b[kb]).max() <= 1e-13, (ka, kb)


def test_linearised_cahn_hilliard_decay_rate():
    """Binary sinusoid c1 = c0 + eps sin(k x) decays at M k^2 [12/D lambda
    phi'(c0) + 3/4 D lambda 2(1 - cos k)] (the D3Q19 Laplacian of a mode along
    x has the symbol -2(1 - cos k), as D2Q9's)."""
    nx, c0, eps, lam, D, M = 48, 0.1, 1e-3, 0.01, 4.0, 0.1
    prm = W.params(sigma=(lam, lam, lam), mobility=M, D=D, tau=(0.9, 0.8))
    x, y, z = W.grid3(nx, 3, 3)
    k = 2 * math.pi / nx
    zero = np.zeros_like(x)
    w = W.Workload3("ch", nx, 3, 3, (0,) * 6, np.zeros(x.shape, np.uint8), prm, c0 + eps * np.sin(k * x),
                    zero, zero, zero.copy(), zero.copy())
    O = run3(w)

    def amp():
        return 2 * np.mean((O.fields()["c1"] - c0) * np.sin(k * x))

    O.step(2000)
    a1 = amp()
    O.step(5000)
    rate = -math.log(amp() / a1) / 5000
    phi_p = 1 - 6 * c0 + 6 * c0 ** 2
    theory = M * k * k * (12 / D * lam * phi_p + 0.75 * D * lam * 2 * (1 - math.cos(k)))
    assert abs(rate / theory - 1) < 0.01


def test_shear_wave_decays_at_the_mixture_viscosity():
    nz, U = 40, 1e-4
    nus = (0.02, 0.15, 0.07)
    c1v, c2v = 0.3, 0.5
    prm = W.params(nu=nus)
    x, y, z = W.grid3(3, 3, nz)
    k = 2 * math.pi / nz
    zero = np.zeros_like(x)
    w = W.Workload3("sw", 3, 3, nz, (0,) * 6, np.zeros(x.shape, np.uint8), prm, zero + c1v, zero + c2v,
                    U * np.sin(k * z), zero.copy(), zero.copy())
    O = run3(w, 100)

    def amp():
        return 2 * np.mean(O.fields()["ux"] * np.sin(k * z))

    a1 = amp()
    O.step(800)
    rate = -math.log(amp() / a1) / 800
    nu = c1v * nus[0] + c2v * nus[1] + (1 - c1v - c2v) * nus[2]
    assert abs(rate / (nu * k * k) - 1) < 3e-3


def test_laplace_jump_of_a_spherical_drop():
    """p_in - p_out -> 2 sigma / R (here within 8% at R = 9, D = 4)."""
    n, R, sig = 30, 9.0, 1e-3
    x, y, z = W.grid3(n, n, n)
    zero = np.zeros_like(x)
    c1 = W.profile3(x, y, z, n / 2, n / 2, n / 2, R, 4.0, (n, n, n))
    w = W.Workload3("sphere", n, n, n, (0,) * 6, np.zeros(x.shape, np.uint8), W.params(sigma=(sig,) * 3), c1,
                    zero, zero, zero.copy(), zero.copy())
    f = run3(w, 1200).fields()
    dp = f["p"][n // 2, n // 2, n // 2] - f["p"][0, 0, 0]
    assert abs(dp * R / (2 * sig) - 1.0) < 0.08
    assert max(np.abs(f[k]).max() for k in ("ux", "uy", "uz")) < 2e-5


def test_state_uniform_in_z_converges_to_the_d2q9_oracle():
    """Two drops on a wetting wall, uniform in z: the D3Q19 run approaches the
    D2Q9 run as the pressure transients decay (the steady equations are the
    same: uniform mu in each phase, the same wetting ghosts), and the contact
    angle theta_n of Sec. III.A agrees to 0.01 deg after 2000 steps."""
    w2 = W.binary_drops_on_wall(nx=64, ny=32, R=10.0, sep=24.0)
    nz = 3
    st = lambda a: np.repeat(a[None], nz, 0)  # noqa: E731
    w3 = W.Workload3("z-uniform", w2.nx, w2.ny, nz, tuple(w2.edges) + (0, 0), st(w2.mask), w2.params,
                     st(w2.c1), st(w2.c2), st(w2.ux), st(w2.uy), np.zeros((nz, w2.ny, w2.nx)))
    O2 = OracleLattice(w2.nx, w2.ny, w2.edges, w2.mask, w2.params)
    O2.set_fields(w2.c1, w2.c2, w2.ux, w2.uy)
    O3 = run3(w3)
    O2.step(2000)
    O3.step(2000)
    a, b = O2.fields(), O3.fields()
    for k in ("c1", "c2"):
        assert np.abs(b[k] - b[k][:1]).max() < 1e-14  # stays uniform in z
        assert np.abs(b[k][0] - a[k]).max() < 1e-4, k
    assert np.abs(b["ux"][0] - a["ux"]).max() < 1e-3 * np.abs(a["ux"]).max()
    assert np.abs(b["uz"]).max() < 1e-15
    for comp in ("c1", "c2"):
        t2, t3 = oracle.contact_angle_deg(a[comp]), oracle.contact_angle_deg(b[comp][0])
        assert len(t2) == len(t3) == 1 and abs(t2[0] - t3[0]) < 0.01, (comp, t2, t3)


# ---- moments of the D3Q19 equilibria and sources (Eqs. 2a, 2b, 4, 11a, 11b)

RNG = np.random.default_rng(19)


@pytest.mark.parametrize("trial", range(5))
def test_equilibrium_moments(trial):
    e, w, _ = oracle.lattice3_vectors()
    e = e.astype(float)
    u = RNG.uniform(-0.08, 0.08, 3)
    c, mu, eta = RNG.uniform(0, 1), RNG.normal(0, 1e-3), RNG.uniform(0.3, 3)
    f = np.array([oracle.feq3(k, c, mu, eta, u) for k in range(19)])
    assert np.isclose(f.sum(), c, rtol=1e-14, atol=1e-16)
    assert np.allclose(e.T @ f, c * u, rtol=1e-13, atol=1e-17)
    assert np.allclose(np.einsum("k,ka,kb->ab", f, e, e), eta * mu / 3 * np.eye(3), rtol=1e-12, atol=1e-18)
    p, rho = RNG.normal(0, 1e-3), RNG.uniform(0.5, 10)
    s = np.array([oracle.sk3(k, u) for k in range(19)])
    g = np.array([oracle.geq3(k, p, rho, u) for k in range(19)])
    assert abs(s.sum()) < 1e-17 and np.allclose(e.T @ s, u, atol=1e-16)
    assert np.allclose(np.einsum("k,ka,kb->ab", s, e, e), np.outer(u, u), atol=1e-16)
    assert abs(g.sum()) < 1e-15
    assert np.allclose(e.T @ g, rho * u, rtol=1e-13, atol=1e-16)
    assert np.allclose(np.einsum("k,ka,kb->ab", g, e, e), p * np.eye(3) + rho * np.outer(u, u),
                       rtol=1e-12, atol=1e-16)


@pytest.mark.parametrize("trial", range(5))
def test_source_moments(trial):
    e, w, _ = oracle.lattice3_vectors()
    e = e.astype(float)
    tau = RNG.uniform(0.55, 1.5)
    dcu = RNG.normal(0, 1e-3, 3)
    F = np.array([oracle.src_f3(k, tau, dcu) for k in range(19)])
    assert abs(F.sum()) < 1e-18
    assert np.allclose(e.T @ F, (1 - 0.5 / tau) * dcu, rtol=1e-13, atol=1e-19)
    assert np.allclose(np.einsum("k,ka,kb->ab", F, e, e), 0, atol=1e-18)
    taug = RNG.uniform(0.55, 1.5)
    u = RNG.uniform(-0.08, 0.08, 3)
    gr, Ft, Fa = RNG.normal(0, 0.1, 3), RNG.normal(0, 1e-4, 3), RNG.normal(0, 1e-5, 3)
    G = np.array([oracle.src_g3(k, taug, u, gr, Ft, Fa) for k in range(19)])
    a = 1 - 0.5 / taug
    assert np.isclose(G.sum(), a * (u @ gr), rtol=1e-12, atol=1e-17)
    assert np.allclose(e.T @ G, a * Ft + Fa, rtol=1e-11, atol=1e-17)


def _translation_error3(s):
    """A dense layer of fluid 1 (rho 10 in 1) across z, translating at U along
    x while it diffuses: u = U is exact (Eq. 17b); the lattice error must
    vanish at second order, which needs F_a (Eq. 12)."""
    U = 0.02
    nz, D = 64 * s, 4.0 * s
    prm = W.params(sigma=(1e-3,) * 3, rho=(10.0, 1.0, 1.0), mobility=1.0 * s, D=D, tau=(1.0, 1.0))
    x, y, z = W.grid3(3, 3, nz)
    c1 = 0.5 + 0.5 * np.tanh(2 * (16 * s - np.abs(z - 32 * s)) / (2 * D))
    zero = np.zeros_like(x)
    w = W.Workload3("layer", 3, 3, nz, (0,) * 6, np.zeros(x.shape, np.uint8), prm, c1, zero, U + zero,
                    zero.copy(), zero.copy())
    O = run3(w)
    r0 = O.fields()["rho"][:, 0, 0]
    O.step(400 * s * s)
    f = O.fields()
    du = f["ux"][:, 0, 0] - U
    dr = (f["rho"][:, 0, 0] - r0) / f["rho"][:, 0, 0]
    return np.polyfit(dr, du, 1)[0] / U


def test_uniform_translation_with_density_contrast_converges():
    e2, e4 = _translation_error3(2), _translation_error3(4)
    assert abs(e4) < 0.04
    assert abs(e2 / e4) > 3.0


def test_solid_layer_in_mask_equals_wall_edge():
    """A wetting wall given as a solid layer of the mask (the lattice one layer
    taller, periodic in y) and the same wall given as the y- edge give the same
    fields: Eqs. 42-44 do not depend on how the solid is described."""
    nx, ny, nz = 16, 12, 10
    x, y, z = W.grid3(nx, ny, nz)
    c1 = W.profile3(x, y, z, 6, -0.5, 5, 5, 4.0, (nx, None, nz))
    c2 = W.profile3(x, y, z, 11, ny - 0.5, 4, 4, 4.0, (nx, None, nz))
    ux = 0.003 * np.sin(2 * np.pi * x / nx)
    uz = 0.002 * np.cos(2 * np.pi * z / nz)
    sig = (1.2e-3, 1.0e-3, 0.9e-3)
    prm = W.params(sigma=sig, theta=(W.theta12_from(*sig, 65, 115), 65, 115), rho=(3.0, 2.0, 1.0))
    zero = np.zeros_like(x)
    A = W.Workload3("edge", nx, ny, nz, (0, 0, 1, 1, 0, 0), np.zeros(x.shape, np.uint8), prm, c1, c2, ux,
                    zero, uz)
    pad = lambda a: np.concatenate([np.zeros((nz, 1, nx)), a], axis=1)  # noqa: E731
    mask = np.zeros((nz, ny + 1, nx), np.uint8)
    mask[:, 0, :] = 1
    B = W.Workload3("mask", nx, ny + 1, nz, (0,) * 6, mask, prm, pad(c1), pad(c2), pad(ux), pad(zero), pad(uz))
    fa, fb = run3(A, 60).fields(), run3(B, 60).fields()
    for k in ("c1", "c2", "ux", "uy", "uz", "p", "mu1", "mu2"):
        assert np.abs(fa[k] - fb[k][:, 1:]).max() <= 1e-14 * max(1.0, np.abs(fa[k]).max()), k


def test_translation_pin_covers_fluid_two():
    """The exact translation solution with the dense layer made of fluid 2
    (the second term of Eq. 14 and of F_a in Eq. 12)."""
    U, s = 0.02, 4
    nz, D = 64 * s, 4.0 * s
    prm = W.params(sigma=(1e-3,) * 3, rho=(1.0, 10.0, 1.0), mobility=1.0 * s, D=D, tau=(1.0, 1.0))
    x, y, z = W.grid3(3, 3, nz)
    c2 = 0.5 + 0.5 * np.tanh(2 * (16 * s - np.abs(z - 32 * s)) / (2 * D))
    zero = np.zeros_like(x)
    w = W.Workload3("layer2", 3, 3, nz, (0,) * 6, np.zeros(x.shape, np.uint8), prm, zero, c2, U + zero,
                    zero.copy(), zero.copy())
    O = run3(w)
    r0 = O.fields()["rho"][:, 0, 0]
    O.step(400 * s * s)
    f = O.fields()
    assert abs(r0.max() - 10.0) < 0.01  # the layer carries fluid 2's density
    slope = np.polyfit((f["rho"][:, 0, 0] - r0) / f["rho"][:, 0, 0], f["ux"][:, 0, 0] - U, 1)[0] / U
    assert abs(slope) < 0.04


def test_body_force_plane_poiseuille_and_hydrostatics():
    """G = rho (gx, gy, 0) (Eqs. 11b, 13b): a plane Poiseuille flow between
    half-way walls in y is parabolic (exact at tau_g - 1/2 = sqrt(3/16)), and a
    closed box at rest builds dp/dy = rho g_y."""
    ny, g = 16, 1e-6
    nu = math.sqrt(3.0) / 12.0
    zero = np.zeros((3, ny, 3))
    mk = lambda prm: W.Workload3("pois", 3, ny, 3, (0, 0, 2, 2, 0, 0), np.zeros(zero.shape, np.uint8), prm,  # noqa: E731
                                 zero, zero, zero, zero, zero)
    f = run3(mk(W.params(nu=(nu,) * 3, g=(g, 0.0))), 20000).fields()
    y = np.arange(ny)
    exact = g / (2 * nu) * (y + 0.5) * (ny - 0.5 - y)
    assert np.abs(f["ux"][0, :, 0] - exact).max() < 1e-7 * exact.max()
    f = run3(mk(W.params(nu=(0.1,) * 3, g=(0.0, -1e-5), rho=(1, 1, 2.0))), 15000).fields()
    assert np.allclose(np.diff(f["p"][0, :, 0]), 2.0 * -1e-5, rtol=1e-9)
    assert max(np.abs(f[k]).max() for k in ("ux", "uy", "uz")) < 1e-15
