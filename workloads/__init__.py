"""Seeded synthetic inputs shaped like the paper's workloads.

This module only builds inputs: lattice sizes, edge kinds, solid masks,
parameter sets and initial fields.  It contains none of the lattice update's
arithmetic, and both the FP64 oracle and the CUDA library consume what it
returns.  Every random draw comes from ``numpy.random.default_rng(seed)``.

Conventions (shared by both implementations):
  * arrays are [ny, nx]; node (i, j) sits at (x, y) = (i, j);
  * edges = (left, right, bottom, top) with 0 periodic, 1 wetting wall,
    2 neutral wall, 3 velocity lid (top only); half-way walls sit half a
    spacing outside the first and last rows/columns;
  * mask: 0 fluid, 1 wetting solid, 2 neutral solid; a cylinder node is solid
    iff its distance to the centre is <= R;
  * the initial order parameter of a drop of radius R is the smooth profile
    0.5 + 0.5 tanh(2 (R - r) / D) of Eqs. 46, 50 and 56, with r the Euclidean
    distance (the printed formulas drop the square root); a compound drop is
    c1 = profile(R_core), c2 = profile(R_shell) - c1;
  * "mobility m" in a workload description means M_1 = m, i.e. M0 = m * lambda_1
    (the paper quotes M_1 = M_2 = 0.1 directly in Sec. III.D).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PERIODIC, WETTING, NEUTRAL, LID = 0, 1, 2, 3


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    edges: tuple
    mask: np.ndarray
    params: dict
    c1: np.ndarray
    c2: np.ndarray
    ux: np.ndarray
    uy: np.ndarray
    p: np.ndarray | None = None
    steps: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def nodes(self) -> int:
        return self.nx * self.ny


def lambda1(s12, s13, s23):
    return s12 + s13 - s23


def theta12_from(s12, s13, s23, th13_deg, th23_deg):
    """theta_12 from the Eq. 39 constraint, given theta_13 and theta_23 (degrees)."""
    c = (s13 * math.cos(math.radians(th13_deg)) - s23 * math.cos(math.radians(th23_deg))) / s12
    if abs(c) > 1.0:
        raise ValueError("no theta_12 satisfies Eq. 39 for these angles")
    return math.degrees(math.acos(c))


def params(*, sigma=(1e-3, 1e-3, 1e-3), theta=(90.0, 90.0, 90.0), rho=(1.0, 1.0, 1.0),
           nu=(0.1, 0.1, 0.1), mobility=0.1, D=4.0, tau=(0.8, 0.8), g=(0.0, 0.0),
           lid_u=0.0, M0=None, mrt=None) -> dict:
    """Parameter set; mrt = (s_f, s_g) selects the MRT collision with those rates
    for the non-conserved, non-flux moments of f^i and the energy moments of g."""
    s12, s13, s23 = sigma
    if M0 is None:
        M0 = mobility * lambda1(s12, s13, s23)
    return dict(sigma12=s12, sigma13=s13, sigma23=s23,
                theta12_deg=theta[0], theta13_deg=theta[1], theta23_deg=theta[2],
                rho1=rho[0], rho2=rho[1], rho3=rho[2], nu1=nu[0], nu2=nu[1], nu3=nu[2],
                M0=M0, D=D, tau1=tau[0], tau2=tau[1], gx=g[0], gy=g[1], lid_u=lid_u,
                collision=0.0 if mrt is None else 1.0,
                mrt_s_f=1.0 if mrt is None else mrt[0], mrt_s_g=1.0 if mrt is None else mrt[1])


def grid(nx, ny):
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    return x, y


def profile(x, y, xc, yc, R, D, period_x=None, period_y=None):
    """0.5 + 0.5 tanh(2 (R - r) / D), r the (minimum-image if periodic) distance."""
    dx = x - xc
    dy = y - yc
    if period_x:
        dx = (dx + period_x / 2) % period_x - period_x / 2
    if period_y:
        dy = (dy + period_y / 2) % period_y - period_y / 2
    r = np.sqrt(dx * dx + dy * dy)
    return 0.5 + 0.5 * np.tanh(2.0 * (R - r) / D)


def _zeros(nx, ny):
    return np.zeros((ny, nx))


def _window(nx, ny, xc, yc, R, D, period_x=None):
    """Rows y0..y1-1 and columns `cols` of the nodes within R + 10 D of (xc, yc)
    (minimum image in x when periodic).  Beyond that distance the profile
    0.5 + 0.5 tanh(2 (R - r) / D) is exactly 0 in FP64 (tanh(-20) rounds to -1),
    so a profile evaluated on this window only is the whole-grid one, bit for bit."""
    reach = R + 10.0 * D
    y0, y1 = max(0, int(np.floor(yc - reach))), min(ny, int(np.ceil(yc + reach)) + 1)
    lo, hi = int(np.floor(xc - reach)), int(np.ceil(xc + reach)) + 1
    if period_x:
        cols = np.arange(lo, hi) % nx if hi - lo < nx else np.arange(nx)
    else:
        cols = np.arange(max(0, lo), min(nx, hi))
    return y0, max(y0, y1), cols


# ---- the paper-shaped workloads -------------------------------------------

def binary_drops_on_wall(nx=128, ny=64, R=16.0, sep=40.0, theta=(60.0, 90.0, 120.0),
                         steps=2000) -> Workload:
    """Two semicircular drops (fluid 1 and fluid 2) on a wetting bottom wall in
    fluid 3, neutral top wall, periodic in x (Sec. III.A set-up at 128x64)."""
    x, y = grid(nx, ny)
    xc1 = nx / 2 - sep / 2
    xc2 = nx / 2 + sep / 2
    c1 = profile(x, y, xc1, -0.5, R, 4.0, period_x=nx)
    c2 = profile(x, y, xc2, -0.5, R, 4.0, period_x=nx)
    P = params(sigma=(1e-3, 1e-3, 1e-3), theta=theta, rho=(1, 1, 1), nu=(0.1, 0.1, 0.1),
               mobility=0.1, D=4.0)
    return Workload("binary_drops_128x64", nx, ny, (PERIODIC, PERIODIC, WETTING, NEUTRAL),
                    np.zeros((ny, nx), np.uint8), P, c1, c2, _zeros(nx, ny), _zeros(nx, ny),
                    steps=steps)


def puddles(g, nx=600, ny=150, R=60.0, rho=(10.0, 5.0, 1.0), sigma=0.1, theta=90.0, M0=0.01,
            steps=200000) -> Workload:
    """Two drops (fluid 1, density 10; fluid 2, density 5) on a wetting bottom
    wall in fluid 3 (density 1) under gravity G = (0, -rho g) (Sec. III.A with
    gravity): L x W = 600 x 150, R = 0.1 L centred on the wall at 0.25 L and
    0.75 L, sigma_ij = 0.1, tau_i = tau_g = 0.8, M0 = 0.01, D = 4,
    theta_13 = theta_23 = theta (theta_12 from Eq. 39), bounce-back top wall."""
    x, y = grid(nx, ny)
    c1 = profile(x, y, 0.25 * nx, -0.5, R, 4.0, period_x=nx)
    c2 = profile(x, y, 0.75 * nx, -0.5, R, 4.0, period_x=nx)
    th12 = theta12_from(sigma, sigma, sigma, theta, theta)
    P = params(sigma=(sigma, sigma, sigma), theta=(th12, theta, theta), rho=rho, nu=(0.1, 0.1, 0.1),
               M0=M0, D=4.0, tau=(0.8, 0.8), g=(0.0, -g))
    return Workload(f"puddles_{nx}x{ny}_g{g:g}", nx, ny, (PERIODIC, PERIODIC, WETTING, NEUTRAL),
                    np.zeros((ny, nx), np.uint8), P, c1, c2, _zeros(nx, ny), _zeros(nx, ny),
                    steps=steps, meta=dict(g=g, R=R, rho=rho, sigma=sigma, theta=theta))


def puddle_thickness(sigma, rho_liquid, g, theta_deg):
    """Eq. 48: H = 2 sqrt(sigma / (rho_l g)) sin(theta_e / 2) (de Gennes' puddle)."""
    return 2.0 * math.sqrt(sigma / (rho_liquid * g)) * math.sin(math.radians(theta_deg) / 2)


def compound_drop_shear(nx=512, ny=256, R_core=30.0, R_shell=50.0, U0=0.01, steps=20000,
                        sigma=(2e-3, 1e-3, 1e-3), theta13=90.0, theta23=135.0) -> Workload:
    """Compound drop (core fluid 1, shell fluid 2) on a wetting wall in fluid 3,
    sheared by a velocity lid (Sec. III.C set-up at 512x256).  theta_12 is
    derived from Eq. 39 (the paper's convention for given theta_13, theta_23)."""
    x, y = grid(nx, ny)
    xc = nx / 2
    c1 = profile(x, y, xc, -0.5, R_core, 4.0, period_x=nx)
    c2 = profile(x, y, xc, -0.5, R_shell, 4.0, period_x=nx) - c1
    th12 = theta12_from(*sigma, theta13, theta23)
    P = params(sigma=sigma, theta=(th12, theta13, theta23), rho=(1.0, 2.0, 1.0),
               nu=(0.05, 0.1, 0.05), mobility=0.1, D=4.0, lid_u=U0)
    ux = _zeros(nx, ny)
    ux[ny - 1, :] = U0
    return Workload(f"compound_drop_shear_{nx}x{ny}", nx, ny,
                    (PERIODIC, PERIODIC, WETTING, LID), np.zeros((ny, nx), np.uint8), P,
                    c1, c2, ux, _zeros(nx, ny), steps=steps)


def compound_drop_on_cylinder(nx=1024, ny=2048, R_cyl=120.0, R_core=60.0, R_shell=100.0,
                              We=10.0, theta=90.0, steps=50000, cyl_center=None,
                              drop_center=None) -> Workload:
    """Compound drop falling onto a wetting circular cylinder, fully periodic
    (Sec. III.D set-up).  sigma_ij = 0.01, rho = (10, 10, 1), nu_i = 0.02,
    M_1 = M_2 = 0.1, theta_12 = 90, theta_13 = theta_23 = theta; the impact
    speed U follows from We = rho_bar xi U^2 / sigma_bar (Eq. 55) with
    xi = 2 R_shell; u0 = (0, -U) (c1 + c2)."""
    x, y = grid(nx, ny)
    cx, cy = cyl_center or (nx / 2, nx / 2)
    dx_, dy_ = drop_center or (nx / 2, nx / 2 + R_cyl + R_shell + 48.0)
    mask = (((x - cx) ** 2 + (y - cy) ** 2) <= R_cyl ** 2).astype(np.uint8)
    c1 = profile(x, y, dx_, dy_, R_core, 4.0, period_x=nx, period_y=ny)
    c2 = profile(x, y, dx_, dy_, R_shell, 4.0, period_x=nx, period_y=ny) - c1
    c1[mask == 1] = 0.0
    c2[mask == 1] = 0.0
    sig = 0.01
    rho_bar = 10.0
    xi = 2.0 * R_shell
    U = math.sqrt(We * sig / (rho_bar * xi))
    P = params(sigma=(sig, sig, sig), theta=(90.0, theta, theta), rho=(10.0, 10.0, 1.0),
               nu=(0.02, 0.02, 0.02), mobility=0.1, D=4.0)
    uy = -U * (c1 + c2)
    return Workload(f"compound_drop_on_cylinder_{nx}x{ny}", nx, ny,
                    (PERIODIC, PERIODIC, PERIODIC, PERIODIC), mask, P, c1, c2,
                    _zeros(nx, ny), uy, steps=steps,
                    meta=dict(We=We, U=U, Re=xi * U / 0.02))


def impact_e5(We=21.6, theta13=30.0, L=240, W=280, single=False, mrt=None) -> Workload:
    """Compound drop impact on a cylinder at the paper's size (Sec. III.D):
    L x W = 240 x 280 fully periodic; cylinder R = L/8 centred at (L/2, L/2);
    drop centred at (L/2, 3L/4), core fluid 1 of radius L/16 in a shell of
    fluid 2 of outer radius L/8 (xi = L/4); rho_1 = rho_2 = 10, rho_3 = 1;
    U = 0.06 downward, Re = xi U / nu = 600; sigma_ij all equal, set by We =
    rho_bar xi U^2 / sigma_bar (Eq. 55); theta_12 = 90, theta_13 = theta_23;
    M_1 = M_2 = 0.1, tau_1 = tau_2 = 0.8.  single=True: c1 = 0 (the
    single-drop comparison).  meta: xi, U, x and y_top of the cylinder top."""
    x, y = grid(L, W)
    xc, yc, Rc = L / 2, L / 2, L / 8
    mask = (((x - xc) ** 2 + (y - yc) ** 2) <= Rc ** 2).astype(np.uint8)
    R_out, R_in = L / 8, L / 16
    c1 = np.zeros((W, L)) if single else profile(x, y, L / 2, 0.75 * L, R_in, 4.0, period_x=L, period_y=W)
    c2 = profile(x, y, L / 2, 0.75 * L, R_out, 4.0, period_x=L, period_y=W) - c1
    c1[mask == 1] = 0.0
    c2[mask == 1] = 0.0
    xi, U = L / 4, 0.06
    nu = xi * U / 600.0
    sig = 10.0 * xi * U * U / We
    P = params(sigma=(sig, sig, sig), theta=(90.0, theta13, theta13), rho=(10.0, 10.0, 1.0),
               nu=(nu, nu, nu), mobility=0.1, D=4.0, tau=(0.8, 0.8), mrt=mrt)
    col = int(round(xc))
    y_top = int(max(yy for yy in range(W) if mask[yy, col]))
    return Workload(f"impact_e5_{L}x{W}_We{We:g}_th{theta13:g}" + ("_single" if single else ""), L, W,
                    (PERIODIC, PERIODIC, PERIODIC, PERIODIC), mask, P, c1, c2, _zeros(L, W), -U * (c1 + c2),
                    steps=int(10 * xi / U), meta=dict(xi=xi, U=U, x_top=col, y_top=y_top, We=We))


def tiled_drops(nx=2048, ny=2048, seed=1710, steps=1000) -> Workload:
    """Large lattice with the binary-drop physics tiled up: drops of fluid 1 and
    fluid 2 (R = 16) every 40 nodes along a wetting bottom wall, a neutral top
    wall, periodic in x, plus seeded free compound drops in the bulk."""
    rng = np.random.default_rng(seed)
    c1 = np.zeros((ny, nx))
    c2 = np.zeros((ny, nx))

    # each drop is evaluated on the window where its profile is nonzero (the
    # same values as on the whole grid; the maxima below leave the rest as is)
    def win(xc, yc, R):
        y0, y1, cols = _window(nx, ny, xc, yc, R, 4.0, period_x=nx)
        xs = cols.astype(float)[None, :]
        ys = np.arange(y0, y1, dtype=float)[:, None]
        return (slice(y0, y1), cols), xs, ys

    for i, xc in enumerate(np.arange(20.0, nx, 40.0)):
        ix, xs, ys = win(xc, -0.5, 16.0)
        prof = profile(xs, ys, xc, -0.5, 16.0, 4.0, period_x=nx)
        tgt = c1 if i % 2 == 0 else c2
        tgt[ix] = np.maximum(tgt[ix], prof)
    n_free = max(1, (nx * ny) // 60000)
    for _ in range(n_free):
        xc = rng.uniform(0, nx)
        yc = rng.uniform(80, ny - 60)
        rs = rng.uniform(10, 24)
        ix, xs, ys = win(xc, yc, rs)
        prof_s = profile(xs, ys, xc, yc, rs, 4.0, period_x=nx)
        prof_c = profile(xs, ys, xc, yc, 0.55 * rs, 4.0, period_x=nx)
        a, b = c1[ix], c2[ix]
        keep = a + b < 0.01
        c1[ix] = np.where(keep, np.maximum(a, prof_c), a)
        c2[ix] = np.where(keep, np.maximum(b, prof_s - prof_c), b)
    P = params(sigma=(1e-3, 1e-3, 1e-3), theta=(60.0, 90.0, 120.0), mobility=0.1, D=4.0)
    return Workload(f"tiled_drops_{nx}x{ny}", nx, ny, (PERIODIC, PERIODIC, WETTING, NEUTRAL),
                    np.zeros((ny, nx), np.uint8), P, np.clip(c1, 0, 1), np.clip(c2, 0, 1),
                    _zeros(nx, ny), _zeros(nx, ny), steps=steps)


# ---- random small lattices for parity tests -------------------------------

def random_lattice(nx, ny, seed, edges=None, solids=("disc",), u_amp=0.01, rho=(1.0, 3.0, 1.0),
                   lid_u=0.0) -> Workload:
    """Random drops, a random solid mask (discs, pillars, L-shaped concave
    corners), small random velocity.  Used to reach every branch of the wall
    rules in parity tests."""
    rng = np.random.default_rng(seed)
    if edges is None:
        edges = (PERIODIC, PERIODIC, WETTING, NEUTRAL)
    x, y = grid(nx, ny)
    mask = np.zeros((ny, nx), np.uint8)
    for kind in solids:
        kind_val = int(rng.integers(1, 3))
        if kind == "disc":
            cx, cy, R = rng.uniform(0.3 * nx, 0.7 * nx), rng.uniform(0.3 * ny, 0.7 * ny), rng.uniform(3, max(4, min(nx, ny) / 6))
            mask[((x - cx) ** 2 + (y - cy) ** 2) <= R * R] = kind_val
        elif kind == "pillar":
            px, py = int(rng.integers(3, nx - 3)), int(rng.integers(3, ny - 3))
            mask[py, px] = kind_val
        elif kind == "corner":
            px, py = int(rng.integers(4, nx - 8)), int(rng.integers(4, ny - 8))
            mask[py:py + 4, px:px + 2] = kind_val
            mask[py:py + 2, px:px + 5] = kind_val
    # keep the lid row and the row below it fluid
    if edges[3] == LID:
        mask[ny - 3:, :] = 0
    c1 = np.zeros((ny, nx))
    c2 = np.zeros((ny, nx))
    for i in range(int(rng.integers(2, 5))):
        xc, yc = rng.uniform(0, nx), rng.uniform(0, ny)
        R = rng.uniform(3, max(4, min(nx, ny) / 4))
        prof = profile(x, y, xc, yc, R, 4.0, period_x=nx if edges[0] == PERIODIC else None,
                       period_y=ny if edges[2] == PERIODIC else None)
        if i % 2 == 0:
            c1 = np.maximum(c1, prof)
        else:
            c2 = np.maximum(c2, prof)
    s = c1 + c2
    over = s > 1
    c1[over] /= s[over]
    c2[over] /= s[over]
    c1[mask > 0] = 0
    c2[mask > 0] = 0
    ux = u_amp * rng.standard_normal((ny, nx))
    uy = u_amp * rng.standard_normal((ny, nx))
    ux[mask > 0] = 0
    uy[mask > 0] = 0
    sigma = tuple(rng.uniform(0.8e-3, 1.5e-3, 3))
    # keep lambda_i > 0.5 lambda_T (the well-posedness condition stated after Eq. 7) by drawing near-equal tensions
    th13, th23 = rng.uniform(40, 140, 2)
    try:
        th12 = theta12_from(*sigma, th13, th23)
    except ValueError:
        th13, th23 = 90.0, 90.0
        th12 = theta12_from(*sigma, th13, th23)
    P = params(sigma=sigma, theta=(th12, th13, th23), rho=rho,
               nu=tuple(rng.uniform(0.05, 0.15, 3)), mobility=float(rng.uniform(0.05, 0.15)),
               D=float(rng.choice([3.0, 4.0, 5.0])), tau=tuple(rng.uniform(0.7, 1.0, 2)),
               g=(0.0, -1e-6), lid_u=lid_u)
    if edges[3] == LID:
        ux[ny - 1, :] = lid_u
        uy[ny - 1, :] = 0
    return Workload(f"random_{nx}x{ny}_s{seed}", nx, ny, tuple(edges), mask, P, c1, c2, ux, uy,
                    steps=0)


# ---- many independent lattices (batched / served workloads) ------------------

def _draw_tensions_and_angles(rng):
    """sigma_ij ~ U[5e-4, 2e-3] each, redrawn until lambda_i > lambda_T / 2 (the
    well-posed range stated after Eq. 7); theta_13, theta_23 ~ U[30, 150] deg with
    theta_12 from Eq. 39, redrawn until it exists."""
    while True:
        s = rng.uniform(5e-4, 2e-3, 3)
        lam = np.array([s[0] + s[1] - s[2], s[0] + s[2] - s[1], s[1] + s[2] - s[0]])
        if np.any(lam <= 0):
            continue
        lamT = 3.0 / np.sum(1.0 / lam)
        if np.any(lam <= 0.5 * lamT):
            continue
        th13, th23 = rng.uniform(30.0, 150.0, 2)
        try:
            th12 = theta12_from(*s, th13, th23)
        except ValueError:
            continue
        return tuple(s), (th12, th13, th23)


def drops_on_wall(n, seed, rng=None):
    """A square lattice of side n (x-periodic, wetting bottom wall, neutral top)
    with 1-4 non-overlapping drops of radius U[8, 40] (fluid 1 or 2), on the wall
    or free; random admissible tensions and contact angles."""
    rng = rng or np.random.default_rng(seed)
    x, y = grid(n, n)
    c1 = np.zeros((n, n))
    c2 = np.zeros((n, n))
    placed = []
    for _ in range(int(rng.integers(1, 5))):
        for _attempt in range(20):
            R = float(rng.uniform(8.0, min(40.0, n / 4)))
            on_wall = rng.random() < 0.5
            xc = float(rng.uniform(0, n))
            yc = -0.5 if on_wall else float(rng.uniform(R + 4, n - R - 4))
            if all(np.hypot(((xc - px + n / 2) % n) - n / 2, yc - py) > R + pr + 6 for px, py, pr in placed):
                placed.append((xc, yc, R))
                prof = profile(x, y, xc, yc, R, 4.0, period_x=n)
                if rng.random() < 0.5:
                    c1 = np.maximum(c1, prof)
                else:
                    c2 = np.maximum(c2, prof)
                break
    sigma, theta = _draw_tensions_and_angles(rng)
    P = params(sigma=sigma, theta=theta, rho=(1.0, 1.0, 1.0), nu=(0.1, 0.1, 0.1), mobility=0.1, D=4.0)
    z = np.zeros((n, n))
    return Workload(f"drops_on_wall_{n}", n, n, (PERIODIC, PERIODIC, WETTING, NEUTRAL),
                    np.zeros((n, n), np.uint8), P, c1, c2, z, z.copy())


def batch_population(count=256, seed=1710, lo=64, hi=512):
    """`count` lattices with square sides log-uniform in [lo, hi] rounded to
    multiples of 8, each a drops-on-wall problem (the batched workload)."""
    rng = np.random.default_rng(seed)
    sides = np.exp(rng.uniform(np.log(lo), np.log(hi), count))
    sides = np.clip((np.round(sides / 8) * 8).astype(int), lo, hi)
    return [drops_on_wall(int(n), 0, rng) for n in sides]


def drop_on_cylinder(n, rng):
    """A fully periodic square lattice of side n with a wetting cylinder of
    radius n/8 and a compound drop (core n/24, shell n/12) above it falling at
    the speed of a random Weber number in [1, 50] (the impact set-up)."""
    sig = float(rng.uniform(5e-3, 1.5e-2))
    th = float(rng.uniform(30.0, 150.0))
    w = compound_drop_on_cylinder(nx=n, ny=n, R_cyl=n / 8, R_core=n / 24, R_shell=n / 12,
                                  We=float(rng.uniform(1.0, 50.0)), theta=th,
                                  cyl_center=(n / 2, n / 2), drop_center=(n / 2, n / 2 + n / 8 + n / 12 + 6))
    s12 = sig
    w.params.update(params(sigma=(s12, sig, sig), theta=(90.0, th, th), rho=(10.0, 10.0, 1.0),
                           nu=(0.02, 0.02, 0.02), mobility=0.1, D=4.0))
    w.name = f"drop_on_cylinder_{n}"
    return w


def served_requests(count=200, seed=1710, lo=128, hi=2048, steps_lo=1000, steps_hi=20000):
    """The served workload: `count` jobs, half drops on a wetting wall and half
    compound drops onto a cylinder, square sides log-uniform in [lo, hi]
    (multiples of 8) and step counts log-uniform in [steps_lo, steps_hi].
    Returns a list of (workload, steps)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(np.clip(round(math.exp(rng.uniform(math.log(lo), math.log(hi))) / 8) * 8, lo, hi))
        steps = int(round(math.exp(rng.uniform(math.log(steps_lo), math.log(steps_hi)))))
        w = drops_on_wall(n, 0, rng) if rng.random() < 0.5 else drop_on_cylinder(n, rng)
        out.append((w, steps))
    return out


# ---- three-dimensional (D3Q19) inputs ----------------------------------------

@dataclass
class Workload3:
    """A D3Q19 problem: arrays are [nz, ny, nx]; edges = (x-, x+, y-, y+, z-,
    z+), each PERIODIC, WETTING or NEUTRAL."""
    name: str
    nx: int
    ny: int
    nz: int
    edges: tuple
    mask: np.ndarray
    params: dict
    c1: np.ndarray
    c2: np.ndarray
    ux: np.ndarray
    uy: np.ndarray
    uz: np.ndarray
    p: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def nodes(self) -> int:
        return self.nx * self.ny * self.nz


def grid3(nx, ny, nz):
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx].astype(np.float64)
    return x, y, z


def profile3(x, y, z, xc, yc, zc, R, D, periods=(None, None, None)):
    """0.5 + 0.5 tanh(2 (R - r) / D) with r the Euclidean (minimum-image on
    the periodic axes) distance to (xc, yc, zc)."""
    d = []
    for a, c, per in ((x, xc, periods[0]), (y, yc, periods[1]), (z, zc, periods[2])):
        v = a - c
        if per:
            v = (v + per / 2) % per - per / 2
        d.append(v)
    r = np.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2)
    return 0.5 + 0.5 * np.tanh(2.0 * (R - r) / D)


def random_lattice3(nx, ny, nz, seed, edges=None, solids=("sphere",), u_amp=0.01, rho=(1.0, 3.0, 1.0)):
    """Random drops of fluids 1 and 2, random solids (a sphere, a pillar, an
    L-shaped concave corner), small random velocity, random admissible
    tensions and angles: reaches every branch of the 3D wall rules."""
    rng = np.random.default_rng(seed)
    if edges is None:
        edges = (PERIODIC, PERIODIC, WETTING, NEUTRAL, PERIODIC, PERIODIC)
    x, y, z = grid3(nx, ny, nz)
    mask = np.zeros((nz, ny, nx), np.uint8)
    for kind in solids:
        kv = int(rng.integers(1, 3))
        if kind == "sphere":
            c = [rng.uniform(0.3 * n, 0.7 * n) for n in (nx, ny, nz)]
            R = rng.uniform(2.5, max(3.0, min(nx, ny, nz) / 5))
            mask[((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) <= R * R] = kv
        elif kind == "pillar":
            px, py = int(rng.integers(2, nx - 2)), int(rng.integers(2, ny - 2))
            mask[:, py, px] = kv
        elif kind == "corner":
            px, py, pz = int(rng.integers(2, nx - 6)), int(rng.integers(2, ny - 6)), int(rng.integers(2, nz - 4))
            mask[pz:pz + 3, py:py + 4, px:px + 2] = kv
            mask[pz:pz + 3, py:py + 2, px:px + 4] = kv
    per = tuple(n if edges[2 * a] == PERIODIC else None for a, n in enumerate((nx, ny, nz)))
    c1 = np.zeros((nz, ny, nx))
    c2 = np.zeros((nz, ny, nx))
    for i in range(int(rng.integers(2, 5))):
        c = [rng.uniform(0, n) for n in (nx, ny, nz)]
        R = rng.uniform(2.5, max(3.0, min(nx, ny, nz) / 4))
        prof = profile3(x, y, z, *c, R, 4.0, per)
        if i % 2 == 0:
            c1 = np.maximum(c1, prof)
        else:
            c2 = np.maximum(c2, prof)
    s = c1 + c2
    over = s > 1
    c1[over] /= s[over]
    c2[over] /= s[over]
    c1[mask > 0] = 0
    c2[mask > 0] = 0
    u = [u_amp * rng.standard_normal((nz, ny, nx)) for _ in range(3)]
    for a in u:
        a[mask > 0] = 0
    sigma = tuple(rng.uniform(0.8e-3, 1.5e-3, 3))
    th13, th23 = rng.uniform(40, 140, 2)
    try:
        th12 = theta12_from(*sigma, th13, th23)
    except ValueError:
        th13, th23 = 90.0, 90.0
        th12 = theta12_from(*sigma, th13, th23)
    P = params(sigma=sigma, theta=(th12, th13, th23), rho=rho,
               nu=tuple(rng.uniform(0.05, 0.15, 3)), mobility=float(rng.uniform(0.05, 0.15)),
               D=float(rng.choice([3.0, 4.0, 5.0])), tau=tuple(rng.uniform(0.7, 1.0, 2)), g=(0.0, -1e-6))
    return Workload3(f"random3_{nx}x{ny}x{nz}_s{seed}", nx, ny, nz, tuple(edges), mask, P, c1, c2, *u)


def drops3d_on_wall(nx=128, ny=64, nz=128, R=16.0, theta=(60.0, 90.0, 120.0), sigma=1e-3, seed=1710):
    """The 3D counterpart of the two-drop wetting case, tiled: hemispherical
    drops of fluid 1 and fluid 2 (radius R) every 2.5 R along x and z on a
    wetting bottom wall (y-), neutral top wall, periodic in x and z, in fluid
    3; rho = 1, nu = 0.1, equal tensions, angles (theta_12, theta_13,
    theta_23), mobility 0.1, D = 4."""
    x, y, z = grid3(nx, ny, nz)
    c1 = np.zeros((nz, ny, nx))
    c2 = np.zeros((nz, ny, nx))
    step = 2.5 * R
    for iz, zc in enumerate(np.arange(step / 2, nz, step)):
        for ix, xc in enumerate(np.arange(step / 2, nx, step)):
            prof = profile3(x, y, z, xc, -0.5, zc, R, 4.0, (nx, None, nz))
            if (ix + iz) % 2 == 0:
                c1 = np.maximum(c1, prof)
            else:
                c2 = np.maximum(c2, prof)
    P = params(sigma=(sigma, sigma, sigma), theta=theta, rho=(1.0, 1.0, 1.0), nu=(0.1, 0.1, 0.1),
               mobility=0.1, D=4.0)
    zero = np.zeros((nz, ny, nx))
    return Workload3(f"drops3d_on_wall_{nx}x{ny}x{nz}", nx, ny, nz,
                     (PERIODIC, PERIODIC, WETTING, NEUTRAL, PERIODIC, PERIODIC),
                     np.zeros((nz, ny, nx), np.uint8), P, c1, c2, zero, zero.copy(), zero.copy())
