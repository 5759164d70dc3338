"""Lattice-level invariants of the oracle's full time step.

Conservation (Eqs. 1a, 13a, 44 conserve each order parameter), exact fixed
points, Galilean translation of a uniform state and the symmetries of the
D2Q9 update.  A wrong streaming direction, bounce-back slot, neighbour index
or ghost rule breaks at least one of these.
"""
import numpy as np
import pytest

import workloads as W
from oracle import OracleLattice


def _lattice(w):
    L = OracleLattice(w.nx, w.ny, w.edges, w.mask, w.params)
    L.set_fields(w.c1, w.c2, w.ux, w.uy, w.p)
    return L


@pytest.mark.parametrize("seed,edges,solids", [
    (1, (0, 0, 1, 2), ("disc",)),
    (2, (1, 2, 1, 1), ("pillar", "corner")),
    (3, (0, 0, 0, 0), ("disc", "pillar", "corner")),
    (4, (2, 1, 2, 1), ()),
])
def test_mass_of_each_component_is_conserved(seed, edges, solids):
    w = W.random_lattice(40, 30, seed, edges=edges, solids=solids)
    L = _lattice(w)
    m0 = L.mass()
    L.step(200)
    m1 = L.mass()
    assert np.all(np.abs(m1 - m0) <= 1e-12 * np.abs(m0).max())


@pytest.mark.parametrize("edges", [(0, 0, 0, 0), (0, 0, 2, 2), (2, 2, 2, 2)])
def test_uniform_rest_state_is_a_fixed_point(edges):
    nx, ny = 12, 10
    prm = W.params(sigma=(1.2e-3, 0.9e-3, 1.1e-3), rho=(2.0, 3.0, 1.0))
    L = OracleLattice(nx, ny, edges, None, prm)
    c1 = np.full((ny, nx), 0.3)
    c2 = np.full((ny, nx), 0.45)
    z = np.zeros((ny, nx))
    L.set_fields(c1, c2, z, z)
    s0 = L.state()
    L.step(50)
    assert np.abs(L.state() - s0).max() < 2e-14  # round-off of the BGK update


def test_uniform_flow_stays_uniform():
    """Galilean translation: uniform c and u on a periodic lattice are steady."""
    nx, ny = 9, 7
    prm = W.params(sigma=(1.2e-3, 0.9e-3, 1.1e-3), rho=(2.0, 3.0, 1.0))
    L = OracleLattice(nx, ny, (0, 0, 0, 0), None, prm)
    c1, c2 = np.full((ny, nx), 0.2), np.full((ny, nx), 0.5)
    L.set_fields(c1, c2, np.full((ny, nx), 0.04), np.full((ny, nx), -0.03))
    L.step(100)
    f = L.fields()
    for k, v in (("c1", 0.2), ("c2", 0.5), ("ux", 0.04), ("uy", -0.03)):
        assert np.abs(f[k] - v).max() < 1e-14


def _mirror_workload(nx, ny, edges):
    x, y = W.grid(nx, ny)
    xm = (nx - 1) / 2
    c1 = W.profile(x, y, xm - 7, 3, 6, 4.0) + W.profile(x, y, xm + 7, 3, 6, 4.0)
    c2 = W.profile(x, y, xm, ny - 6, 5, 4.0)
    ux = 0.01 * np.sin(2 * np.pi * (x - xm) / nx) * np.exp(-((y - ny / 2) / 5) ** 2)
    uy = 0.01 * np.cos(2 * np.pi * (x - xm) / nx)
    mask = np.zeros((ny, nx), np.uint8)
    mask[ny // 2 - 2:ny // 2 + 2, int(xm) - 1:int(xm) + 2 + (nx % 2 == 0)] = 1
    prm = W.params(sigma=(1.3e-3, 1.0e-3, 1.1e-3), theta=(W.theta12_from(1.3e-3, 1.0e-3, 1.1e-3, 70, 100), 70, 100),
                   rho=(3.0, 2.0, 1.0), g=(0.0, -1e-6))
    return c1, c2, ux, uy, mask, prm


@pytest.mark.parametrize("nx", [24, 25])
def test_mirror_symmetry_in_x(nx):
    """x -> nx-1-x maps the problem to itself; c stays even, u_x odd."""
    ny = 20
    c1, c2, ux, uy, mask, prm = _mirror_workload(nx, ny, None)
    L = OracleLattice(nx, ny, (0, 0, 1, 2), mask, prm)
    L.set_fields(c1, c2, ux, uy)
    L.step(150)
    f = L.fields()
    for k in ("c1", "c2", "uy", "p", "mu1", "rho"):
        assert np.abs(f[k] - f[k][:, ::-1]).max() < 1e-13, k
    assert np.abs(f["ux"] + f["ux"][:, ::-1]).max() < 1e-13


def test_transpose_symmetry():
    """Swapping x and y on a square lattice with the same wall on every side
    commutes with the update (fixes the y half of the direction table)."""
    n = 22
    x, y = W.grid(n, n)
    c1 = W.profile(x, y, 5, 8, 6, 4.0)
    c2 = W.profile(x, y, 15, 13, 5, 4.0)
    ux = 0.01 * np.sin(x / 3.0) * np.cos(y / 4.0)
    uy = -0.005 * np.cos(x / 5.0)
    prm = W.params(sigma=(1.3e-3, 1.0e-3, 1.1e-3), theta=(W.theta12_from(1.3e-3, 1.0e-3, 1.1e-3, 70, 100), 70, 100),
                   rho=(3.0, 2.0, 1.0))
    mask = np.zeros((n, n), np.uint8)
    mask[10:13, 16:18] = 2
    A = OracleLattice(n, n, (1, 1, 1, 1), mask, prm)
    A.set_fields(c1, c2, ux, uy)
    B = OracleLattice(n, n, (1, 1, 1, 1), mask.T.copy(), prm)
    B.set_fields(c1.T, c2.T, uy.T, ux.T)
    A.step(100)
    B.step(100)
    fa, fb = A.fields(), B.fields()
    for k in ("c1", "c2", "p", "rho", "mu2"):
        assert np.abs(fa[k] - fb[k].T).max() < 1e-13, k
    assert np.abs(fa["ux"] - fb["uy"].T).max() < 1e-13
    assert np.abs(fa["uy"] - fb["ux"].T).max() < 1e-13


def test_absent_phase_stays_absent():
    """Sec. II.B consistency: a phase absent at t = 0 never appears (Eq. 32).
    With c3 = 0 the sum c1 + c2 only feels the weak compressibility of the
    flow (here |u| ~ 1e-6 while the interface relaxes), so c3 stays at that
    level; a ghost offset that broke Eq. 31 at the wetting walls would put
    O(4/D c1 c2 cos) ~ 1e-1 into c3 at the first step."""
    nx, ny = 6, 40
    x, y = W.grid(nx, ny)
    c1 = 0.5 + 0.5 * np.tanh(2 * (y - 20) / 4.0)
    z = np.zeros((ny, nx))
    prm = W.params(sigma=(1e-3, 1e-3, 1e-3), theta=(60.0, 70.0, 110.0))
    L = OracleLattice(nx, ny, (0, 0, 1, 1), None, prm)
    L.set_fields(c1, 1 - c1, z, z)
    L.step(300)
    f = L.fields()
    assert np.abs(f["uy"]).max() < 1e-5
    assert np.abs(f["c3"]).max() < 1e-4
