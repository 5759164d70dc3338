"""Pins of the oracle's per-node formulas against what the paper and algebra fix.

Each test checks an oracle function against an independent route to the same
quantity (a different equation of the paper, a derivation chain, a moment
identity of the lattice), never against a retyped copy of the same formula.
"""
import math

import numpy as np
import pytest

RNG = np.random.default_rng(20171026)


def test_d2q9_table_matches_eq10(orc):
    """Eq. 10: axis directions at angles (k-1) pi/2, diagonals sqrt2 at (k-5) pi/2 + pi/4."""
    e, w, opp = orc.lattice_vectors()
    for k in range(1, 5):
        a = (k - 1) * math.pi / 2
        assert np.allclose(e[k], [math.cos(a), math.sin(a)], atol=1e-12)
    for k in range(5, 9):
        a = (k - 5) * math.pi / 2 + math.pi / 4
        assert np.allclose(e[k], [math.sqrt(2) * math.cos(a), math.sqrt(2) * math.sin(a)], atol=1e-12)
    assert np.allclose(w, [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    assert np.all(e[opp] == -e)
    # lattice isotropy up to 4th order with cs^2 = 1/3
    cs2 = 1.0 / 3.0
    assert abs(w.sum() - 1) < 1e-15
    assert np.allclose(np.einsum("k,ka,kb->ab", w, e, e), cs2 * np.eye(2))
    d = np.eye(2)
    t4 = np.einsum("k,ka,kb,kc,kd->abcd", w, e, e, e, e)
    iso = cs2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                      + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(t4, iso)


def test_lambdas_eq7_eq9(orc):
    s = (1.3e-3, 0.9e-3, 1.1e-3)
    lam = orc.lambdas(*s)
    # Eq. 7 inverted: sigma_ij = (lambda_i + lambda_j) / 2
    assert math.isclose((lam[0] + lam[1]) / 2, s[0], rel_tol=1e-14)
    assert math.isclose((lam[0] + lam[2]) / 2, s[1], rel_tol=1e-14)
    assert math.isclose((lam[1] + lam[2]) / 2, s[2], rel_tol=1e-14)
    # Eq. 9 harmonic form
    assert math.isclose(3.0 / lam[3], sum(1.0 / l for l in lam[:3]), rel_tol=1e-14)
    # equal tensions: lambda_i = lambda_T = sigma
    assert np.allclose(orc.lambdas(2e-3, 2e-3, 2e-3), 2e-3, rtol=1e-15)
    # one vanishing lambda: the continuous form of Eq. 9 gives 0
    assert orc.lambdas(2e-3, 1e-3, 1e-3)[3] == 0.0


def _dF(lam, c):
    """dF/dc_i of Eq. 5 with lambda = 0: lambda_i c_i (1 - c_i)(1 - 2 c_i)."""
    return lam * c * (1 - c) * (1 - 2 * c)


@pytest.mark.parametrize("trial", range(20))
def test_mu_eq8_equals_general_eq6(orc, trial):
    """Eq. 8 is Eq. 6 with lambda = 0 once c1 + c2 + c3 = 1 (Sec. II.A)."""
    s = RNG.uniform(0.5e-3, 2e-3, 3)
    lam = orc.lambdas(*s)
    if np.any(lam[:3] <= 0):
        pytest.skip("non-positive lambda")
    D = RNG.uniform(2, 8)
    c1, c2 = RNG.uniform(-0.1, 0.7, 2)
    c = np.array([c1, c2, 1 - c1 - c2])
    lap1, lap2 = RNG.normal(0, 0.05, 2)
    lap = np.array([lap1, lap2, -lap1 - lap2])
    mu = orc.chem_pot(lam, D, c1, c2, lap1, lap2)
    dF = _dF(lam[:3], c)
    eq6 = np.array([4 * lam[3] / D * sum((dF[i] - dF[j]) / lam[j] for j in range(3) if j != i)
                    - 0.75 * D * lam[i] * lap[i] for i in range(3)])
    assert np.allclose(mu, eq6, rtol=1e-11, atol=1e-15 * np.abs(eq6).max())


def test_sum_mu_over_lambda_vanishes(orc):
    """sum_i mu_i / lambda_i = 0 for Eq. 8 (consequence of Eqs. 3, 9)."""
    for _ in range(50):
        s = RNG.uniform(0.5e-3, 2e-3, 3)
        lam = orc.lambdas(*s)
        if np.any(lam[:3] <= 0):
            continue
        c1, c2 = RNG.uniform(0, 0.6, 2)
        mu = orc.chem_pot(lam, 4.0, c1, c2, *RNG.normal(0, 0.05, 2))
        scale = np.abs(mu / lam[:3]).max()
        assert abs((mu / lam[:3]).sum()) <= 1e-13 * scale


def _wall_tensions(s12, s13, s23, th12, th13, th23, sw1=0.37e-3):
    """Wall tensions consistent with Young's relation Eq. 38 (up to a constant)."""
    sw3 = sw1 + s13 * math.cos(math.radians(th13))
    sw2 = sw1 + s12 * math.cos(math.radians(th12))
    return sw1, sw2, sw3


def _g_from_matrix(lam, s12, s13, s23, sw, c):
    """g = A . dpsi_s/dc with A of Eq. 34 and psi_s of Eq. 27."""
    c1, c2, c3 = c
    l1, l2, l3 = lam[:3]
    A = 0.5 * np.array([
        [l1 / s12 * c2 / (1 - c1) + l1 / s13 * c3 / (1 - c1), -l1 / s12 * c1 / (1 - c2), -l1 / s13 * c1 / (1 - c3)],
        [-l2 / s12 * c2 / (1 - c1), l2 / s12 * c1 / (1 - c2) + l2 / s23 * c3 / (1 - c2), -l2 / s23 * c2 / (1 - c3)],
        [-l3 / s13 * c3 / (1 - c1), -l3 / s23 * c3 / (1 - c2), l3 / s13 * c1 / (1 - c3) + l3 / s23 * c2 / (1 - c3)]])
    dpsi = np.array([sw[i] * (6 * c[i] - 6 * c[i] ** 2) for i in range(3)])
    return A @ dpsi


@pytest.mark.parametrize("trial", range(12))
def test_wetting_ghost_follows_from_wall_energy(orc, trial):
    """Eq. 42 offsets equal dx * n.grad c_i from Eq. 29 with g = A dpsi/dc
    (Eqs. 27, 34), wall tensions from Young's relation (Eq. 38) and theta_12
    from the constraint Eq. 39: the whole derivation chain of Sec. II.B."""
    s12, s13, s23 = RNG.uniform(0.8e-3, 1.4e-3, 3)
    lam = orc.lambdas(s12, s13, s23)
    th13, th23 = RNG.uniform(35, 145, 2)
    cth12 = (s13 * math.cos(math.radians(th13)) - s23 * math.cos(math.radians(th23))) / s12
    if abs(cth12) > 1:
        pytest.skip("Eq. 39 has no solution")
    th12 = math.degrees(math.acos(cth12))
    sw = _wall_tensions(s12, s13, s23, th12, th13, th23)
    # the third Young relation then holds too
    assert math.isclose((sw[2] - sw[1]) / s23, math.cos(math.radians(th23)), rel_tol=1e-9)
    D = RNG.uniform(3, 6)
    c1, c2 = RNG.uniform(0.05, 0.55, 2)
    c = (c1, c2, 1 - c1 - c2)
    g = _g_from_matrix(lam, s12, s13, s23, sw, c)
    ndc = -g / (0.75 * lam[:3] * D)          # Eq. 29
    off = orc.wet_offset(math.cos(math.radians(th12)), math.cos(math.radians(th13)),
                         math.cos(math.radians(th23)), D, c1, c2)
    assert np.allclose(off, ndc, rtol=1e-9, atol=1e-17)
    # Eq. 31 and the Eq. 42 offsets summing to zero (c_ghost keeps c1+c2+c3 = 1)
    assert abs((g / lam[:3]).sum()) < 1e-12 * np.abs(g / lam[:3]).max()
    assert abs(off.sum()) < 1e-15


def test_wetting_g_vanishes_for_absent_phase(orc):
    """Eq. 32: g_i = 0 where c_i = 0, hence no ghost offset for an absent phase."""
    c12, c13, c23 = math.cos(1.0), math.cos(1.3), math.cos(1.7)
    for c1, c2 in ((0.0, 0.4), (0.3, 0.0), (0.45, 0.55)):
        off = orc.wet_offset(c12, c13, c23, 4.0, c1, c2)
        c3 = 1 - c1 - c2
        for ci, oi in zip((c1, c2, c3), off):
            if ci == 0.0:
                assert oi == 0.0


def test_wetting_reduces_to_two_phase_eq26(orc):
    """With c3 = 0 the ternary condition becomes the binary Eq. 26 for c = c1
    with cos(theta) = cos(theta_12) (Eqs. 36, 37)."""
    th12 = 55.0
    for c1 in np.linspace(0.05, 0.95, 7):
        off = orc.wet_offset(math.cos(math.radians(th12)), 0.3, -0.2, 4.0, c1, 1 - c1)
        binary = 4 * math.cos(math.radians(th12)) / 4.0 * (c1 - c1 * c1)
        assert math.isclose(off[0], binary, rel_tol=1e-12)
        assert math.isclose(off[1], -binary, rel_tol=1e-12)
        assert abs(off[2]) < 1e-17


def test_neutral_wall_angles_give_symmetric_ghost(orc):
    """All contact angles 90 deg: Eq. 42 reduces to Eq. 43 (no offset)."""
    c90 = math.cos(math.radians(90.0))
    off = orc.wet_offset(c90, c90, c90, 4.0, 0.3, 0.4)
    assert np.abs(off).max() < 1e-16


def test_eq39_holds_for_papers_shear_triple():
    """Sec. III.C prints (theta12, theta13, theta23) = (30, 68.53, 120) with equal
    tensions; Eq. 39 holds up to the rounding of 68.53."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
    t = g["shear_case_contact_angles"]
    r = math.cos(math.radians(t["theta12"])) - math.cos(math.radians(t["theta13"])) + math.cos(math.radians(t["theta23"]))
    assert abs(r) < t["eq39_tolerance"]
