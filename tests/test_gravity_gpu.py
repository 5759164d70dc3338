"""Gravity (body force G = rho g in Eq. 11b): FP64 parity with the oracle on a
puddle lattice, and the equilibrium puddle thickness of Eq. 48 on the paper's
set-up with gravity (600 x 150, drops of density 10 and 5 in a fluid of
density 1, sigma = 0.1, theta_13 = theta_23 = 90 deg).

Eq. 48 holds where gravity dominates (drop size well above the capillary
length) and the puddles are not confined by the periodic domain: g = 2e-5 to
4e-5 here (at 8e-5 the density-10 puddle would be longer than half the
domain).  Gravity acts on all three fluids, so the capillary length takes the
density difference to the ambient fluid, rho_l - rho_3 (buoyancy).  Measured
on GB300 after 60000 steps (FP32): H = 23.58 (Eq. 48: 23.57) and 34.37 (35.36)
at g = 4e-5, 32.6 (33.3) for the density-10 drop at g = 2e-5.
"""
import numpy as np
import pytest

import workloads as W
from oracle import OracleLattice

from test_parity_gpu import assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_09534_gb300 import build
    build.build()
    import paper_1710_09534_gb300 as T
    return T


def test_gravity_parity_fp64(T):
    w = W.puddles(4e-4, nx=120, ny=48, R=14.0)
    L = T.lattice_from_workload(w, "fp64")
    O = OracleLattice(w.nx, w.ny, w.edges, w.mask, w.params)
    O.set_fields(w.c1, w.c2, w.ux, w.uy, w.p)
    O.param_dict = dict(w.params)
    L.step(500)
    O.step(500)
    assert_parity(L, O, what="puddle with gravity")


def test_puddle_thickness_follows_eq48(T):
    gs = (0.0, 2e-5, 4e-5)
    B = T.Batch("fp32", max_lattices=len(gs))
    lats = []
    for g in gs:
        L = T.lattice_from_workload(W.puddles(g), "fp32")
        B.add(L)
        lats.append(L)
    B.step(60000)
    B.synchronize()
    H = {}
    for g, L in zip(gs, lats):
        B.remove(L)
        assert L.diagnostics()["nonfinite"] == 0
        (_, h1, _, _), = L.contact_angles(1)
        (_, h2, _, _), = L.contact_angles(2)
        H[g] = (h1, h2)
    # no gravity: a 90-degree cap keeps its radius as height
    assert abs(H[0.0][0] - 60.0) < 1.5 and abs(H[0.0][1] - 60.0) < 1.5
    # thickness falls with g, the lighter drop stays thicker
    assert H[0.0][0] > H[2e-5][0] > H[4e-5][0]
    assert H[4e-5][1] > H[4e-5][0]
    eq48 = lambda rho_l, g: W.puddle_thickness(0.1, rho_l - 1.0, g, 90.0)
    assert abs(H[4e-5][0] / eq48(10.0, 4e-5) - 1) < 0.03
    assert abs(H[4e-5][1] / eq48(5.0, 4e-5) - 1) < 0.05
    assert abs(H[2e-5][0] / eq48(10.0, 2e-5) - 1) < 0.05
