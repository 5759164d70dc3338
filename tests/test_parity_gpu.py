"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

FP64 storage/arithmetic must match the oracle within 1e-12 relative max-norm
on every macroscopic field and on every plane of the raw state (27
distributions and the 4 c_i u planes of Eq. 19); the norms and their scale
floors are defined in parity.py.
"""
import numpy as np
import pytest

import workloads as W
from oracle import OracleLattice
from parity import FIELDS, TOL64, field_errors, floors, is_mrt, relnorm, state_error as _plane_state_error  # noqa: F401

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


def pair(T, w, precision="fp64"):
    L = T.lattice_from_workload(w, precision)
    O = OracleLattice(w.nx, w.ny, w.edges, w.mask, w.params)
    O.set_fields(w.c1, w.c2, w.ux, w.uy, w.p)
    O.param_dict = dict(w.params)
    return L, O


def assert_parity(L, O, tol=TOL64, what=""):
    """Every field and every raw-state plane of L within `tol` of the oracle."""
    errs = field_errors(L.fields(), O.fields(), O.param_dict)
    bad = {k: v for k, v in errs.items() if not v < tol}
    assert not bad, f"{what} field errors above {tol}: {bad}"
    se, q = _plane_state_error(L.state(), O.state(), is_mrt(O.param_dict))
    assert se < tol, f"{what} raw state error {se:.3e} in plane {q}"


def test_binary_drops_128x64_fp64_1000_and_2000_steps(T):
    """The 128x64 two-drop wetting case, checked after 1000 and 2000 steps."""
    w = W.binary_drops_on_wall()
    L, O = pair(T, w)
    for _ in range(2):
        L.step(1000)
        O.step(1000)
        assert_parity(L, O, what="128x64")


@pytest.mark.parametrize("nx,ny,seed,edges,solids,lid_u", [
    (67, 45, 11, (0, 0, 1, 2), ("disc",), 0.0),                      # ragged, wetting bottom
    (33, 29, 12, (1, 2, 2, 1), ("pillar", "corner"), 0.0),           # walls on all sides
    (70, 40, 13, (0, 0, 0, 0), ("disc", "pillar", "corner"), 0.0),  # fully periodic + solids
    (64, 40, 14, (0, 0, 1, 3), ("corner",), 0.02),                   # velocity lid
    (37, 21, 15, (2, 1, 1, 3), ("pillar",), 0.01),                   # lid + side walls (corners)
    (130, 70, 16, (0, 0, 2, 1), ("disc", "disc"), 0.0),
])
def test_random_lattices_fp64(T, nx, ny, seed, edges, solids, lid_u):
    w = W.random_lattice(nx, ny, seed, edges=edges, solids=solids, lid_u=lid_u)
    L, O = pair(T, w)
    L.step(150)
    O.step(150)
    assert_parity(L, O, what=w.name)


def test_smallest_lattices(T):
    for nx, ny, edges in ((3, 3, (0, 0, 0, 0)), (4, 6, (0, 0, 1, 3)), (5, 3, (1, 1, 0, 0))):
        w = W.random_lattice(nx, ny, 7, edges=edges, solids=(), lid_u=0.01 if edges[3] == 3 else 0.0)
        L, O = pair(T, w)
        L.step(20)
        O.step(20)
        assert_parity(L, O, what=f"{nx}x{ny}")


def test_zero_steps_is_identity(T):
    w = W.random_lattice(40, 30, 3)
    L, O = pair(T, w)
    L.step(0)
    assert_parity(L, O, what="init")


def test_compound_drop_shear_512x256_fp64(T):
    """Full-size 512x256 lid-driven compound drop: every node compared."""
    w = W.compound_drop_shear()
    L, O = pair(T, w)
    L.step(30)
    O.step(30)
    assert_parity(L, O, what="512x256 shear")


def test_cylinder_impact_fp64(T):
    w = W.compound_drop_on_cylinder(nx=256, ny=512, R_cyl=30, R_core=15, R_shell=25, We=10.0, theta=30.0)
    L, O = pair(T, w)
    L.step(60)
    O.step(60)
    assert_parity(L, O, what="cylinder")


def test_tiled_drops_2048_fp64_full_size(T):
    """The 2048x2048 benchmark lattice, two steps, every node compared."""
    w = W.tiled_drops()
    L, O = pair(T, w)
    L.step(2)
    O.step(2)
    assert_parity(L, O, what="2048^2")


def test_mass_diagnostics_fp64(T):
    w = W.random_lattice(80, 50, 21, edges=(0, 0, 1, 2), solids=("disc", "corner"))
    L, O = pair(T, w)
    d0 = L.diagnostics()
    L.step(200)
    O.step(200)
    d1 = L.diagnostics()
    assert d1["nonfinite"] == 0
    assert np.allclose(d1["mass"], O.mass(), rtol=1e-13, atol=1e-12)
    assert np.allclose(d1["mass"], d0["mass"], rtol=1e-12)  # conserved with walls


def test_checkpoint_resume_is_bit_identical(T):
    w = W.random_lattice(50, 40, 5, edges=(0, 0, 1, 3), solids=("pillar",), lid_u=0.01)
    A = T.lattice_from_workload(w)
    A.step(40)
    blob = A.export_state()
    A.step(25)
    B = T.lattice_from_workload(w)
    B.import_state(blob)
    B.step(25)
    assert np.array_equal(A.state(), B.state())


def test_deterministic(T):
    w = W.random_lattice(70, 40, 9, solids=("disc",))
    A = T.lattice_from_workload(w)
    B = T.lattice_from_workload(w)
    A.step(50)
    B.step(50)
    assert np.array_equal(A.state(), B.state())


def test_error_codes(T):
    w = W.random_lattice(20, 20, 1)
    L = T.Lattice(20, 20, "fp64", w.edges)
    with pytest.raises(T.TlbError) as e:
        L.step(1)
    assert e.value.code == T.ESTATE
    bad = dict(w.params)
    bad["theta12_deg"] = bad["theta12_deg"] + 20.0
    with pytest.raises(T.TlbError) as e:
        L.set_params(bad)
    assert e.value.code == T.EINVAL and "Eq. 39" in str(e.value)
    L.set_params(w.params)
    L.set_fields(w.c1, w.c2, w.ux, w.uy)
    with pytest.raises(T.TlbError) as e:
        L.set_geometry(np.full((20, 20), 7, np.uint8))
    assert e.value.code == T.EINVAL


def test_sync_deadline(T):
    """tlb_sync returns TLB_ETIMEOUT when work is still queued at the deadline."""
    w = W.tiled_drops(1024, 1024)
    L = T.lattice_from_workload(w)
    L.sync()
    L.step(200)
    with pytest.raises(T.TlbError) as e:
        L.sync(0)
    assert e.value.code == T.ETIMEOUT
    assert L.sync(-1) == 0


def test_nonfinite_state_is_reported(T):
    w = W.random_lattice(30, 20, 2)
    L = T.lattice_from_workload(w)
    c1 = w.c1.copy()
    c1[5, 5] = np.nan
    L.set_fields(c1, w.c2, w.ux, w.uy)
    d = L.diagnostics()
    assert d["rc"] == T.EUNSTABLE and d["nonfinite"] >= 1


def test_contact_line_diagnostic_fp64(T):
    """tlb_contact_angles (FP64 on the device) against the oracle's measurement
    of theta_n = 2 atan(2 H_d / L_s) (Sec. III.A) on the oracle's own fields."""
    import oracle
    w = W.binary_drops_on_wall()
    L, O = pair(T, w)
    L.step(1000)
    O.step(1000)
    fo = O.fields()
    for comp in (1, 2):
        got = L.contact_angles(comp)
        ref = oracle.drop_geometry(fo[f"c{comp}"])
        assert len(got) == len(ref) == 1
        (Ls, Hd, th, xm), (Ls0, Hd0, xm0) = got[0], ref[0]
        assert abs(Ls - Ls0) < 1e-9 * Ls0 and abs(Hd - Hd0) < 1e-9 * Hd0
        assert abs(th - oracle.contact_angle_deg(fo[f"c{comp}"])[0]) < 1e-8
        assert abs(xm - xm0) < 1e-9 * w.nx


def test_contact_line_diagnostic_counts_drops_across_the_periodic_edge(T):
    nx, ny = 96, 32
    x, y = W.grid(nx, ny)
    c1 = np.maximum(W.profile(x, y, 4.0, -0.5, 10, 4.0, period_x=nx),
                    W.profile(x, y, 50.0, -0.5, 8, 4.0, period_x=nx))
    z = np.zeros((ny, nx))
    w = W.Workload("two", nx, ny, (0, 0, 1, 2), np.zeros((ny, nx), np.uint8), W.params(), c1, z, z, z)
    L = T.lattice_from_workload(w)
    got = sorted(L.contact_angles(1), key=lambda r: r[3])
    import oracle
    ref = sorted(oracle.drop_geometry(L.fields()["c1"]), key=lambda r: r[2])
    assert len(got) == len(ref) == 2
    for (Ls, Hd, _, xm), (Ls0, Hd0, xm0) in zip(got, ref):
        assert abs(Ls - Ls0) < 1e-12 * Ls0 and abs(Hd - Hd0) < 1e-12 * Hd0 and abs(xm - xm0) < 1e-9
