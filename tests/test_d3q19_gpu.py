"""The D3Q19 form on the GPU (through the C ABI) against the 3D FP64 oracle:
every field and every raw-state plane within 1e-12 (the norms of parity.py,
with the D3Q19 plane groups), on random lattices with every kind of edge and
solid, drops on a wetting wall, the smallest lattices, a state that reaches
a ragged tail of blocks in x, and a full-size lattice of the benchmark."""
import numpy as np
import pytest

import workloads as W
from oracle import OracleLattice3D
from parity import BOUNDS, assert_oracle_parity3

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
    L = T.lattice3_from_workload(w, precision=precision)
    O = OracleLattice3D(w.nx, w.ny, w.nz, w.edges, w.mask, w.params)
    O.set_fields(w.c1, w.c2, w.ux, w.uy, w.uz, w.p)
    return L, O


@pytest.mark.parametrize("shape,seed,edges,solids", [
    ((20, 18, 16), 1, (0, 0, 1, 2, 0, 0), ("sphere",)),
    ((17, 13, 11), 2, (1, 2, 1, 1, 2, 1), ("pillar", "corner")),
    ((24, 12, 14), 3, (0, 0, 0, 0, 0, 0), ("sphere", "corner")),
    ((131, 9, 7), 4, (2, 1, 0, 0, 1, 2), ("pillar",)),       # a ragged second block in x
    ((12, 20, 9), 5, (0, 0, 2, 1, 0, 0), ("sphere", "sphere")),
])
def test_random_lattices_fp64(T, shape, seed, edges, solids):
    w = W.random_lattice3(*shape, seed, edges=edges, solids=solids)
    L, O = pair(T, w)
    for n in (1, 30):
        L.step(n)
        O.step(n)
        assert_oracle_parity3(L, O, w.params, what=f"{w.name} after {n}")


@pytest.mark.parametrize("seed,edges", [(11, (0, 0, 1, 2, 1, 1)), (12, (2, 2, 0, 0, 1, 2))])
def test_uniform_property_update_with_solids_and_body_force(T, seed, edges):
    """Equal densities and viscosities select the update without grad rho,
    F_a and lap mu; walls on several faces, a sphere, a corner, gx and gy."""
    w = W.random_lattice3(19, 15, 13, seed, edges=edges, solids=("sphere", "corner"))
    w.params.update(rho1=1.0, rho2=1.0, rho3=1.0, nu1=0.1, nu2=0.1, nu3=0.1, gx=3e-6, gy=-2e-6)
    L, O = pair(T, w)
    for n in (1, 40):
        L.step(n)
        O.step(n)
        assert_oracle_parity3(L, O, w.params, what=f"{w.name} uniform after {n}")


def test_drops_on_a_wetting_wall_300_steps(T):
    w = W.drops3d_on_wall(48, 24, 40, R=10.0)
    L, O = pair(T, w)
    L.step(300)
    O.step(300)
    assert_oracle_parity3(L, O, w.params, what=w.name)


def test_drops_1000_steps_with_density_contrast(T):
    """1000 steps of a small drops-on-wall lattice with fluid 2 three times as
    dense and the viscosities apart (the general update), against the oracle."""
    w = W.drops3d_on_wall(40, 20, 40, R=8.0)
    w.params.update(rho2=3.0, nu1=0.08, nu2=0.12, nu3=0.1, gy=-1e-6)
    L, O = pair(T, w)
    L.step(1000)
    O.step(1000)
    assert_oracle_parity3(L, O, w.params, what=f"{w.name} general, 1000 steps")


def test_zero_steps_and_smallest_lattices(T):
    for shape, edges in (((3, 3, 3), (0,) * 6), ((4, 5, 3), (1, 2, 0, 0, 2, 2)), ((3, 4, 6), (0, 0, 1, 2, 0, 0))):
        w = W.random_lattice3(*shape, 7, edges=edges, solids=())
        L, O = pair(T, w)
        assert_oracle_parity3(L, O, w.params, what=f"{shape} init")
        L.step(12)
        O.step(12)
        assert_oracle_parity3(L, O, w.params, what=f"{shape}")


def test_mass_diagnostics_fp64(T):
    w = W.random_lattice3(22, 16, 14, 8, edges=(0, 0, 1, 2, 1, 1), solids=("sphere", "corner"))
    L, O = pair(T, w)
    d0 = L.diagnostics()
    L.step(60)
    O.step(60)
    d1 = L.diagnostics()
    assert d1["nonfinite"] == 0 and d1["rc"] == 0
    assert np.allclose(d1["mass"], O.mass(), rtol=1e-13, atol=1e-11)
    assert np.allclose(d1["mass"][:2], d0["mass"][:2], rtol=1e-12)


def test_error_codes(T):
    w = W.random_lattice3(8, 8, 8, 9, solids=())
    L = T.Lattice3D(8, 8, 8, w.edges)
    with pytest.raises(T.TlbError) as e:
        L.step(1)
    assert e.value.code == T.ESTATE
    for bad in (dict(collision=1.0), dict(lid_u=0.01), dict(theta12_deg=w.params["theta12_deg"] + 20)):
        with pytest.raises(T.TlbError) as e:
            L.set_params(dict(w.params, **bad))
        assert e.value.code == T.EINVAL
    with pytest.raises(T.TlbError) as e:
        T.Lattice3D(8, 8, 8, (0, 1, 0, 0, 0, 0))  # periodic edge paired with a wall
    assert e.value.code == T.EINVAL


def test_full_size_benchmark_lattice_fp64(T):
    """The benchmark's 3D lattice, two steps, every node compared."""
    w = W.drops3d_on_wall(192, 96, 192)
    L, O = pair(T, w)
    L.step(2)
    O.step(2)
    assert_oracle_parity3(L, O, w.params, what=w.name)


# FP32 storage: the 2D FP32 bounds against the oracle (uz as ux)
BOUNDS3_FP32 = dict(BOUNDS["fp32"], uz=BOUNDS["fp32"]["ux"])


def fp32_errors(fg, fo):
    out = {}
    for k, (kind, bound) in BOUNDS3_FP32.items():
        err = float(np.abs(fg[k] - fo[k]).max())
        if kind == "rel":
            err /= max(float(np.abs(fo[k]).max()), 1e-12)
        out[k] = (err, bound)
    return out


@pytest.mark.parametrize("shape,seed,edges,solids,steps", [
    ((20, 18, 16), 21, (0, 0, 1, 2, 0, 0), ("sphere",), 200),
    ((17, 13, 11), 22, (1, 2, 1, 1, 2, 1), ("pillar", "corner"), 120),
    ((131, 9, 7), 24, (2, 1, 0, 0, 1, 2), ("pillar",), 60),
])
def test_fp32_storage_within_bounds_of_the_oracle(T, shape, seed, edges, solids, steps):
    w = W.random_lattice3(*shape, seed, edges=edges, solids=solids)
    L, O = pair(T, w, "fp32")
    L.step(steps)
    O.step(steps)
    bad = {k: v for k, v in fp32_errors(L.fields(), O.fields()).items() if not v[0] < v[1]}
    assert not bad, f"{w.name} fp32 after {steps}: {bad}"


def test_fp32_drops_500_steps_within_bounds_and_mass_conserved(T):
    w = W.drops3d_on_wall(48, 24, 40, R=10.0)
    L, O = pair(T, w, "fp32")
    m0 = np.array(L.diagnostics()["mass"])
    L.step(500)
    O.step(500)
    bad = {k: v for k, v in fp32_errors(L.fields(), O.fields()).items() if not v[0] < v[1]}
    assert not bad, f"{w.name} fp32: {bad}"
    m1 = np.array(L.diagnostics()["mass"])
    drift = np.abs(m1[:2] - m0[:2]) / np.abs(m0[:2])
    assert (drift < 1e-10).all(), drift
    # the raw state (rest populations as hi + lo) against the oracle's
    assert np.abs(L.state() - O.state()).max() < BOUNDS3_FP32["c1"][1]


def test_fp32_and_fp64_lattices_coexist(T):
    """An FP32 and an FP64 lattice stepped alternately on one stream keep
    their own results (each equals a lattice of its precision stepped alone)."""
    w = W.random_lattice3(16, 12, 10, 25, solids=("sphere",))
    a32, a64 = T.lattice3_from_workload(w, precision="fp32"), T.lattice3_from_workload(w)
    b32, b64 = T.lattice3_from_workload(w, precision="fp32"), T.lattice3_from_workload(w)
    for _ in range(5):
        a32.step(7)
        a64.step(7)
    b32.step(35)
    b64.step(35)
    assert np.array_equal(a32.state(), b32.state())
    assert np.array_equal(a64.state(), b64.state())
