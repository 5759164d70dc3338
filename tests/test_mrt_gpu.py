"""GPU parity of the MRT collision option against the oracle's MRT update.

The same bars as the BGK path: FP64 within 1e-12 relative max-norm on every
macroscopic field (with the per-field scale floors of the BGK parity tests)
and on the raw state; FP32 within the FP32 bounds and conserving each
component's mass.  Also: MRT with the BGK rates reproduces the GPU's BGK step,
batches run MRT members like lattices stepped alone, and a batch refuses to
mix collision models.
"""
import numpy as np
import pytest

import workloads as W
from oracle import OracleLattice

from test_parity_gpu import TOL64, assert_parity
from test_parity_fp32_gpu import check_fields

pytestmark = pytest.mark.gpu

RATES = [(1.3, 1.3), (1.6, 1.1)]


@pytest.fixture(scope="module")
def T():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_09534_gb300 import build
    build.build()
    import paper_1710_09534_gb300 as T
    return T


def mrt_workload(w, rates):
    w.params.update(collision=1.0, mrt_s_f=rates[0], mrt_s_g=rates[1])
    return w


def pair(T, w, precision="fp64"):
    L = T.lattice_from_workload(w, precision)
    O = OracleLattice(w.nx, w.ny, w.edges, w.mask, w.params)
    O.set_fields(w.c1, w.c2, w.ux, w.uy, w.p)
    O.param_dict = dict(w.params)
    return L, O


@pytest.mark.parametrize("rates", RATES)
@pytest.mark.parametrize("nx,ny,seed,edges,solids,lid_u", [
    (67, 45, 11, (0, 0, 1, 2), ("disc",), 0.0),                      # ragged, wetting bottom
    (33, 29, 12, (1, 2, 2, 1), ("pillar", "corner"), 0.0),           # walls on all sides
    (70, 40, 13, (0, 0, 0, 0), ("disc", "pillar", "corner"), 0.0),  # periodic + solids
    (64, 40, 14, (0, 0, 1, 3), ("corner",), 0.02),                   # velocity lid
    (37, 21, 15, (2, 1, 1, 3), ("pillar",), 0.01),                   # lid + side walls
    (260, 70, 16, (0, 0, 2, 1), ("disc", "disc"), 0.0),              # several interior tiles
])
def test_mrt_random_lattices_fp64(T, rates, nx, ny, seed, edges, solids, lid_u):
    w = mrt_workload(W.random_lattice(nx, ny, seed, edges=edges, solids=solids, lid_u=lid_u), rates)
    L, O = pair(T, w)
    L.step(150)
    O.step(150)
    assert_parity(L, O, what=f"MRT {rates} {w.name}")


def test_mrt_binary_drops_fp64_1000_steps(T):
    w = mrt_workload(W.binary_drops_on_wall(), (1.2, 1.4))
    L, O = pair(T, w)
    L.step(1000)
    O.step(1000)
    assert_parity(L, O, what="MRT 128x64")


def test_mrt_with_bgk_rates_is_the_bgk_step_on_gpu(T):
    w = W.random_lattice(64, 40, 14, edges=(0, 0, 1, 3), solids=("corner",), lid_u=0.02)
    w.params.update(tau1=0.85, tau2=0.85, nu1=0.1, nu2=0.1, nu3=0.1)
    A = T.lattice_from_workload(w, "fp64")
    w.params.update(collision=1.0, mrt_s_f=1 / 0.85, mrt_s_g=1 / (3 * 0.1 + 0.5))
    B = T.lattice_from_workload(w, "fp64")
    A.step(100)
    B.step(100)
    sa, sb = A.state(), B.state()
    assert float(np.abs(sa - sb).max() / np.abs(sa).max()) < TOL64


@pytest.mark.parametrize("seed,edges,lid_u", [(11, (0, 0, 1, 2), 0.0), (14, (0, 0, 1, 3), 0.02),
                                               (15, (2, 1, 1, 3), 0.01)])
def test_mrt_fp32_random_lattices(T, seed, edges, lid_u):
    w = mrt_workload(W.random_lattice(67, 45, seed, edges=edges, solids=("disc", "corner"), lid_u=lid_u),
                     (1.3, 1.3))
    L, O = pair(T, w, "fp32")
    L.step(150)
    O.step(150)
    check_fields(L, O, f"MRT fp32 {w.name}")


def test_mrt_fp32_mass_conserved(T):
    w = mrt_workload(W.binary_drops_on_wall(), (1.2, 1.4))
    L = T.lattice_from_workload(w, "fp32")
    m0 = np.array(L.diagnostics()["mass"])
    L.step(5000)
    d = L.diagnostics()
    assert d["nonfinite"] == 0
    assert np.all(np.abs(np.array(d["mass"]) - m0) <= 1e-6 * np.abs(m0).max())


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mrt_batch_members_match_alone(T, precision):
    tol = dict(fp64=1e-12, fp32=1e-5)[precision]
    ws = [mrt_workload(W.random_lattice(nx, ny, 200 + i, edges=e, solids=s, lid_u=u), (1.3, 1.3))
          for i, (nx, ny, e, s, u) in enumerate([(90, 50, (0, 0, 1, 2), ("disc",), 0.0),
                                                  (40, 70, (0, 0, 1, 3), ("corner",), 0.01),
                                                  (150, 33, (1, 2, 2, 1), ("pillar",), 0.0)])]
    alone = [T.lattice_from_workload(w, precision) for w in ws]
    mem = [T.lattice_from_workload(w, precision) for w in ws]
    B = T.Batch(precision, max_lattices=8)
    for L in mem:
        B.add(L)
    B.step(7)
    B.synchronize()
    for L in alone:
        L.step(7)
    for a, m in zip(alone, mem):
        sa, sm = a.state(), m.state()
        assert float(np.abs(sa - sm).max() / max(np.abs(sa).max(), 1e-6)) < tol


def test_mrt_parameter_errors_and_mixed_batch(T):
    w = W.random_lattice(30, 20, 1)
    L = T.lattice_from_workload(w, "fp64")
    for bad in (dict(collision=2.0), dict(collision=1.0, mrt_s_f=0.0, mrt_s_g=1.0),
                dict(collision=1.0, mrt_s_f=1.0, mrt_s_g=2.0)):
        p = dict(w.params)
        p.update(bad)
        with pytest.raises(T.TlbError) as e:
            L.set_params(p)
        assert e.value.code == T.EINVAL
    B = T.Batch("fp64", max_lattices=4)
    B.add(L)
    B.add(T.lattice_from_workload(mrt_workload(W.random_lattice(30, 20, 2), (1.3, 1.3)), "fp64"))
    with pytest.raises(T.TlbError) as e:
        B.step(1)
    assert e.value.code == T.EINVAL
