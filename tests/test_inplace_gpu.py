"""In-place (AA-pattern) streaming through the C ABI: one distribution buffer
instead of two.

The in-place update computes the same per-node arithmetic as the two-buffer
update (Eqs. 1a, 1b with the push of Eq. 44 written as reads and writes of
the node's own set of slots), so with FP64 it must match the two-buffer
result and the FP64 oracle within 1e-12 (relative max-norm with the field
floors of the FP64 parity tests), after even and odd step counts and across
several calls.  FP32 and 16-bit storage differ from the two-buffer update
only in the order in which the rest pair sums the moving differences, and
are held to the bounds of their own parity tests against the oracle.
"""
import numpy as np
import pytest

import workloads as W
from oracle import OracleLattice

pytestmark = pytest.mark.gpu

FIELDS = ("c1", "c2", "c3", "rho", "ux", "uy", "p", "mu1", "mu2", "mu3")
TOL64 = 1e-12

# edges, solids, lid velocity: every wall rule (periodic, wetting, neutral,
# lid, solid discs, pillars, concave corners)
SPECS = [((0, 0, 1, 2), ("disc",), 0.0), ((0, 0, 1, 3), ("corner",), 0.02), ((0, 0, 0, 0), ("pillar",), 0.0),
         ((1, 2, 2, 1), (), 0.0), ((0, 0, 1, 2), ("disc", "corner"), 0.0), ((2, 1, 1, 3), ("pillar",), 0.01)]


@pytest.fixture(scope="module")
def T():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_09534_gb300 import build
    build.build()
    import paper_1710_09534_gb300 as T
    return T


def floors(params):
    smax = max(params["sigma12"], params["sigma13"], params["sigma23"])
    mu = smax / params["D"]
    return dict(c1=1.0, c2=1.0, c3=1.0, rho=1.0, ux=1e-4, uy=1e-4, p=smax / 32, mu1=mu, mu2=mu, mu3=mu)


def relnorm(a, b, floor):
    return float(np.abs(a - b).max() / max(float(np.abs(b).max()), floor))


def field_errors(fa, fb, params):
    fl = floors(params)
    return {k: relnorm(fa[k], fb[k], fl[k]) for k in FIELDS}


def spec_workload(i, nx=67, ny=45, seed=300):
    edges, solids, lid = SPECS[i]
    return W.random_lattice(nx, ny, seed + i, edges=edges, solids=solids, lid_u=lid)


@pytest.mark.parametrize("steps", [1, 2, 7])
@pytest.mark.parametrize("spec", range(len(SPECS)))
def test_fp64_inplace_equals_two_buffer(T, spec, steps):
    """Fields, raw state and mass totals after `steps` steps, twice (so that a
    call may start on either parity of the total count)."""
    w = spec_workload(spec)
    A = T.lattice_from_workload(w, "fp64")
    B = T.lattice_from_workload(w, "fp64", inplace=True)
    for _ in range(2):
        A.step(steps)
        B.step(steps)
        errs = field_errors(B.fields(), A.fields(), w.params)
        bad = {k: v for k, v in errs.items() if not v < TOL64}
        assert not bad, f"spec {spec}, {steps} steps: {bad}"
        sa, sb = A.state(), B.state()
        assert np.abs(sb - sa).max() <= TOL64 * max(float(np.abs(sa).max()), 1e-6)
        ma, mb = np.array(A.diagnostics()["mass"]), np.array(B.diagnostics()["mass"])
        assert np.all(np.abs(mb - ma) <= 1e-12 * np.abs(ma))


@pytest.mark.parametrize("seed,edges,lid_u,mrt", [(11, (0, 0, 1, 2), 0.0, None), (14, (0, 0, 1, 3), 0.02, None),
                                                   (15, (2, 1, 1, 3), 0.01, None), (14, (0, 0, 1, 3), 0.02, (1.3, 1.3))])
def test_fp64_inplace_matches_oracle(T, seed, edges, lid_u, mrt):
    w = W.random_lattice(67, 45, seed, edges=edges, solids=("disc", "corner"), lid_u=lid_u)
    if mrt:
        w.params.update(collision=1.0, mrt_s_f=mrt[0], mrt_s_g=mrt[1])
    L = T.lattice_from_workload(w, "fp64", inplace=True)
    O = OracleLattice(w.nx, w.ny, w.edges, w.mask, w.params)
    O.set_fields(w.c1, w.c2, w.ux, w.uy, w.p)
    L.step(151)
    O.step(151)
    errs = field_errors(L.fields(), O.fields(), w.params)
    bad = {k: v for k, v in errs.items() if not v < TOL64}
    assert not bad, bad
    so = O.state()
    assert np.abs(L.state() - so).max() <= TOL64 * float(np.abs(so).max())


def test_fp64_inplace_binary_drops_1000_steps(T):
    """The 128x64 two-drop wetting case against the oracle after 1000 steps."""
    w = W.binary_drops_on_wall()
    L = T.lattice_from_workload(w, "fp64", inplace=True)
    O = OracleLattice(w.nx, w.ny, w.edges, w.mask, w.params)
    O.set_fields(w.c1, w.c2, w.ux, w.uy, w.p)
    L.step(1000)
    O.step(1000)
    errs = field_errors(L.fields(), O.fields(), w.params)
    assert all(v < TOL64 for v in errs.values()), errs


# bounds of the FP32 and 16-bit parity tests against the oracle
LOW_BOUNDS = {
    "fp32": dict(c1=("abs", 2e-4), c2=("abs", 2e-4), ux=("rel", 1e-3), uy=("rel", 1e-3), p=("rel", 1e-3)),
    "fp16": dict(c1=("abs", 2e-4), c2=("abs", 2e-4), ux=("rel", 3e-2), uy=("rel", 3e-2), p=("rel", 6e-2)),
    "bf16": dict(c1=("abs", 2e-3), c2=("abs", 2e-3), ux=("rel", 0.2), uy=("rel", 0.2), p=("rel", 0.5)),
}


@pytest.mark.parametrize("precision", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("seed,edges,lid_u", [(11, (0, 0, 1, 2), 0.0), (14, (0, 0, 1, 3), 0.02)])
def test_low_precision_inplace_matches_oracle(T, precision, seed, edges, lid_u):
    w = W.random_lattice(67, 45, seed, edges=edges, solids=("disc", "corner"), lid_u=lid_u)
    L = T.lattice_from_workload(w, precision, inplace=True)
    O = OracleLattice(w.nx, w.ny, w.edges, w.mask, w.params)
    O.set_fields(w.c1, w.c2, w.ux, w.uy, w.p)
    m0 = np.array(L.diagnostics()["mass"])
    L.step(151)
    O.step(151)
    fg, fo = L.fields(), O.fields()
    for k, (kind, bound) in LOW_BOUNDS[precision].items():
        err = float(np.abs(fg[k] - fo[k]).max())
        if kind == "rel":
            err /= max(float(np.abs(fo[k]).max()), 1e-12)
        assert err < bound, f"{precision}: {k} error {err:.3e} >= {bound}"
    if lid_u == 0.0:  # the lid is not mass-conserving
        drift = np.abs(np.array(L.diagnostics()["mass"]) - m0) / np.abs(m0)
        assert np.all(drift < 1e-9), drift


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
@pytest.mark.parametrize("edges", [(0, 0, 0, 0), (0, 0, 1, 2), (0, 0, 1, 3)])
def test_banded_host_set_up_equals_two_buffer_set_up(T, precision, edges):
    """Host set-up of an in-place lattice goes through the order-parameter
    planes in bands of rows (several bands at 96x160); the state it builds
    equals the two-buffer set-up exactly."""
    w = W.random_lattice(96, 160, 5, edges=edges, solids=("disc",), lid_u=0.01 if edges[3] == 3 else 0.0)
    A = T.lattice_from_workload(w, precision)
    B = T.lattice_from_workload(w, precision, inplace=True)
    assert np.array_equal(A.state(), B.state())


def test_batch_rejects_inplace_lattice(T):
    w = W.random_lattice(30, 20, 1)
    B = T.Batch("fp64", max_lattices=2)
    L = T.lattice_from_workload(w, "fp64", inplace=True)
    with pytest.raises(T.TlbError):
        B.add(L)
    B.close()
