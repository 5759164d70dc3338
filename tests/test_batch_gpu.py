"""Batched execution: every member matches the FP64 oracle, and a lattice's
result is the same alone and in a batch.

The batch runs the same per-tile and per-node device code as tlb_step, with
the member's parameters read from its device descriptor instead of kernel
arguments; the library is built with every fused multiply-add explicit
(-fmad=false), so both kernels round identically.  Every member's raw state
must equal that of the same lattice stepped alone bit for bit, whatever else
is in the batch, across odd and even step counts, membership changes and
tuning.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import OracleLattice
from parity import assert_bounded, assert_oracle_parity

pytestmark = pytest.mark.gpu


def same(a, m, precision):
    """The raw states of two lattices are equal bit for bit (`precision` names
    the storage in failure messages)."""
    sa, sm = a.state(), m.state()
    return bool(np.array_equal(sa, sm))


def oracle_of(w):
    O = OracleLattice(w.nx, w.ny, w.edges, w.mask, w.params)
    O.set_fields(w.c1, w.c2, w.ux, w.uy, w.p)
    return O


def _members_for_oracle():
    """A mixed population: random walls, solids and densities, velocity lids
    (two of them), a curved wetting cylinder with a falling compound drop and
    a drops-on-wall lattice."""
    ws = _mix(5, seed=41)
    ws.append(W.compound_drop_on_cylinder(nx=96, ny=144, R_cyl=12, R_core=7, R_shell=13, We=10.0, theta=40.0,
                                          cyl_center=(48, 40), drop_center=(48, 80)))
    ws.append(W.drops_on_wall(72, 5))
    return ws


@pytest.fixture(scope="module")
def T():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_09534_gb300 import build
    build.build()
    import paper_1710_09534_gb300 as T
    return T


def _mix(n=6, seed=3):
    rng = np.random.default_rng(seed)
    out = []
    specs = [((0, 0, 1, 2), ("disc",), 0.0), ((0, 0, 1, 3), ("corner",), 0.01), ((0, 0, 0, 0), ("pillar",), 0.0),
             ((1, 2, 2, 1), (), 0.0), ((0, 0, 1, 2), ("disc", "corner"), 0.0), ((2, 1, 1, 3), ("pillar",), 0.02)]
    for i in range(n):
        nx, ny = (int(v) for v in rng.integers(20, 200, 2))
        edges, solids, lid = specs[i % len(specs)]
        out.append(W.random_lattice(nx, ny, 100 + i, edges=edges, solids=solids, lid_u=lid))
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("steps", [1, 2, 7])
def test_members_match_lattices_stepped_alone(T, precision, steps):
    ws = _mix()
    alone = [T.lattice_from_workload(w, precision) for w in ws]
    mem = [T.lattice_from_workload(w, precision) for w in ws]
    B = T.Batch(precision, max_lattices=16)
    for L in mem:
        B.add(L)
    B.step(steps)
    B.step(steps + 1)
    for L in alone:
        L.step(2 * steps + 1)
    for a, m, w in zip(alone, mem, ws):
        assert same(a, m, precision), w.name


def test_membership_changes_keep_results(T):
    ws = _mix(5, seed=9)
    alone = [T.lattice_from_workload(w, "fp32") for w in ws]
    mem = [T.lattice_from_workload(w, "fp32") for w in ws]
    B = T.Batch("fp32", max_lattices=8)
    for L in mem[:3]:
        B.add(L)
    B.step(10)
    B.remove(mem[1])
    B.add(mem[3])
    B.step(5)
    B.add(mem[4])
    B.step(4)
    # each member's total steps: 0 -> 19, 1 -> 10, 2 -> 19, 3 -> 9, 4 -> 4
    for L, n in zip(alone, (19, 10, 19, 9, 4)):
        L.step(n)
    for a, m, w in zip(alone, mem, ws):
        assert same(a, m, "fp32"), w.name


def test_tune_and_config_keep_results(T):
    ws = _mix(4, seed=5)
    alone = [T.lattice_from_workload(w, "fp32") for w in ws]
    mem = [T.lattice_from_workload(w, "fp32") for w in ws]
    B = T.Batch("fp32", max_lattices=4)
    for L in mem:
        B.add(L)
    cfg = B.tune(trial_steps=2)
    assert cfg["threads"] in (64, 128) and cfg["ms_per_step"] > 0
    B.config(64, 8, 32, 100)
    B.step(3)
    for L in alone:
        L.step(3)  # tuning advanced no member
    for a, m in zip(alone, mem):
        assert same(a, m, "fp32")


def test_batch_errors(T):
    w = W.random_lattice(30, 20, 1)
    L = T.lattice_from_workload(w, "fp32")
    L64 = T.lattice_from_workload(w, "fp64")
    B = T.Batch("fp32", max_lattices=1)
    with pytest.raises(T.TlbError):
        B.add(L64)
    B.add(L)
    with pytest.raises(T.TlbError) as e:
        L.step(1)
    assert e.value.code == T.ESTATE
    with pytest.raises(T.TlbError) as e:
        B.add(T.lattice_from_workload(w, "fp32"))
    assert e.value.code == T.ENOMEM
    B.remove(L)
    L.step(1)


def test_fp64_batch_members_match_the_oracle(T):
    """Each member of a mixed FP64 batch -- walls, solids, lids, a cylinder --
    against its own oracle lattice at 1e-12 per field and per raw-state plane,
    after odd and even step counts and a membership change."""
    ws = _members_for_oracle()
    mem = [T.lattice_from_workload(w, "fp64") for w in ws]
    orc = [oracle_of(w) for w in ws]
    B = T.Batch("fp64", max_lattices=len(ws))
    for L in mem[:-2]:
        B.add(L)
    B.step(5)                      # odd: members end on the other buffer
    B.remove(mem[2])
    B.add(mem[-2])
    B.add(mem[-1])
    B.step(8)
    B.step(3)
    steps = [16, 16, 5, 16, 16, 11, 11]
    for L, O, n, w in zip(mem, orc, steps, ws):
        O.step(n)
        assert_oracle_parity(L, O, w.params, what=f"batch member {w.name}")
    B.close()


def test_fp64_mrt_batch_members_match_the_oracle(T):
    ws = _mix(3, seed=43)
    for w in ws:
        w.params.update(collision=1.0, mrt_s_f=1.2, mrt_s_g=1.3)
    mem = [T.lattice_from_workload(w, "fp64") for w in ws]
    B = T.Batch("fp64", max_lattices=3)
    for L in mem:
        B.add(L)
    B.step(9)
    for L, w in zip(mem, ws):
        O = oracle_of(w)
        O.step(9)
        assert_oracle_parity(L, O, w.params, what=f"MRT batch member {w.name}")
    B.close()


@pytest.mark.parametrize("precision", ["fp32", "fp16", "bf16"])
def test_reduced_precision_batch_members_within_their_bounds_of_the_oracle(T, precision):
    ws = _members_for_oracle()
    mem = [T.lattice_from_workload(w, precision) for w in ws]
    B = T.Batch(precision, max_lattices=len(ws))
    for L in mem:
        B.add(L)
    B.step(60)
    for L, w in zip(mem, ws):
        O = oracle_of(w)
        O.step(60)
        assert_bounded(L.fields(), O.fields(), precision, what=f"batch member {w.name}")
    B.close()


def test_tune_leaves_members_unchanged(T):
    """A batch's results are identical with and without a tune() call before
    step(): the tuner's trial steps write only the spare buffers and the c_i u
    planes it restores."""
    ws = _mix(4, seed=5)
    for precision in ("fp64", "fp32"):
        plain = [T.lattice_from_workload(w, precision) for w in ws]
        tuned = [T.lattice_from_workload(w, precision) for w in ws]
        Bp, Bt = T.Batch(precision, max_lattices=4), T.Batch(precision, max_lattices=4)
        for a, b in zip(plain, tuned):
            Bp.add(a)
            Bt.add(b)
        Bp.step(3)
        Bt.step(3)
        cfg = Bt.tune(trial_steps=2)
        Bp.config(cfg["threads"], cfg["rows_small"], cfg["rows_large"], cfg["small_ny"])
        Bp.step(4)
        Bt.step(4)
        for a, b in zip(plain, tuned):
            assert np.array_equal(a.state(), b.state())
        Bp.close()
        Bt.close()
