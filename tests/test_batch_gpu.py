"""Batched execution: a lattice's result is the same alone and in a batch.

The batch runs the same per-tile and per-node device code as tlb_step, with
the member's parameters read from its device descriptor instead of kernel
arguments; the compiler may fuse multiply-adds differently in the two
kernels, so results agree to rounding, not bit for bit.  Every member must
match the same lattice stepped alone within the FP64 parity tolerance
(1e-12 relative max-norm of the raw state) or, in FP32, within 1e-5 of the
state's scale (a few FP32 roundings amplified over tens of steps), whatever
else is in the batch, across odd and even step counts, membership changes
and tuning.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


TOL = dict(fp64=1e-12, fp32=1e-5)


def same(a, m, precision):
    sa, sm = a.state(), m.state()
    return float(np.abs(sa - sm).max() / max(np.abs(sa).max(), 1e-6)) < TOL[precision]


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
        L.step(8 * (2 + 2) + 3)
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
