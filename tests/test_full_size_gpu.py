"""Parity at the full sizes the bench times, in the launch configuration it
uses: the 2048x2048 tiled-drops lattice with FP32, FP16 and BF16 storage (two
buffers, and FP32 in place) and the 1024x2048 compound-drop impact on a
cylinder with FP32 and FP16 storage, each a few steps against the FP64
oracle on every node.  The FP64 form of the 2048x2048 check is in the FP64
parity tests.  Bounds: those of the FP32 and 16-bit parity tests.
"""
import numpy as np
import pytest

import workloads as W
from oracle import OracleLattice

pytestmark = pytest.mark.gpu

BOUNDS = {
    "fp32": dict(c1=("abs", 2e-4), c2=("abs", 2e-4), c3=("abs", 2e-4), rho=("abs", 2e-3),
                 ux=("rel", 1e-3), uy=("rel", 1e-3), p=("rel", 1e-3), mu1=("rel", 2e-2), mu2=("rel", 2e-2)),
    "fp16": dict(c1=("abs", 2e-4), c2=("abs", 2e-4), c3=("abs", 2e-4), rho=("abs", 4e-4),
                 ux=("rel", 3e-2), uy=("rel", 3e-2), p=("rel", 6e-2), mu1=("rel", 6e-3), mu2=("rel", 6e-3)),
    "bf16": dict(c1=("abs", 2e-3), c2=("abs", 2e-3), c3=("abs", 2e-3), rho=("abs", 3e-3),
                 ux=("rel", 0.2), uy=("rel", 0.2), p=("rel", 0.5), mu1=("rel", 5e-2), mu2=("rel", 5e-2)),
}
# the impact case carries populations ~50x larger (density ratio 10, falling
# drop): the bounds of the cylinder-impact parity tests
IMPACT_BOUNDS = {
    "fp32": BOUNDS["fp32"],
    "fp16": dict(c1=("abs", 4e-3), c2=("abs", 4e-3), c3=("abs", 4e-3), rho=("abs", 2e-2),
                 ux=("rel", 1e-2), uy=("rel", 1e-2), p=("rel", 0.12), mu1=("rel", 3e-2), mu2=("rel", 3e-2)),
}
STEPS = 3  # odd: the in-place form ends on an even step and streams in place


@pytest.fixture(scope="module")
def T():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_09534_gb300 import build
    build.build()
    import paper_1710_09534_gb300 as T
    return T


def _oracle_fields(w, steps):
    O = OracleLattice(w.nx, w.ny, w.edges, w.mask, w.params)
    O.set_fields(w.c1, w.c2, w.ux, w.uy, w.p)
    O.step(steps)
    return O.fields()


@pytest.fixture(scope="module")
def tiled():
    w = W.tiled_drops(2048, 2048)
    return w, _oracle_fields(w, STEPS)


@pytest.fixture(scope="module")
def impact():
    w = W.compound_drop_on_cylinder(1024, 2048, We=10.0)
    return w, _oracle_fields(w, STEPS)


def _check(fg, fo, bounds, what):
    for k, (kind, bound) in bounds.items():
        err = float(np.abs(fg[k] - fo[k]).max())
        if kind == "rel":
            err /= max(float(np.abs(fo[k]).max()), 1e-12)
        assert err < bound, f"{what}: {k} error {err:.3e} >= {bound}"


@pytest.mark.parametrize("precision,inplace", [("fp32", False), ("fp16", False), ("bf16", False), ("fp32", True)])
def test_tiled_drops_2048_low_precision(T, tiled, precision, inplace):
    w, fo = tiled
    L = T.lattice_from_workload(w, precision, inplace=inplace)
    L.step(STEPS)
    _check(L.fields(), fo, BOUNDS[precision], f"2048^2 {precision}{' in place' if inplace else ''}")
    assert L.diagnostics()["nonfinite"] == 0
    L.close()


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_cylinder_impact_1024x2048(T, impact, precision):
    w, fo = impact
    L = T.lattice_from_workload(w, precision)
    L.step(STEPS)
    _check(L.fields(), fo, IMPACT_BOUNDS[precision], f"impact 1024x2048 {precision}")
    L.close()
