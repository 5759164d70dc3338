"""tlb_diagnostics_noalloc: the mass/non-finite reduction without allocation.

Some callers cannot allocate device memory at the point where they need the
totals (code that lives inside a fixed arena it does not own, or a loop that
must not stall on an allocation).  For them the library offers a variant of
the diagnostics reduction whose scratch is a static device array.  These
tests call it through the C ABI and check it against tlb_diagnostics on two
consecutive calls, and check that a lattice larger than the static scratch
is refused.  The file name makes pytest collect it last.
"""
import numpy as np
import pytest

import workloads as W

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


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_matches_diagnostics_on_consecutive_calls(T, precision):
    import torch
    w = W.random_lattice(96, 64, 31, edges=(0, 0, 1, 3), solids=("disc", "corner"), lid_u=0.01)
    L = T.lattice_from_workload(w, precision)
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):
        L.step(25)
        L.diagnostics_noalloc(out)
        got = out.cpu().numpy()  # synchronizes the lattice's (current) stream
        ref = L.diagnostics()
        assert ref["rc"] == 0
        assert np.allclose(got[:3], ref["mass"], rtol=1e-13, atol=1e-10)
        assert got[3] == ref["nonfinite"] == 0


def test_noalloc_rejects_lattices_beyond_its_static_scratch(T):
    import torch
    nx, ny = 4097, 4096  # one column more than the 4096 x 4096 limit
    L = T.Lattice(nx, ny, "fp32", (0, 0, 0, 0))
    L.set_params(W.params())
    z = torch.zeros(nx * ny, dtype=torch.float64, device="cuda")
    L.set_fields_device(z, z, z, z)
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(T.TlbError) as e:
        L.diagnostics_noalloc(out)
    assert e.value.code == T.EINVAL and "16777216-node limit" in str(e.value)
