"""The C-ABI library builds, loads and exports every symbol include/tlbm.h
declares; host-only entry points behave as documented (no GPU needed)."""
import ctypes
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tlbm.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tlb3?_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1710_09534_gb300 import build
    build.build()
    import paper_1710_09534_gb300 as T
    return T.load_library()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("tlb_create_lattice", "tlb_set_geometry", "tlb_set_params", "tlb_set_fields",
                     "tlb_step", "tlb_read_fields", "tlb_diagnostics", "tlb_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_workspace_size_validation(lib):
    import paper_1710_09534_gb300 as T
    assert lib.tlb_workspace_bytes(2, 64, 0) == T.EINVAL
    assert lib.tlb_workspace_bytes(64, 64, 7) == T.EINVAL
    b64 = lib.tlb_workspace_bytes(128, 64, T.FP64)
    b32 = lib.tlb_workspace_bytes(128, 64, T.FP32)
    # 2 x 27 distribution planes + 4 c_i u planes per node, plus classes/list
    assert b64 >= 128 * 64 * (54 + 4) * 8
    assert b32 >= 128 * 64 * (54 + 4) * 4
    assert b64 > b32


def test_d3q19_workspace_size_validation(lib):
    """tlb3_workspace_bytes: FP64 and FP32 storage, and invalid sizes or
    precisions (host-only)."""
    import paper_1710_09534_gb300 as T
    f = lib.tlb3_workspace_bytes
    w64, w32 = f(64, 32, 48, T.FP64), f(64, 32, 48, T.FP32)
    assert w64 > 0 and w32 > 0
    plane = 64 * 32 * 48
    assert w64 >= (2 * 57 + 6 + 4) * 8 * plane and w32 >= (2 * 59 + 6 + 4) * 4 * plane
    assert w32 < 0.6 * w64
    assert f(2, 32, 48, T.FP64) == T.EINVAL and f(64, 32, 48, T.FP16) == T.EINVAL
    assert f(65536, 65536, 4, T.FP64) == T.EINVAL  # 2^34 nodes: beyond one 32-bit thread index per node


def test_inplace_workspace_is_smaller(lib):
    """One distribution buffer plus two order-parameter planes instead of two
    buffers: 0.57 (FP64, FP32) and 0.62 (16-bit) of the two-buffer workspace
    at 2048x2048; an unknown precision with the flag is still rejected."""
    import paper_1710_09534_gb300 as T
    for p, ratio in ((T.FP64, 0.58), (T.FP32, 0.58), (T.FP16, 0.63), (T.BF16, 0.63)):
        two = lib.tlb_workspace_bytes(2048, 2048, p)
        one = lib.tlb_workspace_bytes(2048, 2048, p | T.INPLACE)
        assert 0 < one < ratio * two, (p, one, two)
    assert lib.tlb_workspace_bytes(64, 64, 4 | T.INPLACE) == T.EINVAL
    assert lib.tlb_workspace_bytes(2, 64, T.FP32 | T.INPLACE) == T.EINVAL


def test_theta12_helper_applies_eq39(lib):
    import paper_1710_09534_gb300 as T
    th = T.theta12_from(1e-3, 1e-3, 1e-3, 90.0, 120.0)
    assert math.isclose(th, 60.0, rel_tol=1e-12)
    # paper's shear triple (Sec. III.C): theta13 = 68.53 from theta12 = 30, theta23 = 120
    th = T.theta12_from(0.01, 0.01, 0.01, 68.53, 120.0)
    assert abs(th - 30.0) < 0.02
    out = ctypes.c_double()
    assert lib.tlb_theta12_from(1e-3, 1e-3, 1e-3, 10.0, 170.0, ctypes.byref(out)) == T.EINVAL
    assert "Eq. 39" in T.last_error()


def test_create_rejects_bad_arguments_without_touching_the_device(lib):
    import paper_1710_09534_gb300 as T
    h = ctypes.c_void_p()
    e = (ctypes.c_int32 * 4)(0, 1, 1, 2)  # unpaired periodic edge
    assert lib.tlb_create_lattice(16, 16, 0, e, None, 0, None, ctypes.byref(h)) == T.EINVAL
    e = (ctypes.c_int32 * 4)(3, 3, 1, 2)  # lid on a side edge
    assert lib.tlb_create_lattice(16, 16, 0, e, None, 0, None, ctypes.byref(h)) == T.EINVAL
    e = (ctypes.c_int32 * 4)(0, 0, 1, 2)
    assert lib.tlb_create_lattice(16, 16, 0, e, None, 0, None, ctypes.byref(h)) == T.EINVAL
    assert "workspace" in T.last_error()
    assert lib.tlb_step(None, 1) == T.EINVAL
    hf = ctypes.c_double()
    assert lib.tlb_film_thickness(None, 0, 0, 3, ctypes.byref(hf)) == T.EINVAL


def test_python_params_mirror_the_header_struct():
    """The binding's ctypes Params has the fields of tlb_params, in order."""
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    body = re.search(r"typedef struct \{([^}]*)\} tlb_params;", src).group(1)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if decl:
            assert decl.startswith("double ")
            names += [n.strip() for n in decl[len("double "):].split(",")]
    import paper_1710_09534_gb300 as T
    assert [n for n, _ in T.Params._fields_] == names
