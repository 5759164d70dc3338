"""GB300 lattice library for the ternary phase-field lattice Boltzmann model with
wetting boundaries (Liang et al., arXiv:1710.09534, Sec. II).

This module is argument marshalling only: every step of the update runs in the
CUDA kernels of ``libtlbm.so`` behind the C ABI of ``include/tlbm.h``.  PyTorch
provides the device workspace and the stream.  There is no CPU fallback: if
the library or a CUDA device is missing, constructing a lattice raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtlbm.so")

FP64, FP32, FP16, BF16 = 0, 1, 2, 3
INPLACE = 0x100  # OR-ed into the precision: one distribution buffer, in-place streaming
EDGE_PERIODIC, EDGE_WETTING, EDGE_NEUTRAL, EDGE_LID = 0, 1, 2, 3
OK, EINVAL, ENOMEM, ECUDA, EUNSTABLE, ETIMEOUT, ESTATE = 0, -1, -2, -3, -4, -5, -6
FIELDS = ("c1", "c2", "c3", "rho", "ux", "uy", "p", "mu1", "mu2", "mu3")
F_ALL = (1 << 10) - 1
PRECISIONS = {"fp64": FP64, "f64": FP64, "fp32": FP32, "f32": FP32, "fp16": FP16, "f16": FP16, "bf16": BF16}

_lib = None


class TlbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"tlbm error {code}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    """``tlb_params`` of include/tlbm.h."""

    _fields_ = [(n, ctypes.c_double) for n in (
        "sigma12", "sigma13", "sigma23", "theta12_deg", "theta13_deg", "theta23_deg",
        "rho1", "rho2", "rho3", "nu1", "nu2", "nu3", "M0", "D", "tau1", "tau2",
        "gx", "gy", "lid_u", "collision", "mrt_s_f", "mrt_s_g")]

    @classmethod
    def from_dict(cls, d: dict) -> "Params":
        p = cls()
        full = dict(tau1=0.8, tau2=0.8, gx=0.0, gy=0.0, lid_u=0.0, collision=0.0, mrt_s_f=1.0, mrt_s_g=1.0)
        full.update(d)
        for name, _ in cls._fields_:
            setattr(p, name, float(full[name]))
        return p


class Diag(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double * 3), ("nonfinite", ctypes.c_int64)]


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libtlbm.so (build it first with ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: run `python -c 'import __graft_entry__ as g; g.build()'`")
    import torch  # noqa: F401  (loads the CUDA runtime the library links against)
    L = ctypes.CDLL(path)
    vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
    sig = {
        "tlb_workspace_bytes": (i64, [i32, i32, i32]),
        "tlb_create_lattice": (i32, [i32, i32, i32, ctypes.POINTER(ctypes.c_int32), vp, i64, vp,
                                     ctypes.POINTER(vp)]),
        "tlb_set_geometry": (i32, [vp, ctypes.POINTER(ctypes.c_uint8)]),
        "tlb_set_params": (i32, [vp, ctypes.POINTER(Params)]),
        "tlb_set_fields": (i32, [vp, dp, dp, dp, dp, dp]),
        "tlb_set_fields_device": (i32, [vp, vp, vp, vp, vp, vp]),
        "tlb_step": (i32, [vp, i64]),
        "tlb_sync": (i32, [vp, i64]),
        "tlb_read_fields": (i32, [vp, ctypes.c_uint32, dp]),
        "tlb_read_fields_device": (i32, [vp, ctypes.c_uint32, vp]),
        "tlb_diagnostics": (i32, [vp, ctypes.POINTER(Diag)]),
        "tlb_read_state": (i32, [vp, dp]),
        "tlb_state_bytes": (i64, [vp]),
        "tlb_export_state": (i32, [vp, vp, i64]),
        "tlb_import_state": (i32, [vp, vp, i64]),
        "tlb_theta12_from": (i32, [ctypes.c_double] * 5 + [dp]),
        "tlb_wall_nodes": (i64, [vp]),
        "tlb_diagnostics_noalloc": (i32, [vp, vp]),
        "tlb_contact_angles": (i32, [vp, i32, dp, i32, ctypes.POINTER(ctypes.c_int)]),
        "tlb_film_thickness": (i32, [vp, i32, i32, i32, dp]),
        "tlb_profile": (i32, [vp, i32]),
        "tlb_profile_read": (i32, [vp, dp, ctypes.POINTER(ctypes.c_int64)]),
        "tlb_destroy": (None, [vp]),
        "tlb_fma_peak": (i32, [i32, vp, dp, dp]),
        "tlb_batch_workspace_bytes": (i64, [i32, i64, i64]),
        "tlb_batch_tiles_needed": (i64, [i32, i32]),
        "tlb_batch_create": (i32, [i32, i32, i64, i64, vp, i64, vp, ctypes.POINTER(vp)]),
        "tlb_batch_add": (i32, [vp, vp]),
        "tlb_batch_remove": (i32, [vp, vp]),
        "tlb_batch_size": (i32, [vp]),
        "tlb_batch_step": (i32, [vp, i64]),
        "tlb_batch_config": (i32, [vp, i32, i32, i32, i32]),
        "tlb_batch_tune_scratch_bytes": (i64, [vp]),
        "tlb_batch_tune": (i32, [vp, i32, vp, i64, ctypes.POINTER(ctypes.c_int), dp]),
        "tlb_batch_destroy": (None, [vp]),
        "tlb_last_error": (ctypes.c_char_p, []),
        "tlb3_workspace_bytes": (i64, [i32, i32, i32, i32]),
        "tlb3_create": (i32, [i32, i32, i32, i32, ctypes.POINTER(ctypes.c_int32), vp, i64, vp, ctypes.POINTER(vp)]),
        "tlb3_set_geometry": (i32, [vp, ctypes.POINTER(ctypes.c_uint8)]),
        "tlb3_set_params": (i32, [vp, ctypes.POINTER(Params)]),
        "tlb3_set_fields": (i32, [vp, dp, dp, dp, dp, dp, dp]),
        "tlb3_step": (i32, [vp, i64]),
        "tlb3_sync": (i32, [vp]),
        "tlb3_read_fields": (i32, [vp, ctypes.c_uint32, dp]),
        "tlb3_read_state": (i32, [vp, dp]),
        "tlb3_diagnostics": (i32, [vp, ctypes.POINTER(Diag)]),
        "tlb3_profile": (i32, [vp, i32]),
        "tlb3_profile_read": (i32, [vp, dp, ctypes.POINTER(ctypes.c_int64)]),
        "tlb3_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def last_error() -> str:
    return load_library().tlb_last_error().decode()


def _check(rc):
    if rc < 0:
        raise TlbError(rc, last_error())
    return rc


def _f64(a, n):
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    if a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Lattice:
    """One lattice on the current CUDA device, advanced on ``stream``.

    The device workspace is a torch uint8 tensor owned by this object.
    Arrays are [ny, nx] (x fastest).
    """

    def __init__(self, nx: int, ny: int, precision="fp64", edges=(0, 0, 1, 2), stream=None, device=None,
                 inplace=False):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("tlbm needs a CUDA device; there is no CPU fallback")
        self.lib = load_library()
        self.nx, self.ny = int(nx), int(ny)
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.inplace = bool(inplace)
        flags = self.precision | (INPLACE if self.inplace else 0)
        self.edges = tuple(int(e) for e in edges)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            nbytes = _check(self.lib.tlb_workspace_bytes(self.nx, self.ny, flags))
            self.workspace = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
            h = ctypes.c_void_p()
            e = (ctypes.c_int32 * 4)(*self.edges)
            _check(self.lib.tlb_create_lattice(self.nx, self.ny, flags, e,
                                               ctypes.c_void_p(self.workspace.data_ptr()),
                                               int(nbytes), ctypes.c_void_p(self.stream.cuda_stream),
                                               ctypes.byref(h)))
        self._h = h
        self.mask = np.zeros((self.ny, self.nx), np.uint8)

    @property
    def n(self):
        return self.nx * self.ny

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self.lib.tlb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_geometry(self, mask=None):
        if mask is None:
            m = np.zeros((self.ny, self.nx), np.uint8)
        else:
            m = np.ascontiguousarray(mask, dtype=np.uint8).reshape(self.ny, self.nx)
        _check(self.lib.tlb_set_geometry(self._h, m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))))
        self.mask = m.copy()

    def set_params(self, params):
        p = params if isinstance(params, Params) else Params.from_dict(params)
        _check(self.lib.tlb_set_params(self._h, ctypes.byref(p)))
        self.params = p

    def set_fields(self, c1, c2, ux, uy, p=None):
        arrs = [_f64(a, self.n) for a in (c1, c2, ux, uy)]
        pp = _f64(p, self.n) if p is not None else None
        _check(self.lib.tlb_set_fields(self._h, *(_dp(a) for a in arrs), _dp(pp) if pp is not None else None))

    def set_fields_device(self, c1, c2, ux, uy, p=None):
        """Device FP64 tensors of nx*ny elements each (asynchronous)."""
        ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
        _check(self.lib.tlb_set_fields_device(self._h, ptr(c1), ptr(c2), ptr(ux), ptr(uy), ptr(p)))

    def step(self, n: int = 1):
        _check(self.lib.tlb_step(self._h, int(n)))

    def sync(self, timeout_ms: int = -1):
        return _check(self.lib.tlb_sync(self._h, int(timeout_ms)))

    def fields(self, names=FIELDS, out=None) -> dict:
        """Host copies of the selected fields; `out` may be a preallocated
        (e.g. pinned) float64 array of shape [len(names), ny, nx]."""
        mask = 0
        for nm in names:
            mask |= 1 << FIELDS.index(nm)
        order = [f for i, f in enumerate(FIELDS) if mask & (1 << i)]
        if out is None:
            out = np.empty((len(order), self.ny, self.nx))
        assert out.dtype == np.float64 and out.flags.c_contiguous and out.size == len(order) * self.n
        _check(self.lib.tlb_read_fields(self._h, mask, _dp(out)))
        return {k: out[i] for i, k in enumerate(order)}

    def fields_device(self, out, names=FIELDS):
        mask = 0
        for nm in names:
            mask |= 1 << FIELDS.index(nm)
        _check(self.lib.tlb_read_fields_device(self._h, mask, ctypes.c_void_p(out.data_ptr())))

    def diagnostics(self):
        d = Diag()
        rc = self.lib.tlb_diagnostics(self._h, ctypes.byref(d))
        if rc < 0 and rc != EUNSTABLE:
            raise TlbError(rc, last_error())
        return dict(mass=np.array(d.mass[:]), nonfinite=int(d.nonfinite), rc=rc)

    def diagnostics_noalloc(self, dev_out):
        """Allocation-free reduction into a device float64 tensor of >= 4
        elements: [sum c1, sum c2, sum c3, non-finite count] (asynchronous)."""
        _check(self.lib.tlb_diagnostics_noalloc(self._h, ctypes.c_void_p(dev_out.data_ptr())))

    def contact_angles(self, component: int = 1, max_drops: int = 64):
        """Drops of `component` on the bottom wall: list of (L_s, H_d, theta_n deg, x_mid)."""
        out = np.zeros(4 * max_drops)
        n = ctypes.c_int()
        _check(self.lib.tlb_contact_angles(self._h, int(component), _dp(out), int(max_drops), ctypes.byref(n)))
        k = min(n.value, max_drops)
        return [tuple(out[4 * i:4 * i + 4]) for i in range(k)]

    def film_thickness(self, x: int, y_top: int, comps: int = 3) -> float:
        """Film thickness above solid node (x, y_top) of c1 (comps=1), c2 (2) or
        c1 + c2 (3): see tlb_film_thickness."""
        h = ctypes.c_double()
        _check(self.lib.tlb_film_thickness(self._h, int(x), int(y_top), int(comps), ctypes.byref(h)))
        return h.value

    def state(self) -> np.ndarray:
        out = np.empty((31, self.ny, self.nx))
        _check(self.lib.tlb_read_state(self._h, _dp(out)))
        return out

    def export_state(self) -> bytes:
        n = _check(self.lib.tlb_state_bytes(self._h))
        buf = ctypes.create_string_buffer(int(n))
        _check(self.lib.tlb_export_state(self._h, buf, n))
        return buf.raw

    def import_state(self, data: bytes):
        buf = ctypes.create_string_buffer(data, len(data))
        _check(self.lib.tlb_import_state(self._h, buf, len(data)))

    def profile(self, enable: bool = True):
        _check(self.lib.tlb_profile(self._h, int(bool(enable))))

    def profile_read(self):
        """(interior_ms, wall_ms, interior_launches, wall_launches) since profile(True)."""
        ms = (ctypes.c_double * 2)()
        n = (ctypes.c_int64 * 2)()
        _check(self.lib.tlb_profile_read(self._h, ms, n))
        return ms[0], ms[1], n[0], n[1]

    def wall_nodes(self) -> int:
        return _check(self.lib.tlb_wall_nodes(self._h))


def fma_peak(precision="fp64") -> dict:
    """Measured fused-multiply-add rate of the current device (tlb_fma_peak):
    {"tflops": ..., "ms": ...}."""
    import torch
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _check(load_library().tlb_fma_peak(PRECISIONS[precision], ctypes.c_void_p(sink.data_ptr()),
                                       ctypes.byref(tf), ctypes.byref(ms)))
    return {"tflops": tf.value, "ms": ms.value}


def theta12_from(s12, s13, s23, th13, th23) -> float:
    out = ctypes.c_double()
    _check(load_library().tlb_theta12_from(s12, s13, s23, th13, th23, ctypes.byref(out)))
    return out.value


def lattice_from_workload(w, precision="fp64", stream=None, inplace=False) -> Lattice:
    """Create and initialise a Lattice from a ``workloads.Workload``."""
    L = Lattice(w.nx, w.ny, precision, w.edges, stream=stream, inplace=inplace)
    L.set_geometry(w.mask)
    L.set_params(w.params)
    L.set_fields(w.c1, w.c2, w.ux, w.uy, w.p)
    return L


class Batch:
    """Lattices advanced together by one persistent kernel per step (see the
    "Batches" section of include/tlbm.h).  Capacity is fixed at creation:
    `max_lattices` members whose tiles and near-wall nodes sum to at most
    `max_tiles` (tlb_batch_tiles_needed per member) and `max_wall_nodes`."""

    def __init__(self, precision="fp32", max_lattices=256, max_tiles=1 << 16, max_wall_nodes=1 << 20,
                 stream=None, device=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("tlbm needs a CUDA device; there is no CPU fallback")
        self.lib = load_library()
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
            nbytes = _check(self.lib.tlb_batch_workspace_bytes(int(max_lattices), int(max_tiles),
                                                              int(max_wall_nodes)))
            self.workspace = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
            h = ctypes.c_void_p()
            _check(self.lib.tlb_batch_create(self.precision, int(max_lattices), int(max_tiles),
                                             int(max_wall_nodes), ctypes.c_void_p(self.workspace.data_ptr()),
                                             int(nbytes), ctypes.c_void_p(self.stream.cuda_stream),
                                             ctypes.byref(h)))
        self._h = h
        self.members = []

    @staticmethod
    def tiles_needed(nx, ny) -> int:
        return _check(load_library().tlb_batch_tiles_needed(int(nx), int(ny)))

    def add(self, lattice: "Lattice"):
        _check(self.lib.tlb_batch_add(self._h, lattice._h))
        self.members.append(lattice)

    def remove(self, lattice: "Lattice"):
        _check(self.lib.tlb_batch_remove(self._h, lattice._h))
        self.members.remove(lattice)

    def __len__(self):
        return _check(self.lib.tlb_batch_size(self._h))

    def step(self, n: int = 1):
        _check(self.lib.tlb_batch_step(self._h, int(n)))

    def config(self, threads=128, rows_small=16, rows_large=16, small_ny=128):
        _check(self.lib.tlb_batch_config(self._h, int(threads), int(rows_small), int(rows_large), int(small_ny)))

    def tune(self, trial_steps: int = 5):
        """Pick the fastest tile shape by timing the candidates on the current
        members; every member's state is left as it was (the library saves
        and restores the c_i u planes in a scratch buffer allocated here)."""
        import torch
        cfg = (ctypes.c_int * 4)()
        ms = ctypes.c_double()
        nbytes = _check(self.lib.tlb_batch_tune_scratch_bytes(self._h))
        with torch.cuda.device(self.device):
            scratch = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=self.device)
            _check(self.lib.tlb_batch_tune(self._h, int(trial_steps), ctypes.c_void_p(scratch.data_ptr()),
                                           int(scratch.numel()), cfg, ctypes.byref(ms)))
        del scratch
        return dict(threads=cfg[0], rows_small=cfg[1], rows_large=cfg[2], small_ny=cfg[3], ms_per_step=ms.value)

    def synchronize(self):
        self.stream.synchronize()

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self.lib.tlb_batch_destroy(self._h)
            self._h = None
            self.members = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


FIELDS3 = ("c1", "c2", "c3", "rho", "ux", "uy", "uz", "p", "mu1", "mu2", "mu3")


class Lattice3D:
    """One D3Q19 lattice (FP64 or FP32 storage and arithmetic) on the current CUDA device, advanced on
    ``stream`` (see the "D3Q19" section of include/tlbm.h).  Arrays are
    [nz, ny, nx]; edges = (x-, x+, y-, y+, z-, z+)."""

    def __init__(self, nx: int, ny: int, nz: int, edges=(0, 0, 1, 2, 0, 0), stream=None, device=None,
                 precision="fp64"):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("tlbm needs a CUDA device; there is no CPU fallback")
        self.lib = load_library()
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.shape = (self.nz, self.ny, self.nx)
        self.edges = tuple(int(e) for e in edges)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
            nbytes = _check(self.lib.tlb3_workspace_bytes(self.nx, self.ny, self.nz, self.precision))
            self.workspace = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
            h = ctypes.c_void_p()
            e = (ctypes.c_int32 * 6)(*self.edges)
            _check(self.lib.tlb3_create(self.nx, self.ny, self.nz, self.precision, e,
                                        ctypes.c_void_p(self.workspace.data_ptr()),
                                        int(nbytes), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self._h = h

    @property
    def n(self):
        return self.nx * self.ny * self.nz

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self.lib.tlb3_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_geometry(self, mask=None):
        m = np.zeros(self.shape, np.uint8) if mask is None else np.ascontiguousarray(mask, np.uint8).reshape(self.shape)
        _check(self.lib.tlb3_set_geometry(self._h, m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))))

    def set_params(self, params):
        p = params if isinstance(params, Params) else Params.from_dict(params)
        _check(self.lib.tlb3_set_params(self._h, ctypes.byref(p)))

    def set_fields(self, c1, c2, ux, uy, uz, p=None):
        arrs = [_f64(a, self.n) for a in (c1, c2, ux, uy, uz)]
        pp = _f64(p, self.n) if p is not None else None
        _check(self.lib.tlb3_set_fields(self._h, *(_dp(a) for a in arrs), _dp(pp) if pp is not None else None))

    def step(self, n: int = 1):
        _check(self.lib.tlb3_step(self._h, int(n)))

    def sync(self):
        return _check(self.lib.tlb3_sync(self._h))

    def fields(self, names=FIELDS3) -> dict:
        mask = 0
        for nm in names:
            mask |= 1 << FIELDS3.index(nm)
        order = [f for i, f in enumerate(FIELDS3) if mask & (1 << i)]
        out = np.empty((len(order),) + self.shape)
        _check(self.lib.tlb3_read_fields(self._h, mask, _dp(out)))
        return {k: out[i] for i, k in enumerate(order)}

    def state(self) -> np.ndarray:
        out = np.empty((63,) + self.shape)
        _check(self.lib.tlb3_read_state(self._h, _dp(out)))
        return out

    def profile(self, enable: bool = True):
        _check(self.lib.tlb3_profile(self._h, int(bool(enable))))

    def profile_read(self):
        """((csum_ms, mu_ms, update_ms), (launches...)) since profile(True)."""
        ms = (ctypes.c_double * 3)()
        n = (ctypes.c_int64 * 3)()
        _check(self.lib.tlb3_profile_read(self._h, ms, n))
        return tuple(ms), tuple(n)

    def diagnostics(self):
        d = Diag()
        rc = self.lib.tlb3_diagnostics(self._h, ctypes.byref(d))
        if rc < 0 and rc != EUNSTABLE:
            raise TlbError(rc, last_error())
        return dict(mass=np.array(d.mass[:]), nonfinite=int(d.nonfinite), rc=rc)


def lattice3_from_workload(w, stream=None, precision="fp64") -> Lattice3D:
    """Create and initialise a Lattice3D from a ``workloads.Workload3``
    (precision "fp64" or "fp32")."""
    L = Lattice3D(w.nx, w.ny, w.nz, w.edges, stream=stream, precision=precision)
    L.set_geometry(w.mask)
    L.set_params(w.params)
    L.set_fields(w.c1, w.c2, w.ux, w.uy, w.uz, w.p)
    return L
