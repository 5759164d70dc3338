"""FP64 CPU oracle of the ternary phase-field lattice Boltzmann update with wetting.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use this package; the CUDA library never does.

The arithmetic lives in ``tlb_oracle.c`` (plain C, FP64, one pass per stage of
the update, written from Sec. II of Liang et al., arXiv:1710.09534).  This
module only compiles it with gcc, marshals arrays through ctypes and adds the
contact-angle measurement of Sec. III.A in numpy.

The D3Q19 form of the same model (Sec. II.A states it for D dimensions) lives
in ``tlb_oracle3d.c`` (``OracleLattice3D``), built into the same library.

Parity status: every function is pinned by ``tests/test_oracle_*.py`` and
``tests/test_oracle3d.py`` except the figure values of Figs. 3, 5 and 14,
which the paper text does not carry (parity unpinned for those; no function
here reproduces them).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tlb_oracle.c")
_SRC3 = os.path.join(_HERE, "tlb_oracle3d.c")
_HDR = os.path.join(_HERE, "tlb_oracle.h")
_LIB = os.path.join(_HERE, "libtlb_oracle.so")
_lock = threading.Lock()
_lib = None

EDGE_PERIODIC, EDGE_WETTING, EDGE_NEUTRAL, EDGE_LID = 0, 1, 2, 3
FIELDS = ("c1", "c2", "c3", "rho", "ux", "uy", "p", "mu1", "mu2", "mu3")


class Params(ctypes.Structure):
    """Model parameters; field order matches ``orc_params`` in tlb_oracle.c."""

    _fields_ = [(n, ctypes.c_double) for n in (
        "sigma12", "sigma13", "sigma23",
        "theta12_deg", "theta13_deg", "theta23_deg",
        "rho1", "rho2", "rho3", "nu1", "nu2", "nu3",
        "M0", "D", "tau1", "tau2", "gx", "gy", "lid_u", "collision", "mrt_s_f", "mrt_s_g")]


def build(force: bool = False) -> str:
    """Compile tlb_oracle.c into libtlb_oracle.so next to it (gcc -O2, OpenMP over nodes)."""
    with _lock:
        stale = not os.path.exists(_LIB) or any(os.path.getmtime(_LIB) < os.path.getmtime(f)
                                                for f in (_SRC, _SRC3, _HDR))
        if force or stale:
            tmp = _LIB + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC",
                                   "-shared", "-std=c11", "-o", tmp, _SRC, _SRC3, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        L.orc_create.restype = ctypes.c_void_p
        L.orc_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        L.orc_set_geometry.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_ubyte)]
        L.orc_set_params.argtypes = [ctypes.c_void_p, ctypes.POINTER(Params)]
        L.orc_set_fields.argtypes = [ctypes.c_void_p, dp, dp, dp, dp, dp]
        L.orc_set_fields.restype = ctypes.c_int
        L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_long]
        L.orc_step.restype = ctypes.c_int
        L.orc_read_fields.argtypes = [ctypes.c_void_p, dp]
        L.orc_read_fields.restype = ctypes.c_int
        L.orc_read_aux.argtypes = [ctypes.c_void_p, dp]
        L.orc_read_aux.restype = ctypes.c_int
        L.orc_get_state.argtypes = [ctypes.c_void_p, dp]
        L.orc_set_state.argtypes = [ctypes.c_void_p, dp]
        L.orc_lambdas.argtypes = [ctypes.c_double] * 3 + [dp]
        L.orc_chem_pot.argtypes = [dp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, dp]
        L.orc_wet_offset.argtypes = [ctypes.c_double] * 6 + [dp]
        L.orc_grad.argtypes = [dp, dp]
        L.orc_lap.argtypes = [dp]
        L.orc_lap.restype = ctypes.c_double
        for name, nargs in (("orc_sk", 2), ("orc_feq", 5), ("orc_geq", 4),
                            ("orc_src_f", 3), ("orc_src_g", 9)):
            fn = getattr(L, name)
            fn.argtypes = [ctypes.c_int] + [ctypes.c_double] * nargs
            fn.restype = ctypes.c_double
        for name in ("orc_ex", "orc_ey", "orc_opp"):
            getattr(L, name).argtypes = [ctypes.c_int]
            getattr(L, name).restype = ctypes.c_int
        L.orc_threads.restype = ctypes.c_int
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_mrt_matrix.argtypes = [dp]
        L.orc_mrt_inverse.argtypes = [dp]
        L.orc_mrt_relax.argtypes = [dp, dp, dp, dp, dp]
        L.orc_w.argtypes = [ctypes.c_int]
        L.orc_w.restype = ctypes.c_double
        # D3Q19 form (tlb_oracle3d.c)
        L.orc3_create.restype = ctypes.c_void_p
        L.orc3_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        L.orc3_destroy.argtypes = [ctypes.c_void_p]
        L.orc3_set_geometry.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_ubyte)]
        L.orc3_set_params.argtypes = [ctypes.c_void_p, ctypes.POINTER(Params)]
        L.orc3_set_fields.argtypes = [ctypes.c_void_p, dp, dp, dp, dp, dp, dp]
        L.orc3_set_fields.restype = ctypes.c_int
        L.orc3_step.argtypes = [ctypes.c_void_p, ctypes.c_long]
        L.orc3_step.restype = ctypes.c_int
        L.orc3_read_fields.argtypes = [ctypes.c_void_p, dp]
        L.orc3_read_fields.restype = ctypes.c_int
        L.orc3_get_state.argtypes = [ctypes.c_void_p, dp]
        L.orc3_set_state.argtypes = [ctypes.c_void_p, dp]
        L.orc3_grad.argtypes = [dp, dp]
        L.orc3_lap.argtypes = [dp]
        L.orc3_lap.restype = ctypes.c_double
        L.orc3_e.argtypes = [ctypes.c_int, ctypes.c_int]
        L.orc3_e.restype = ctypes.c_int
        L.orc3_opp.argtypes = [ctypes.c_int]
        L.orc3_opp.restype = ctypes.c_int
        L.orc3_w.argtypes = [ctypes.c_int]
        L.orc3_w.restype = ctypes.c_double
        L.orc3_feq.argtypes = [ctypes.c_int] + [ctypes.c_double] * 6
        L.orc3_feq.restype = ctypes.c_double
        L.orc3_geq.argtypes = [ctypes.c_int] + [ctypes.c_double] * 5
        L.orc3_geq.restype = ctypes.c_double
        L.orc3_sk.argtypes = [ctypes.c_int] + [ctypes.c_double] * 3
        L.orc3_sk.restype = ctypes.c_double
        L.orc3_src_f.argtypes = [ctypes.c_int] + [ctypes.c_double] * 4
        L.orc3_src_f.restype = ctypes.c_double
        L.orc3_src_g.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp, dp, dp]
        L.orc3_src_g.restype = ctypes.c_double
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def make_params(**kw) -> Params:
    P = Params()
    defaults = dict(tau1=0.8, tau2=0.8, gx=0.0, gy=0.0, lid_u=0.0, collision=0.0, mrt_s_f=1.0, mrt_s_g=1.0)
    defaults.update(kw)
    for name, _ in Params._fields_:
        setattr(P, name, float(defaults[name]))
    return P


class OracleLattice:
    """One nx-by-ny lattice advanced by the FP64 oracle (arrays are [ny, nx])."""

    def __init__(self, nx: int, ny: int, edges=(0, 0, 1, 2), mask=None, params=None):
        self.nx, self.ny = int(nx), int(ny)
        self.edges = tuple(int(e) for e in edges)
        e = (ctypes.c_int * 4)(*self.edges)
        self._h = lib().orc_create(self.nx, self.ny, e)
        if not self._h:
            raise ValueError("oracle: invalid lattice size")
        m = np.zeros((self.ny, self.nx), np.uint8) if mask is None else np.ascontiguousarray(mask, np.uint8)
        assert m.shape == (self.ny, self.nx)
        self.mask = m.copy()
        lib().orc_set_geometry(self._h, self.mask.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)))
        if params is not None:
            self.set_params(params)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def set_params(self, params):
        if not isinstance(params, Params):
            params = make_params(**params)
        self.params = params
        lib().orc_set_params(self._h, ctypes.byref(params))

    def set_fields(self, c1, c2, ux, uy, p=None):
        arrs = [_f64(a).reshape(self.ny, self.nx) for a in (c1, c2, ux, uy)]
        pp = _f64(p).reshape(self.ny, self.nx) if p is not None else None
        rc = lib().orc_set_fields(self._h, *(_dp(a) for a in arrs),
                                  _dp(pp) if pp is not None else None)
        if rc:
            raise RuntimeError("oracle: set_params first")

    def step(self, n: int = 1):
        if lib().orc_step(self._h, int(n)):
            raise RuntimeError("oracle: set_params first")

    def fields(self) -> dict:
        out = np.zeros((10, self.ny, self.nx))
        lib().orc_read_fields(self._h, _dp(out))
        return {k: out[i] for i, k in enumerate(FIELDS)}

    def aux(self) -> dict:
        """Forces and gradients: Fsx, Fsy, Fax, Fay, lap_mu1, lap_mu2, grx, gry."""
        out = np.zeros((8, self.ny, self.nx))
        lib().orc_read_aux(self._h, _dp(out))
        names = ("Fsx", "Fsy", "Fax", "Fay", "lap_mu1", "lap_mu2", "grx", "gry")
        return {k: out[i] for i, k in enumerate(names)}

    def state(self) -> np.ndarray:
        """Raw state [31, ny, nx]: f1 k=0..8, f2 k=0..8, g k=0..8, c1ux, c1uy, c2ux, c2uy."""
        out = np.zeros((31, self.ny, self.nx))
        lib().orc_get_state(self._h, _dp(out))
        return out

    def set_state(self, s):
        s = _f64(s).reshape(31, self.ny, self.nx)
        lib().orc_set_state(self._h, _dp(s))

    def mass(self) -> np.ndarray:
        """sum over fluid nodes of c1, c2, c3."""
        f = self.fields()
        fl = self.mask == 0
        return np.array([f[k][fl].sum() for k in ("c1", "c2", "c3")])


FIELDS3 = ("c1", "c2", "c3", "rho", "ux", "uy", "uz", "p", "mu1", "mu2", "mu3")


class OracleLattice3D:
    """One nx-by-ny-by-nz D3Q19 lattice advanced by the FP64 oracle (arrays are
    [nz, ny, nx]; edges = (x-, x+, y-, y+, z-, z+), each periodic, wetting or
    neutral)."""

    def __init__(self, nx: int, ny: int, nz: int, edges=(0, 0, 1, 2, 0, 0), mask=None, params=None):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.shape = (self.nz, self.ny, self.nx)
        self.edges = tuple(int(e) for e in edges)
        e = (ctypes.c_int * 6)(*self.edges)
        self._h = lib().orc3_create(self.nx, self.ny, self.nz, e)
        if not self._h:
            raise ValueError("oracle: invalid lattice size")
        m = np.zeros(self.shape, np.uint8) if mask is None else np.ascontiguousarray(mask, np.uint8)
        assert m.shape == self.shape
        self.mask = m.copy()
        lib().orc3_set_geometry(self._h, self.mask.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)))
        if params is not None:
            self.set_params(params)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc3_destroy(h)
            self._h = None

    def set_params(self, params):
        if not isinstance(params, Params):
            params = make_params(**params)
        self.params = params
        lib().orc3_set_params(self._h, ctypes.byref(params))

    def set_fields(self, c1, c2, ux, uy, uz, p=None):
        arrs = [_f64(a).reshape(self.shape) for a in (c1, c2, ux, uy, uz)]
        pp = _f64(p).reshape(self.shape) if p is not None else None
        rc = lib().orc3_set_fields(self._h, *(_dp(a) for a in arrs), _dp(pp) if pp is not None else None)
        if rc:
            raise RuntimeError("oracle: set_params first")

    def step(self, n: int = 1):
        if lib().orc3_step(self._h, int(n)):
            raise RuntimeError("oracle: set_params first")

    def fields(self) -> dict:
        out = np.zeros((11,) + self.shape)
        lib().orc3_read_fields(self._h, _dp(out))
        return {k: out[i] for i, k in enumerate(FIELDS3)}

    def state(self) -> np.ndarray:
        """Raw state [63, nz, ny, nx]: f1 k=0..18, f2 k=0..18, g k=0..18, then
        c1 ux, c1 uy, c1 uz, c2 ux, c2 uy, c2 uz."""
        out = np.zeros((63,) + self.shape)
        lib().orc3_get_state(self._h, _dp(out))
        return out

    def set_state(self, s):
        s = _f64(s).reshape((63,) + self.shape)
        lib().orc3_set_state(self._h, _dp(s))

    def mass(self) -> np.ndarray:
        """sum over fluid nodes of c1, c2, c3."""
        f = self.fields()
        fl = self.mask == 0
        return np.array([f[k][fl].sum() for k in ("c1", "c2", "c3")])


def lattice3_vectors():
    """D3Q19 velocities e_k (19 x 3), weights w_k and the opposite table of the 3D oracle."""
    e = np.array([[lib().orc3_e(k, a) for a in range(3)] for k in range(19)])
    w = np.array([lib().orc3_w(k) for k in range(19)])
    opp = np.array([lib().orc3_opp(k) for k in range(19)])
    return e, w, opp


def feq3(k, c, mu, eta, u):
    return lib().orc3_feq(k, c, mu, eta, *map(float, u))


def geq3(k, p, rho, u):
    return lib().orc3_geq(k, p, rho, *map(float, u))


def sk3(k, u):
    return lib().orc3_sk(k, *map(float, u))


def src_f3(k, tau, dcu):
    return lib().orc3_src_f(k, tau, *map(float, dcu))


def src_g3(k, taug, u, gr, Ft, Fa):
    a = [_f64(v) for v in (u, gr, Ft, Fa)]
    return lib().orc3_src_g(k, taug, *(_dp(v) for v in a))


def grad3(v):
    v = _f64(v)
    out = np.zeros(3)
    lib().orc3_grad(_dp(v), _dp(out))
    return out


def lap3(v):
    return lib().orc3_lap(_dp(_f64(v)))


# ---- exported per-node formulas (the same C functions the step uses) --------

def lambdas(s12, s13, s23):
    out = np.zeros(4)
    lib().orc_lambdas(s12, s13, s23, _dp(out))
    return out


def chem_pot(lam4, D, c1, c2, lap1, lap2):
    lam4 = _f64(lam4)
    out = np.zeros(3)
    lib().orc_chem_pot(_dp(lam4), D, c1, c2, lap1, lap2, _dp(out))
    return out


def wet_offset(cos12, cos13, cos23, D, c1, c2):
    out = np.zeros(3)
    lib().orc_wet_offset(cos12, cos13, cos23, D, c1, c2, _dp(out))
    return out


def grad9(v):
    v = _f64(v)
    out = np.zeros(2)
    lib().orc_grad(_dp(v), _dp(out))
    return out


def lap9(v):
    v = _f64(v)
    return lib().orc_lap(_dp(v))


def sk(k, ux, uy):
    return lib().orc_sk(k, ux, uy)


def feq(k, c, mu, eta, ux, uy):
    return lib().orc_feq(k, c, mu, eta, ux, uy)


def geq(k, p, rho, ux, uy):
    return lib().orc_geq(k, p, rho, ux, uy)


def src_f(k, tau, dx, dy):
    return lib().orc_src_f(k, tau, dx, dy)


def src_g(k, taug, ux, uy, grx, gry, Ftx, Fty, Fax, Fay):
    return lib().orc_src_g(k, taug, ux, uy, grx, gry, Ftx, Fty, Fax, Fay)


def threads() -> int:
    """OpenMP threads the oracle's passes run on."""
    return lib().orc_threads()


def set_threads(n: int) -> None:
    """Run the oracle's passes on n OpenMP threads (results do not depend on n)."""
    lib().orc_set_threads(int(n))


def mrt_matrices():
    """The MRT moment matrix M and its inverse (reading R8 of tlb_oracle.c)."""
    m = np.zeros(81)
    mi = np.zeros(81)
    lib().orc_mrt_matrix(_dp(m))
    lib().orc_mrt_inverse(_dp(mi))
    return m.reshape(9, 9), mi.reshape(9, 9)


def mrt_relax(f, feq, src, s):
    out = np.zeros(9)
    args = [_f64(a) for a in (f, feq, src, s)]
    lib().orc_mrt_relax(*(_dp(a) for a in args), _dp(out))
    return out


def lattice_vectors():
    L = lib()
    e = np.array([[L.orc_ex(k), L.orc_ey(k)] for k in range(9)])
    w = np.array([L.orc_w(k) for k in range(9)])
    opp = np.array([L.orc_opp(k) for k in range(9)])
    return e, w, opp


# ---- contact-angle measurement, Sec. III.A (P: theta_n = 2 atan(2 H_d / L_s)) --

def drop_geometry(c: np.ndarray, wall_row: int = 0):
    """Spreading length L_s and height H_d of each drop of the field c[ny, nx].

    Reading of the measurement (the paper gives only theta_n = 2 atan(2H/L)):
    the drop is the region c >= 1/2; L_s is the distance between the two
    c = 1/2 crossings along the wall row (linear interpolation in x, periodic
    in x); H_d is the highest c = 1/2 crossing above that base (linear
    interpolation in y per column) plus 1/2, since the half-way wall lies half
    a lattice spacing below the wall row.  Returns a list of (L_s, H_d, x_mid).
    """
    ny, nx = c.shape
    row = c[wall_row]
    ins = row >= 0.5
    if ins.all() or not ins.any():
        return []
    # rotate so that index 0 is outside a drop
    start = int(np.argmin(ins))
    out = []
    x = 0
    r = np.roll(row, -start)
    ri = np.roll(ins, -start)
    while x < nx:
        if not ri[x]:
            x += 1
            continue
        a = x
        while x < nx and ri[x]:
            x += 1
        b = x - 1  # last inside index
        # left crossing between a-1 and a, right between b and b+1
        xl = (a - 1) + (0.5 - r[a - 1]) / (r[a] - r[a - 1])
        rb1 = r[(b + 1) % nx]
        xr = b + (r[b] - 0.5) / (r[b] - rb1)
        Ls = xr - xl
        H = 0.0
        for xx in range(a, b + 1):
            col = np.roll(c[:, (xx + start) % nx], 0)
            y = wall_row
            while y + 1 < ny and col[y + 1] >= 0.5:
                y += 1
            if y + 1 < ny:
                h = y + (col[y] - 0.5) / (col[y] - col[y + 1])
            else:
                h = float(y)
            H = max(H, h - wall_row + 0.5)
        out.append((Ls, H, ((xl + xr) / 2 + start) % nx))
    return out


def film_thickness(c: np.ndarray, x: int, y_top: int) -> float:
    """Thickness of the liquid film on top of a solid in column x (Sec. III.D,
    the film of the impacting drop on the cylinder top).

    Reading of the measurement (the paper names h but not how it is taken):
    the film is the run of nodes above the solid node y_top with c >= 1/2
    (c the order parameter, or sum of order parameters, of the liquid); h is
    its c = 1/2 crossing (linear interpolation in y) minus the half-way wall
    at y_top + 1/2; 0 if the node above the solid is below 1/2; the top row
    bounds the walk (no wrap)."""
    ny = c.shape[0]
    y = y_top + 1
    if not c[y, x] >= 0.5:
        return 0.0
    while y + 1 < ny and c[y + 1, x] >= 0.5:
        y += 1
    top = y + (c[y, x] - 0.5) / (c[y, x] - c[y + 1, x]) if y + 1 < ny else float(y)
    return top - (y_top + 0.5)


def contact_angle_deg(c: np.ndarray, wall_row: int = 0):
    """theta_n = 2 atan(2 H_d / L_s) for each drop (Sec. III.A)."""
    return [np.degrees(2.0 * np.arctan(2.0 * H / Ls)) for Ls, H, _ in drop_geometry(c, wall_row)]
