"""Norms shared by the GPU parity tests (the CUDA path against the FP64
oracle, element by element on the same seeded inputs).

Fields: the relative max-norm of a field is
max|gpu - oracle| / max(max|oracle|, floor), with a scale floor per field:
1 for c_i and rho, 1e-4 for u, max sigma / 32 for p (the Laplace jump of a
radius-32 drop) and max sigma / D for mu_i.  mu (Eq. 8) is the difference of
two terms of size ~ 12 lambda/D c(1-c)(1-2c) and 3/4 D lambda lap c that
cancel at equilibrium, so its round-off is set by those terms, not by |mu|.

Raw state: every one of the 31 planes (f^1_k, f^2_k, g_k for k = 0..8, then
c1 ux, c1 uy, c2 ux, c2 uy of Eq. 19) is compared element by element and
judged against the scale of its group of planes,
max|gpu_q - oracle_q| / s_G, s_G = the largest |oracle| value in the group:
the rest populations f^i_0 (O(1), about c_i); the moving populations f^i_{k>0}
and all g_k (O(mu, c u, p), some 1e-5..1e-3); the c_i u planes.  That is the
scale round-off has in each group: a moving population is computed from
equilibrium, source and relaxation terms whose size is the size of the
group's populations (a diagonal direction differs only by its weight, a
direction against the flow by the sign of e.u), and the errors of c, mu and u
enter it scaled the same way.  One exception: the MRT collision transforms
every distribution to moments that include the O(1) rest population (the
energy moments weigh f_0 by -4 and 4), so its moving populations carry the
rest populations' absolute round-off, and their group is judged against the
rest scale.  Compared with one scale for all 31 planes (set by the O(1) rest
populations), this checks the moving and c_i u planes 1e3-1e5 times more
tightly.
"""
import numpy as np

FIELDS = ("c1", "c2", "c3", "rho", "ux", "uy", "p", "mu1", "mu2", "mu3")
FIELDS3 = ("c1", "c2", "c3", "rho", "ux", "uy", "uz", "p", "mu1", "mu2", "mu3")
FLOOR = dict(c1=1.0, c2=1.0, c3=1.0, rho=1.0, ux=1e-4, uy=1e-4, uz=1e-4)
TOL64 = 1e-12

REST = (0, 9)
MOVING = tuple(q for q in range(27) if q not in REST)
CU = (27, 28, 29, 30)
# the D3Q19 state: 57 distribution planes (rest populations at 0 and 19), 6 c_i u planes
GROUPS3 = ((0, 19), tuple(q for q in range(57) if q not in (0, 19)), tuple(range(57, 63)))


def floors(params):
    smax = max(params["sigma12"], params["sigma13"], params["sigma23"])
    return dict(FLOOR, p=smax / 32, mu1=smax / params["D"], mu2=smax / params["D"], mu3=smax / params["D"])


def assert_oracle_parity3(L, O, params, tol=TOL64, what=""):
    """FP64 D3Q19 lattice L against the 3D oracle O: every field and every
    raw-state plane within `tol`."""
    errs = field_errors(L.fields(), O.fields(), params, FIELDS3)
    bad = {k: v for k, v in errs.items() if not v < tol}
    assert not bad, f"{what} field errors above {tol}: {bad}"
    se, q = state_error(L.state(), O.state(), False, GROUPS3)
    assert se < tol, f"{what} raw state error {se:.3e} in plane {q}"


def relnorm(a, b, floor):
    return float(np.abs(a - b).max() / max(float(np.abs(b).max()), floor))


def field_errors(fg, fo, params, names=FIELDS):
    fl = floors(params)
    return {k: relnorm(fg[k], fo[k], fl[k]) for k in names}


def plane_errors(sg, so, mrt=False, groups=(REST, MOVING, CU)):
    """Per-plane errors of two raw states [planes][...] against their group
    scales (see the module docstring; `groups` = rest, moving, c_i u planes,
    the D2Q9 layout by default, GROUPS3 for D3Q19); returns one error per
    plane."""
    rest, moving, cu = groups
    scale = {g: max(float(np.abs(so[list(g)]).max()), 1e-300) for g in (rest, moving, cu)}
    if mrt:
        scale[moving] = max(scale[moving], scale[rest])
    err = np.zeros(len(rest) + len(moving) + len(cu))
    for g, s_g in scale.items():
        for q in g:
            err[q] = float(np.abs(sg[q] - so[q]).max()) / s_g
    return err


def state_error(sg, so, mrt=False, groups=(REST, MOVING, CU)):
    """Largest per-plane error and the plane it occurs in."""
    e = plane_errors(sg, so, mrt, groups)
    q = int(np.argmax(e))
    return float(e[q]), q


def is_mrt(params):
    return float(params.get("collision", 0.0)) == 1.0


def assert_oracle_parity(L, O, params, tol=TOL64, what=""):
    """FP64 lattice L against oracle O: every field and every raw-state plane
    within `tol`."""
    errs = field_errors(L.fields(), O.fields(), params)
    bad = {k: v for k, v in errs.items() if not v < tol}
    assert not bad, f"{what} field errors above {tol}: {bad}"
    se, q = state_error(L.state(), O.state(), is_mrt(params))
    assert se < tol, f"{what} raw state error {se:.3e} in plane {q}"


# Bounds of the reduced-precision paths against the oracle: field ->
# (kind, bound), "abs" absolute, "rel" relative to max|oracle| (about ten times
# what was measured on GB300 for FP32 and FP16, three times for BF16; the BF16
# order-parameter bound is the FP16 one times 2^3, the ratio of the two
# formats' unit roundoffs, 8 against 11 significand bits).  The density error
# is taken relative to the largest density, since it is the order-parameter
# error scaled by the density contrast (Eq. 14).
BOUNDS = {
    "fp32": dict(c1=("abs", 2e-4), c2=("abs", 2e-4), c3=("abs", 2e-4), rho=("rel", 1e-3),
                 ux=("rel", 1e-3), uy=("rel", 1e-3), p=("rel", 1e-3), mu1=("rel", 2e-2), mu2=("rel", 2e-2)),
    "fp16": dict(c1=("abs", 2e-4), c2=("abs", 2e-4), c3=("abs", 2e-4), rho=("rel", 2e-4),
                 ux=("rel", 3e-2), uy=("rel", 3e-2), p=("rel", 6e-2), mu1=("rel", 6e-3), mu2=("rel", 6e-3)),
    "bf16": dict(c1=("abs", 1.6e-3), c2=("abs", 1.6e-3), c3=("abs", 1.6e-3), rho=("rel", 1e-3),
                 ux=("rel", 6e-2), uy=("rel", 6e-2), p=("rel", 0.16), mu1=("rel", 5e-2), mu2=("rel", 5e-2)),
}


def bounded_errors(fg, fo, precision):
    """{field: (error, bound)} of a reduced-precision result against the oracle."""
    out = {}
    for k, (kind, bound) in BOUNDS[precision].items():
        err = float(np.abs(fg[k] - fo[k]).max())
        if kind == "rel":
            err /= max(float(np.abs(fo[k]).max()), 1e-12)
        out[k] = (err, bound)
    return out


def assert_bounded(fg, fo, precision, what=""):
    bad = {k: v for k, v in bounded_errors(fg, fo, precision).items() if not v[0] < v[1]}
    assert not bad, f"{what} {precision}: errors above bounds {bad}"
