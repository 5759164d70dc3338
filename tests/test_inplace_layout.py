"""The in-place (AA-pattern) streaming layout, emulated on the CPU.

A small model of the addressing the in-place kernels use (even steps: a node
reads its own slots k and writes f'_k into its own slot k-bar; odd steps: it
reads slot k-bar of x - e_k, or its own slot k across a wall link, and writes
slot k of x + e_k, or its own slot k-bar across a wall link, zero across a lid
link; a call ending on an even step streams by pairwise swaps) is checked
against the two-buffer push with half-way bounce-back (Eq. 44) on random
geometries: after 1 to 5 steps of an arbitrary local linear collision the two
layouts hold the same populations, and within a step every location is read
by at most one node and written by at most one node, the same one (so the
update is race-free in one buffer).
"""
import numpy as np
import pytest

EX = [0, 1, 0, -1, 0, 1, -1, -1, 1]
EY = [0, 0, 1, 0, -1, 1, 1, -1, -1]
OPP = [0, 3, 4, 1, 2, 7, 8, 5, 6]
FLUID, LID, WET, NEU, VOID = 0, 1, 2, 3, 4
PERIODIC, WETTING, NEUTRAL, LIDEDGE = 0, 1, 2, 3


def site(kind, edges, x, y):
    ny, nx = kind.shape
    if x < 0 or x >= nx:
        e = edges[0 if x < 0 else 1]
        if e != PERIODIC:
            return (WET if e == WETTING else NEU), None
        x %= nx
    if y < 0 or y >= ny:
        e = edges[2 if y < 0 else 3]
        if e == LIDEDGE:
            return VOID, None
        if e != PERIODIC:
            return (WET if e == WETTING else NEU), None
        y %= ny
    return kind[y, x], (y, x)


def fluidlike(s):
    return s in (FLUID, LID)


def two_buffer(f, kind, edges, M, n):
    ny, nx = kind.shape
    for _ in range(n):
        B = np.zeros_like(f)
        for y in range(ny):
            for x in range(nx):
                if not fluidlike(kind[y, x]):
                    continue
                o = M @ f[:, y, x]
                B[0, y, x] = o[0]
                for k in range(1, 9):
                    s, d = site(kind, edges, x + EX[k], y + EY[k])
                    if fluidlike(s):
                        B[k, d[0], d[1]] = o[k]
                    elif s in (WET, NEU):
                        B[OPP[k], y, x] = o[k]
        f = B
    return f


def in_place(f, kind, edges, M, n):
    ny, nx = kind.shape
    f = f.copy()
    for step in range(n):
        odd = step & 1
        new = f.copy()
        reader, writer = {}, {}
        for y in range(ny):
            for x in range(nx):
                if not fluidlike(kind[y, x]):
                    continue
                v = np.zeros(9)
                for k in range(9):
                    loc = (k, y, x)
                    if odd and k:
                        s, d = site(kind, edges, x - EX[k], y - EY[k])
                        loc = (OPP[k], d[0], d[1]) if fluidlike(s) else ((k, y, x) if s in (WET, NEU) else None)
                    if loc is not None:
                        assert loc not in reader
                        reader[loc] = (y, x)
                        v[k] = f[loc]
                o = M @ v
                for k in range(9):
                    loc, val = (OPP[k], y, x), o[k]
                    if odd and k:
                        s, d = site(kind, edges, x + EX[k], y + EY[k])
                        if fluidlike(s):
                            loc = (k, d[0], d[1])
                        elif s == VOID:
                            val = 0.0
                    assert loc not in writer
                    writer[loc] = (y, x)
                    new[loc] = val
        for loc, who in writer.items():
            assert reader.get(loc, who) == who, loc  # read and written by one node only
        f = new
        if not odd and step == n - 1:  # streaming of the even layout: pairwise swaps
            g = f.copy()
            for y in range(ny):
                for x in range(nx):
                    if not fluidlike(kind[y, x]):
                        continue
                    for k in range(1, 9):
                        s, d = site(kind, edges, x + EX[k], y + EY[k])
                        if fluidlike(s) and k in (1, 2, 5, 6):
                            g[OPP[k], y, x], g[k, d[0], d[1]] = f[k, d[0], d[1]], f[OPP[k], y, x]
                        elif s == VOID:
                            g[OPP[k], y, x] = 0.0
            f = g
    return f


@pytest.mark.parametrize("trial", range(10))
def test_in_place_layout_equals_two_buffer_push(trial):
    rng = np.random.default_rng(100 + trial)
    nx, ny = int(rng.integers(3, 8)), int(rng.integers(6, 9))
    edges = [(0, 0, 1, 3), (0, 0, 0, 0), (2, 1, 1, 2), (0, 0, 2, 3), (1, 2, 0, 0)][trial % 5]
    kind = np.zeros((ny, nx), int)
    kind[rng.random((ny, nx)) < 0.15] = WET
    if edges[3] == LIDEDGE:
        kind[-2:, :] = FLUID
        kind[-1, :] = LID
    f0 = rng.random((9, ny, nx))
    f0[:, ~np.isin(kind, [FLUID, LID])] = 0
    if edges[3] == LIDEDGE:  # nothing enters the lid row from beyond the lid
        for k in range(1, 9):
            if EY[k] == -1:
                f0[k, -1, :] = 0
    M = rng.random((9, 9)) * 0.3
    fluid = np.isin(kind, [FLUID, LID])
    for n in (1, 2, 3, 4, 5):
        a = two_buffer(f0, kind, edges, M, n)
        b = in_place(f0, kind, edges, M, n)
        assert np.abs(a[:, fluid] - b[:, fluid]).max() < 1e-12, (n, edges)
