"""Tet / hex intersection volumes and the coupling matrix G (oracle).

Test infrastructure (oracle): never imported by the library.

Sec. 5.1: for piecewise-constant spaces on the tet mesh T_h and on the
embedding grid, the coupling entries are g_{tau, c} = int_{tau cap c}
phi_tau phi_c dx with phi = 1 on its element, i.e. the volume of tau cap c.
Sec. 5.2 builds these from a mesh of the intersection and a quadrature
rule; for P0 x P0 the quadrature of 1 over the intersection is its volume,
which this module computes directly.

Method (chosen to be plainly checkable, and unrelated to the device
kernel): the intersection of the tet and the box is a convex polytope.  Each
of its vertices is the meet of three facet planes, so it is one of
  (a) a tet vertex lying in the box,
  (b) a box corner lying in the tet,
  (c) a tet edge crossing a box face plane inside that face,
  (d) a box edge crossing a tet face plane inside the tet.
The volume is that of the convex hull of these points (Qhull), zero when
they span no volume.
"""
import itertools
import math

import numpy as np
from scipy.spatial import ConvexHull, QhullError

_TET_EDGES = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
_TET_FACES = [(1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2)]


def tet_volume(p):
    p = np.asarray(p, dtype=np.float64)
    return abs(np.linalg.det(np.stack([p[1] - p[0], p[2] - p[0], p[3] - p[0]]))) / 6.0


def _barycentric(p, x):
    """Barycentric coordinates of points x [m,3] in tet p [4,3]."""
    t = np.stack([p[1] - p[0], p[2] - p[0], p[3] - p[0]], axis=1)
    lam = np.linalg.solve(t, (x - p[0]).T).T
    return np.concatenate([1.0 - lam.sum(axis=1, keepdims=True), lam], axis=1)


def _face_planes(p):
    """Unit outward normals [4,3] and offsets [4] of the faces of tet p."""
    cen = p.mean(axis=0)
    nrm = np.zeros((4, 3))
    off = np.zeros(4)
    for f, (a, b, c) in enumerate(_TET_FACES):
        v = np.cross(p[b] - p[a], p[c] - p[a])
        v = v / np.linalg.norm(v)
        if v @ (cen - p[a]) > 0.0:
            v = -v
        nrm[f] = v
        off[f] = v @ p[a]
    return nrm, off


def _merge_coincident(pts, tol=1e-14):
    """Keep one point of every group of (numerically) coincident points.

    The candidate list repeats vertices that several facet triples define
    (a tet vertex on a box face is also an edge/plane meet).  The polytope's
    vertex set does not change, but Qhull can stall on exact duplicates.
    """
    keep = []
    for x in pts:
        if not any(np.max(np.abs(x - y)) <= tol for y in keep):
            keep.append(x)
    return np.array(keep)


def tet_box_volume(p, lo, hi, eps=1e-12):
    """Exact volume of tet p [4,3] intersected with the box [lo, hi]."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    # work in coordinates centred on the box and scaled to O(1)
    c = 0.5 * (lo + hi)
    s = float(np.max(hi - lo))
    q = (np.asarray(p, dtype=np.float64) - c) / s
    blo = (lo - c) / s
    bhi = (hi - c) / s
    pts = []
    inside_box = lambda x: np.all((x >= blo - eps) & (x <= bhi + eps), axis=-1)
    # (a) tet vertices in the box
    pts.extend(q[inside_box(q)])
    # membership of the tet by signed distances to its four face planes (unit
    # normals, pointing out), which stay accurate for flat tets where
    # barycentric coordinates lose digits
    fn, fo = _face_planes(q)
    inside_tet = lambda x: np.all(np.atleast_2d(x) @ fn.T - fo <= eps, axis=-1)
    # (b) box corners in the tet
    corners = np.array(list(itertools.product(*zip(blo, bhi))))
    pts.extend(corners[inside_tet(corners)])
    # (c) tet edges against box face planes
    for a, b in _TET_EDGES:
        pa, pb = q[a], q[b]
        for ax in range(3):
            den = pb[ax] - pa[ax]
            if den == 0.0:
                continue
            for plane in (blo[ax], bhi[ax]):
                t = (plane - pa[ax]) / den
                if -eps <= t <= 1.0 + eps:
                    x = pa + t * (pb - pa)
                    x[ax] = plane
                    if inside_box(x):
                        pts.append(x)
    # (d) box edges against tet face planes
    for fa, fb, fc in _TET_FACES:
        nrm = np.cross(q[fb] - q[fa], q[fc] - q[fa])
        off = nrm @ q[fa]
        for ax in range(3):
            if nrm[ax] == 0.0:
                continue
            o1, o2 = [d for d in range(3) if d != ax]
            for v1 in (blo[o1], bhi[o1]):
                for v2 in (blo[o2], bhi[o2]):
                    x = np.zeros(3)
                    x[o1] = v1
                    x[o2] = v2
                    x[ax] = (off - nrm[o1] * v1 - nrm[o2] * v2) / nrm[ax]
                    if blo[ax] - eps <= x[ax] <= bhi[ax] + eps:
                        if inside_tet(x[None, :])[0]:
                            pts.append(x)
    pts = _merge_coincident(np.array(pts))
    if len(pts) < 4:
        return 0.0
    try:
        vol = ConvexHull(pts).volume
    except QhullError:
        return 0.0
    return vol * s ** 3


def coupling_rows(xyz, tets, n, lo=0.0, h=None, rows=None):
    """Rows of G for the listed tets: dict tet -> {cell: volume}.

    The grid has n cells per axis (one number, a cube) or (nx, ny, nz) cells
    (a box) of edge h from lo; cell (i,j,k) has flat index i + nx (j + ny k).
    Candidate cells are those whose closed box meets the tet's bounding box.
    """
    ext = np.broadcast_to(np.asarray(n, dtype=np.int64), (3,))
    h = (1.0 / ext[0]) if h is None else h
    lo = np.broadcast_to(np.asarray(lo, dtype=np.float64), (3,))
    rows = range(len(tets)) if rows is None else rows
    out = {}
    for t in rows:
        p = xyz[tets[t]]
        a = np.clip(np.floor((p.min(axis=0) - lo) / h).astype(int), 0, ext - 1)
        b = np.clip(np.floor((p.max(axis=0) - lo) / h).astype(int), 0, ext - 1)
        row = {}
        for k in range(a[2], b[2] + 1):
            for j in range(a[1], b[1] + 1):
                for i in range(a[0], b[0] + 1):
                    blo = lo + h * np.array([i, j, k])
                    v = tet_box_volume(p, blo, blo + h)
                    if v > 0.0:
                        row[int(i + ext[0] * (j + ext[1] * k))] = v
        out[int(t)] = row
    return out


# ---------------------------------------------------------------------------
# Second statement: exact rational arithmetic by half-space splitting.
#
# The box is the intersection of six half-spaces {s (x_a - b) <= 0}.  Cutting
# a tet by one half-space leaves, depending on how many of its vertices lie
# strictly outside, nothing, the whole tet, a corner tet (one vertex inside),
# a prism (three inside) or a wedge (two inside); prisms and wedges are split
# into three tets along a staircase of diagonals.  After the six cuts the
# intersection is a union of tets with disjoint interiors, and its volume is
# the sum of |det| / 6.  With every coordinate a Fraction (a float converts
# exactly) each cut point is exact, so the result is the exact volume of the
# intersection of the input tet with the input box: no tolerance, no
# rounding.  Slow (big rationals), meant for slivers and small cases.
# ---------------------------------------------------------------------------
from fractions import Fraction


def _exact_point(p):
    return tuple(Fraction(v) for v in p)


def _cut_halfspace(tets, ax, bound, sign):
    """The parts of `tets` in {sign * (x[ax] - bound) <= 0}, as tets."""
    out = []
    for t in tets:
        d = [sign * (p[ax] - bound) for p in t]
        outside = [i for i in range(4) if d[i] > 0]
        if not outside:
            out.append(t)
            continue
        inside = [i for i in range(4) if d[i] <= 0]
        if not any(d[i] < 0 for i in inside):  # what is left lies in the plane: no volume
            continue

        def meet(i, o):
            a, b = t[i], t[o]
            s = d[i] / (d[i] - d[o])
            q = [a[k] + s * (b[k] - a[k]) for k in range(3)]
            q[ax] = bound
            return tuple(q)

        if len(inside) == 1:
            v = inside[0]
            out.append((t[v],) + tuple(meet(v, o) for o in outside))
        elif len(inside) == 3:
            o = outside[0]
            v1, v2, v3 = (t[i] for i in inside)
            p1, p2, p3 = (meet(i, o) for i in inside)
            # prism v1 v2 v3 / p1 p2 p3 (p_k above v_k)
            out += [(v1, v2, v3, p1), (v2, v3, p1, p2), (v3, p1, p2, p3)]
        else:
            (i1, i2), (o1, o2) = inside, outside
            v1, v2 = t[i1], t[i2]
            p11, p12, p21, p22 = meet(i1, o1), meet(i1, o2), meet(i2, o1), meet(i2, o2)
            # wedge: triangle v1 p11 p12 above triangle v2 p21 p22
            out += [(v1, p11, p12, v2), (p11, p12, v2, p21), (p12, v2, p21, p22)]
    return out


def _det6(t):
    a, b, c, d = t
    u = [b[k] - a[k] for k in range(3)]
    v = [c[k] - a[k] for k in range(3)]
    w = [d[k] - a[k] for k in range(3)]
    return (u[0] * (v[1] * w[2] - v[2] * w[1]) - u[1] * (v[0] * w[2] - v[2] * w[0])
            + u[2] * (v[0] * w[1] - v[1] * w[0]))


def tet_volume_exact(p):
    """|tau| as a Fraction."""
    return abs(_det6([_exact_point(q) for q in p])) / 6


def tet_box_volume_exact(p, lo, hi):
    """Exact |tet cap box| as a Fraction; p [4][3] floats or Fractions, lo/hi
    the box corners (floats or Fractions, taken exactly)."""
    pieces = [tuple(_exact_point(q) for q in p)]
    lo = [Fraction(v) for v in lo]
    hi = [Fraction(v) for v in hi]
    for ax in range(3):
        pieces = _cut_halfspace(pieces, ax, lo[ax], -1)
        pieces = _cut_halfspace(pieces, ax, hi[ax], 1)
        if not pieces:
            return Fraction(0)
    return sum((abs(_det6(t)) for t in pieces), Fraction(0)) / 6


def coupling_rows_exact(xyz, tets, n, lo=0.0, h=None, rows=None):
    """Rows of G in exact arithmetic: dict tet -> {cell: Fraction}.

    Same grid and candidate-cell conventions as coupling_rows; the cell of
    index (i, j, k) is the box lo + h [i, i+1] x [j, j+1] x [k, k+1] with lo
    and h taken exactly (h = 1 / nx when not given)."""
    ext = np.broadcast_to(np.asarray(n, dtype=np.int64), (3,))
    hF = Fraction(1, int(ext[0])) if h is None else Fraction(h)
    loF = [Fraction(v) for v in np.broadcast_to(np.asarray(lo, dtype=np.float64), (3,))]
    rows = range(len(tets)) if rows is None else rows
    out = {}
    for t in rows:
        p = [_exact_point(q) for q in np.asarray(xyz)[np.asarray(tets)[t]]]
        rng_ = []
        for ax in range(3):
            mn = min(q[ax] for q in p)
            mx = max(q[ax] for q in p)
            a = max(0, min(int(ext[ax]) - 1, math.floor((mn - loF[ax]) / hF)))
            b = max(0, min(int(ext[ax]) - 1, math.floor((mx - loF[ax]) / hF)))
            rng_.append((a, b))
        row = {}
        for k in range(rng_[2][0], rng_[2][1] + 1):
            for j in range(rng_[1][0], rng_[1][1] + 1):
                for i in range(rng_[0][0], rng_[0][1] + 1):
                    blo = [loF[0] + i * hF, loF[1] + j * hF, loF[2] + k * hF]
                    v = tet_box_volume_exact(p, blo, [x + hF for x in blo])
                    if v > 0:
                        row[int(i + ext[0] * (j + ext[1] * k))] = v
        out[int(t)] = row
    return out
