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
    # (b) box corners in the tet
    corners = np.array(list(itertools.product(*zip(blo, bhi))))
    bc = _barycentric(q, corners)
    pts.extend(corners[np.all(bc >= -eps, axis=1)])
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
                        if np.all(_barycentric(q, x[None, :])[0] >= -eps):
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
