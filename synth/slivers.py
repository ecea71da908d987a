"""Seeded near-degenerate tets (slivers) placed across the planes of a grid.

A jittered Kuhn mesh produces, now and then, tets whose volume is a tiny
fraction of their edge length cubed; the clipping that builds the coupling
matrix (Sec. 5.2) must get their intersection volumes right.  These
generators make such tets on purpose, each one on its own (a tet soup, not a
conforming mesh), with edges of one to three grid cells so that they cross
one to three grid planes per axis:

  flat    four nearly coplanar vertices, all edges long (a "proper" sliver):
          (+-L, 0, -d), (0, +-L, d) in a local frame, volume 4 L^2 d / 3
  needle  one long edge and a thin cross-section: (0,0,0), (l,0,0),
          (x1, e, 0), (x2, 0, e), volume l e^2 / 6
  cap     a large triangle and a fourth vertex just above it, volume A d / 3

then rotated by a random orthogonal matrix and moved to a random point of
the grid, all drawn from NumPy's PCG64.  `plane_tets` adds tets with a face
on, or within a given offset of, a grid plane.
"""
import numpy as np


def _rotation(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def _local_sliver(kind, vol, h, rng):
    if kind == "flat":
        L = rng.uniform(1.0, 1.5) * h
        d = 3.0 * vol / (4.0 * L * L)
        return np.array([[-L, 0.0, -d], [L, 0.0, -d], [0.0, -L, d], [0.0, L, d]])
    if kind == "needle":
        ln = rng.uniform(2.0, 3.0) * h
        e = np.sqrt(6.0 * vol / ln)
        x1, x2 = rng.uniform(0.2, 0.8, size=2) * ln
        return np.array([[0.0, 0.0, 0.0], [ln, 0.0, 0.0], [x1, e, 0.0], [x2, 0.0, e]]) - np.array([ln / 2, 0, 0])
    if kind == "cap":
        L = rng.uniform(1.0, 1.5) * h
        tri = np.array([[-L, -L, 0.0], [L, -0.5 * L, 0.0], [0.0, L, 0.0]])
        area = 0.5 * abs(np.cross(tri[1] - tri[0], tri[2] - tri[0])[2])
        d = 3.0 * vol / area
        w = rng.dirichlet(np.ones(3))
        apex = w @ tri + np.array([0.0, 0.0, d])
        return np.vstack([tri, apex])
    raise ValueError(kind)


def sliver_tets(n, rel_volumes=(1e-3, 1e-5, 1e-8), kinds=("flat", "needle", "cap"), per_case=4, seed=11,
                lo=0.0, size=1.0):
    """(xyz [4T, 3], tets [T, 4] int32, target volumes [T]) for a grid of n cells
    per axis on [lo, lo + size]^3: per_case tets of every (kind, relative volume),
    the relative volume in units of h^3."""
    rng = np.random.default_rng(seed)
    h = size / n
    pts, target = [], []
    for kind in kinds:
        for rv in rel_volumes:
            for _ in range(per_case):
                loc = _local_sliver(kind, rv * h ** 3, h, rng) @ _rotation(rng).T
                ext = np.abs(loc).max()
                c = rng.uniform(lo + ext + h, lo + size - ext - h, size=3)
                pts.append(loc + c)
                target.append(rv * h ** 3)
    xyz = np.concatenate(pts)
    tets = np.arange(len(xyz), dtype=np.int32).reshape(-1, 4)
    return xyz, tets, np.array(target)


def plane_tets(n, offsets=(0.0, 1e-13, -1e-13, 3e-14), heights=(0.8, 1e-5), seed=12, lo=0.0, size=1.0):
    """Tets with three vertices on the plane x_a = (grid plane) + offset * h, for
    every axis a, offset and height of the fourth vertex (in units of h, on
    either side); the face's other coordinates and the apex are drawn so that
    the tet crosses grid planes of the other two axes."""
    rng = np.random.default_rng(seed)
    h = size / n
    pts = []
    for ax in range(3):
        o1, o2 = [a for a in range(3) if a != ax]
        for off in offsets:
            for ht in heights:
                for side in (1.0, -1.0):
                    plane = lo + h * rng.integers(3, n - 3) + off * h
                    base = rng.uniform(lo + 3 * h, lo + size - 3 * h, size=2)
                    tri = np.zeros((3, 3))
                    for v in range(3):
                        ang = 2.0 * np.pi * v / 3.0 + rng.uniform(-0.3, 0.3)
                        r = rng.uniform(1.0, 1.8) * h
                        tri[v, o1] = base[0] + r * np.cos(ang)
                        tri[v, o2] = base[1] + r * np.sin(ang)
                        tri[v, ax] = plane
                    apex = np.zeros(3)
                    apex[[o1, o2]] = base + rng.uniform(-0.5, 0.5, size=2) * h
                    apex[ax] = plane + side * ht * h
                    pts.append(np.vstack([tri, apex]))
    xyz = np.concatenate(pts)
    tets = np.arange(len(xyz), dtype=np.int32).reshape(-1, 4)
    return xyz, tets
