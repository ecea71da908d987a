"""A quarter-cylinder tet mesh with strongly stretched elements.

Stand-in for the paper's crooked-pipe mesh (Sec. 7.1: a quarter cylinder of
radius 2 and height 7 embedded in the box (0,3) x (0,3) x (0,8), meshed with
highly stretched elements that resolve a boundary layer between two material
subdomains; the mesh itself is not available).

Construction: a structured polar lattice (r_i, theta_j, z_k).  The radial
spacing shrinks geometrically toward r = `layer` from both sides (the
boundary layer), theta and z are uniform, so cells near the layer are thin in
r and long in z.  Cells away from the axis are split into the six Kuhn tets
of their (i, j, k) lattice cube; the cells touching the axis are wedges split
into three tets.  Every quad face is cut along the diagonal that runs from the
bottom (lower k) vertex of lower lattice index to the top vertex of higher
index, which is the diagonal the Kuhn split uses, so the mesh is conforming.
The union of the tets is the prism over the polygon through the outer ring
vertices: its volume is height * nt * R^2 sin(pi / (2 nt)) / 2.
"""
from itertools import permutations

import numpy as np


def radial_nodes(nr, radius=2.0, layer=1.0, q=0.8):
    """nr + 1 radii from 0 to radius; cell widths shrink by the factor q toward
    r = layer from both sides (nr // 2 cells inside the layer, the rest outside)."""
    ni = nr // 2
    no = nr - ni
    wi = q ** np.arange(ni)        # from the axis outward, smallest next to the layer
    wi = wi * layer / wi.sum()
    wo = q ** np.arange(no)[::-1]  # from the layer outward, smallest next to the layer
    wo = wo * (radius - layer) / wo.sum()
    r = np.concatenate([[0.0], np.cumsum(wi), layer + np.cumsum(wo)])
    r[ni] = layer
    r[-1] = radius
    return r


def quarter_cylinder_mesh(nr, nt, nz, radius=2.0, height=7.0, axis=(0.5, 0.5), z0=0.5, layer=1.0, q=0.8):
    """Return (xyz float64 [nv, 3], tets int32 [nt, 4]), every tet positively oriented.

    The cylinder's axis is the line x = axis[0], y = axis[1]; it spans angles
    0 .. pi/2 (x, y >= the axis) and z0 .. z0 + height.  With the defaults it
    lies in (0.5, 2.5)^2 x (0.5, 7.5), inside the paper's box (0,3)^2 x (0,8).
    """
    r = radial_nodes(nr, radius, layer, q)
    th = np.linspace(0.0, 0.5 * np.pi, nt + 1)
    z = z0 + height * np.arange(nz + 1) / nz
    z[-1] = z0 + height
    c, s = np.cos(th), np.sin(th)
    c[-1], s[0] = 0.0, 0.0  # the two flat sides are exact planes
    s[-1], c[0] = 1.0, 1.0
    # vertex ids: axis vertex of level k -> k; ring vertex (i >= 1, j, k) -> na + (i-1) + nr (j + (nt+1) k)
    na = nz + 1
    axis_xyz = np.stack([np.full(na, axis[0]), np.full(na, axis[1]), z], axis=1)
    kk, jj, ii = np.meshgrid(np.arange(nz + 1), np.arange(nt + 1), np.arange(1, nr + 1), indexing="ij")
    ring_xyz = np.stack([axis[0] + r[ii] * c[jj], axis[1] + r[ii] * s[jj], z[kk]], axis=-1).reshape(-1, 3)
    xyz = np.concatenate([axis_xyz, ring_xyz])

    def vid(i, j, k):
        return np.where(i == 0, k, na + (i - 1) + nr * (j + (nt + 1) * k))

    tets = []
    # wedges next to the axis: bottom (a, p, q), top (a', p', q'); diagonals a-p', a-q', p-q'
    kw, jw = np.meshgrid(np.arange(nz), np.arange(nt), indexing="ij")
    kw, jw = kw.ravel(), jw.ravel()
    zero = np.zeros_like(kw)
    a, a1 = vid(zero, jw, kw), vid(zero, jw, kw + 1)
    p, p1 = vid(zero + 1, jw, kw), vid(zero + 1, jw, kw + 1)
    qq, q1 = vid(zero + 1, jw + 1, kw), vid(zero + 1, jw + 1, kw + 1)
    tets += [np.stack(t, axis=1) for t in ((a, p, qq, q1), (a, p, p1, q1), (a, a1, p1, q1))]
    # Kuhn split of the lattice cubes (i .. i+1, j .. j+1, k .. k+1), i >= 1
    kc, jc, ic = np.meshgrid(np.arange(nz), np.arange(nt), np.arange(1, nr), indexing="ij")
    kc, jc, ic = kc.ravel(), jc.ravel(), ic.ravel()
    for perm in permutations(range(3)):
        d = np.zeros((4, 3), dtype=np.int64)
        d[1, perm[0]] = 1
        d[2, perm[0]] = 1
        d[2, perm[1]] = 1
        d[3] = 1
        tets.append(np.stack([vid(ic + d[v, 0], jc + d[v, 1], kc + d[v, 2]) for v in range(4)], axis=1))
    tets = np.concatenate(tets).astype(np.int64)
    pts = xyz[tets]
    vol = np.einsum("ij,ij->i", np.cross(pts[:, 1] - pts[:, 0], pts[:, 2] - pts[:, 0]), pts[:, 3] - pts[:, 0])
    flip = vol < 0
    tets[flip, 2], tets[flip, 3] = tets[flip, 3].copy(), tets[flip, 2].copy()
    return xyz, tets.astype(np.int32)


def polygon_prism_volume(nt, radius=2.0, height=7.0):
    """Volume of the union of the mesh's tets (the prism over the outer-ring polygon)."""
    return height * nt * 0.5 * radius ** 2 * np.sin(0.5 * np.pi / nt)
