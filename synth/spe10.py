"""An SPE10-sized box meshed by stretched Cartesian hexahedra, each split into tets.

Stand-in for the paper's second domain (Sec. 7.2): the box of Model 2 of the
tenth SPE comparative solution project, 1200 x 2220 x 170 ft, meshed with
hexahedra and embedded in a 1600 x 2420 x 240 ft bounding box.  The reservoir
data are not available and are not needed by the sampler; only the geometry
is reproduced.  The default hex counts 60 x 220 x 85 give the SPE10 cell size
of 20 x 10 x 2 ft (aspect ratio 10).

The sampler's target meshes are tetrahedral, so each hexahedron is split into
the six tets around its v0 -> v7 diagonal (the Kuhn split, conforming across
hexes); the projection onto a hexahedron is the volume-weighted mean of its
six tets' projections before the exponential.  The vertices are not jittered:
the SPE10 grid is Cartesian.
"""
from itertools import permutations

import numpy as np

SPE10_DOMAIN = (1200.0, 2220.0, 170.0)
SPE10_BOUNDING_BOX = (1600.0, 2420.0, 240.0)
SPE10_CELLS = (60, 220, 85)


def cartesian_kuhn_mesh(lo, hi, counts):
    """Return (xyz float64 [nv, 3], tets int32 [6 nx ny nz, 4]) for the box lo..hi cut into
    counts = (nx, ny, nz) equal hexahedra, six positively oriented tets per hexahedron
    (hexes x fastest, then y, then z; vertex (i, j, k) has id i + (nx+1)(j + (ny+1) k))."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    nx, ny, nz = (int(c) for c in counts)
    axes = [lo[d] + (hi[d] - lo[d]) * np.arange(c + 1) / c for d, c in enumerate((nx, ny, nz))]
    for d in range(3):
        axes[d][-1] = hi[d]
    kk, jj, ii = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    xyz = np.stack([axes[0][ii], axes[1][jj], axes[2][kk]], axis=-1).reshape(-1, 3)
    ck, cj, ci = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    sx, sy = 1, nx + 1
    sz = (nx + 1) * (ny + 1)
    base = (ci * sx + cj * sy + ck * sz).ravel().astype(np.int64)
    step = (sx, sy, sz)
    tets = []
    for perm in permutations(range(3)):
        a = step[perm[0]]
        b = a + step[perm[1]]
        c = sx + sy + sz
        t = np.stack([base, base + a, base + b, base + c], axis=1)
        tets.append(t)
    tets = np.stack(tets, axis=1).reshape(-1, 4)
    p = xyz[tets]
    vol = np.einsum("ij,ij->i", np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), p[:, 3] - p[:, 0])
    flip = vol < 0
    tets[flip, 2], tets[flip, 3] = tets[flip, 3].copy(), tets[flip, 2].copy()
    return xyz, tets.astype(np.int32)


def spe10_mesh(counts=SPE10_CELLS, domain=SPE10_DOMAIN, bounding_box=SPE10_BOUNDING_BOX):
    """The SPE10 box centred in its bounding box, whose corner is the origin (units: ft)."""
    off = [(b - d) / 2.0 for b, d in zip(bounding_box, domain)]
    return cartesian_kuhn_mesh(off, [o + d for o, d in zip(off, domain)], counts)
