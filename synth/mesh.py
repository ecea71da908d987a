"""Jittered Kuhn-split tet meshes of a box or an L-shaped prism.

The target meshes of the sampler are unstructured tetrahedral meshes of a
domain D that sits inside the structured embedding box (Sec. 4.1, Sec. 5).
The paper's own meshes (crooked pipe, SPE10 box) are not available, so
these seeded stand-ins keep the same structure: a tet mesh that does not
match the hex grid, embedded with a margin, built once and reused.

Construction: D is a union of m^3 axis-aligned cubes of edge ht (all of
them for a box, three quarters of them for the L-prism whose quarter
x > xmid, y > ymid is removed).  Each kept cube is split into the six
tetrahedra around its main diagonal v0 -> v7 (the Kuhn split, conforming
across cubes).  Every vertex strictly inside D is moved by an independent
U(-jitter*ht, +jitter*ht) offset per coordinate; vertices on the boundary
of D (outer faces and the re-entrant faces of the L-prism) stay fixed, so
the jittered tets still tile D exactly.  Tets the jitter inverts or flattens
(volume <= min_rel times the undeformed volume, min_rel = 0 by default) get
their interior vertices redrawn; slivers are kept.
"""
from dataclasses import dataclass
from itertools import permutations

import numpy as np


# Redraw threshold of the jitter, relative to the undeformed Kuhn tet: 0 keeps
# every valid tet (slivers included) and redraws only inverted or flat ones;
# 0.02 was an earlier, gentler default and stays available as an argument.
MIN_REL = 0.0


@dataclass(frozen=True)
class MeshSpec:
    lo: tuple
    hi: tuple
    m: int
    lshape: bool
    jitter: float = 0.25
    seed: int = 1
    min_rel: float = MIN_REL


def _kept_cubes(m, lshape):
    keep = np.ones((m, m, m), dtype=bool)  # indexed [k, j, i] (z, y, x)
    if lshape:
        if m % 2:
            raise ValueError("L-prism needs an even cube count per axis")
        keep[:, m // 2:, m // 2:] = False
    return keep


def kuhn_mesh(spec: MeshSpec):
    """Return (xyz float64 [nv,3], tets int32 [nt,4]) for the given spec.

    Tets are listed cube by cube (x fastest, then y, then z), six per cube,
    each positively oriented before jitter.  Vertex ids are compact and
    follow the lexicographic order of the (m+1)^3 lattice.
    """
    m = int(spec.m)
    lo = np.asarray(spec.lo, dtype=np.float64)
    hi = np.asarray(spec.hi, dtype=np.float64)
    ht = (hi - lo) / m
    keep = _kept_cubes(m, spec.lshape)

    # lattice vertex (i, j, k) -> id  i + (m+1) * (j + (m+1) * k)
    m1 = m + 1
    # number of kept cubes touching each lattice vertex
    touch = np.zeros((m1, m1, m1), dtype=np.int32)
    for dk in (0, 1):
        for dj in (0, 1):
            for di in (0, 1):
                touch[dk:dk + m, dj:dj + m, di:di + m] += keep
    used = touch > 0
    interior = touch == 8

    # jitter drawn for every lattice vertex in lexicographic order so that the
    # mesh does not depend on the compaction below
    rng = np.random.default_rng(spec.seed)
    d = rng.uniform(-spec.jitter, spec.jitter, size=(m1, m1, m1, 3)) * ht
    kk, jj, ii = np.meshgrid(np.arange(m1), np.arange(m1), np.arange(m1), indexing="ij")
    pos = np.stack([lo[0] + ii * ht[0], lo[1] + jj * ht[1], lo[2] + kk * ht[2]], axis=-1)
    pos = np.where(interior[..., None], pos + d, pos)
    # exact boundary coordinates (avoid lo + i*ht rounding on the far faces)
    pos[..., 0][:, :, m] = np.where(interior[:, :, m], pos[..., 0][:, :, m], hi[0])
    pos[..., 1][:, m, :] = np.where(interior[:, m, :], pos[..., 1][:, m, :], hi[1])
    pos[..., 2][m, :, :] = np.where(interior[m, :, :], pos[..., 2][m, :, :], hi[2])

    ck, cj, ci = np.nonzero(keep)
    order = np.lexsort((ci, cj, ck))  # x fastest, then y, then z
    ci, cj, ck = ci[order], cj[order], ck[order]
    base = ci + m1 * (cj + m1 * ck)
    step = np.array([1, m1, m1 * m1], dtype=np.int64)
    tets = []
    for perm in permutations(range(3)):
        a = step[perm[0]]
        b = step[perm[0]] + step[perm[1]]
        c = step[0] + step[1] + step[2]
        # the permutation's sign decides the orientation of (v0, v0+a, v0+b, v7)
        inv = sum(1 for x in range(3) for y in range(x + 1, 3) if perm[x] > perm[y])
        if inv % 2 == 0:
            t = np.stack([base, base + a, base + b, base + c], axis=1)
        else:
            t = np.stack([base, base + a, base + c, base + b], axis=1)
        tets.append(t)
    tets = np.stack(tets, axis=1).reshape(-1, 4)  # lattice ids

    # A jitter of +-ht/4 can invert or flatten a Kuhn tet (the volume is cubic
    # in the offsets).  Redraw, from the same stream, the offsets of the
    # interior vertices of every tet thinner than min_rel of its undeformed
    # volume until none is left, so the mesh stays a valid tiling of D.
    # min_rel = 0 redraws inverted and flat tets only and keeps the slivers the
    # jitter makes (down to ~5e-6 h^3 on the 192^3-cube L-prism at n = 256).
    flat = pos.reshape(-1, 3)
    flat_interior = interior.reshape(-1)
    v_ref = float(np.prod(ht)) / 6.0
    for _ in range(1000):
        p = flat[tets]
        vol = np.einsum("ij,ij->i", np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]),
                        p[:, 3] - p[:, 0]) / 6.0
        bad = vol <= spec.min_rel * v_ref
        if not bad.any():
            break
        verts = np.unique(tets[bad].reshape(-1))
        verts = verts[flat_interior[verts]]
        ijk = np.stack([verts % m1, (verts // m1) % m1, verts // (m1 * m1)], axis=1)
        lattice = lo + ijk * ht
        flat[verts] = lattice + rng.uniform(-spec.jitter, spec.jitter, size=(len(verts), 3)) * ht
    else:
        raise RuntimeError("could not remove degenerate tets")

    newid = -np.ones(m1 ** 3, dtype=np.int64)
    flat_used = used.reshape(-1)
    newid[flat_used] = np.arange(int(flat_used.sum()))
    xyz = flat[flat_used].copy()
    tets = newid[tets].astype(np.int32)
    return xyz, tets


def box_mesh(lo, hi, m, jitter=0.25, seed=1, min_rel=MIN_REL):
    return kuhn_mesh(MeshSpec(tuple(lo), tuple(hi), m, False, jitter, seed, min_rel))


def lprism_mesh(m, lo=(0.05, 0.05, 0.05), hi=(0.95, 0.95, 0.95), jitter=0.25, seed=1, min_rel=MIN_REL):
    return kuhn_mesh(MeshSpec(tuple(lo), tuple(hi), m, True, jitter, seed, min_rel))
