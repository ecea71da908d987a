"""The SPE10-sized box mesh (Sec. 7.2's second domain): stretched Cartesian hexes, Kuhn-split."""
import collections

import numpy as np
import pytest

from synth import SPE10_BOUNDING_BOX, SPE10_DOMAIN, cartesian_kuhn_mesh, spe10_mesh


def _vols(xyz, tets):
    p = xyz[tets]
    return np.einsum("ij,ij->i", np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), p[:, 3] - p[:, 0]) / 6.0


@pytest.mark.parametrize("counts", [(1, 1, 1), (3, 2, 4), (6, 22, 9)])
def test_tiles_the_box_conformingly(counts):
    lo, hi = (1.0, -2.0, 0.5), (4.0, 3.0, 1.5)
    xyz, tets = cartesian_kuhn_mesh(lo, hi, counts)
    nx, ny, nz = counts
    v = _vols(xyz, tets)
    hexv = np.prod(np.subtract(hi, lo)) / (nx * ny * nz)
    assert len(tets) == 6 * nx * ny * nz
    assert np.allclose(v, hexv / 6.0, rtol=1e-12)  # the six Kuhn tets of a box have equal volume
    faces = collections.Counter()
    for t in tets:
        for f in ((0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)):
            faces[tuple(sorted(t[list(f)]))] += 1
    assert max(faces.values()) == 2
    # boundary triangles: two per hex face on the box surface
    assert sum(1 for c in faces.values() if c == 1) == 4 * (nx * ny + ny * nz + nx * nz)


def test_spe10_geometry():
    xyz, tets = spe10_mesh(counts=(12, 44, 17))
    off = np.subtract(SPE10_BOUNDING_BOX, SPE10_DOMAIN) / 2.0
    assert np.array_equal(xyz.min(axis=0), off)
    assert np.array_equal(xyz.max(axis=0), off + np.asarray(SPE10_DOMAIN))
    assert abs(_vols(xyz, tets).sum() / np.prod(SPE10_DOMAIN) - 1.0) <= 1e-13
    # full-size hexes are 20 x 10 x 2 ft
    edges = np.diff(np.unique(spe10_mesh()[0][:, 2]))
    assert np.allclose(edges, 2.0)
