"""The quarter-cylinder stand-in for the paper's crooked-pipe mesh (Sec. 7.1)."""
import collections

import numpy as np
import pytest

from synth import polygon_prism_volume, quarter_cylinder_mesh, radial_nodes


def _vols(xyz, tets):
    p = xyz[tets]
    return np.einsum("ij,ij->i", np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), p[:, 3] - p[:, 0]) / 6.0


@pytest.mark.parametrize("nr,nt,nz", [(2, 3, 2), (8, 12, 14), (16, 9, 5)])
def test_tiles_the_polygon_prism(nr, nt, nz):
    xyz, tets = quarter_cylinder_mesh(nr, nt, nz)
    v = _vols(xyz, tets)
    assert v.min() > 0.0
    assert len(tets) == nz * nt * (3 + 6 * (nr - 1))
    assert abs(v.sum() / polygon_prism_volume(nt) - 1.0) <= 1e-13
    # conforming: every face of a tet is shared by at most two tets, and the faces used
    # once are exactly the triangles of the prism's surface
    faces = collections.Counter()
    for t in tets:
        for f in ((0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)):
            faces[tuple(sorted(t[list(f)]))] += 1
    assert max(faces.values()) == 2
    caps = 2 * nt * (2 * nr - 1)   # top and bottom: one wedge triangle and nr-1 quads per sector
    flats = 2 * 2 * nr * nz         # the sides at theta = 0 and pi/2
    curved = 2 * nt * nz            # the outer ring
    assert sum(1 for c in faces.values() if c == 1) == caps + flats + curved


def test_geometry_and_grading():
    xyz, tets = quarter_cylinder_mesh(16, 24, 28)
    assert xyz[:, 0].min() >= 0.5 - 1e-15 and xyz[:, 1].min() >= 0.5 - 1e-15
    assert np.hypot(xyz[:, 0] - 0.5, xyz[:, 1] - 0.5).max() <= 2.0 + 1e-12
    assert xyz[:, 2].min() == 0.5 and xyz[:, 2].max() == 7.5
    assert (xyz[:, :2] < 3.0).all()  # inside the paper's box (0,3)^2 x (0,8)
    r = radial_nodes(16)
    w = np.diff(r)
    assert r[8] == 1.0 and np.all(np.diff(w[:8]) < 0) and np.all(np.diff(w[8:]) > 0)  # finest at the layer
    assert (7.0 / 28) / w.min() > 4.0  # elements at the layer are long and thin (z step over radial width)
