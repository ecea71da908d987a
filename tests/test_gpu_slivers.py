"""Clipping parity on near-degenerate tets (Sec. 5.1-5.2: G[tau][c] = |tau cap c|).

Slivers of 1e-3, 1e-5 and 1e-8 h^3 (flat, needle and cap shapes) crossing one
to three grid planes per axis, tets with a face on or within 1e-13 h of a
grid plane, and the headline L-prism mesh with every valid tet kept (slivers
down to ~1e-4 h^3): the device's coupling rows against the oracle's exact
rational intersection volumes, entry by entry to 1e-12 h^3, and the row sums
against the exact tet volumes.
"""
import numpy as np
import pytest

pytest.importorskip("torch")
import torch  # noqa: E402

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1712_06758_gb300 as pkg  # noqa: E402
from oracle import clip  # noqa: E402
from synth import lprism_mesh  # noqa: E402
from synth.slivers import plane_tets, sliver_tets  # noqa: E402

pytestmark = pytest.mark.gpu

# Row sums: the device adds up each piece's fan sums in cell-local coordinates,
# terms of size h^3 that cancel down to the piece's volume, so its rounding is
# absolute at the scale of the cell: |sum - |tau|| <= 1e-12 |tau| + 128 eps h^3.
# A vertex within 1e-12 h of a grid plane is moved onto it before clipping, which
# changes the volume by up to that distance times a face area: tets built on
# such planes get 1e-12 h^3, the bound of the entries.
ROW_ABS = 128 * 2.0 ** -52


def _check_rows(xyz, tets, n, rows, row_abs=ROW_ABS):
    smp = pkg.Sampler()
    smp.add_level(0, n)
    smp.attach_mesh(0, xyz, tets)  # the library itself checks every row sum
    rowptr, col, g, vol = pkg.spde_mesh_copy_csr(smp.ctx, 0)
    smp.close()
    h3 = (1.0 / n) ** 3
    worst_e, worst_s = 0.0, 0.0
    for t, ref in rows.items():
        got = dict(zip(col[rowptr[t]:rowptr[t + 1]].tolist(), g[rowptr[t]:rowptr[t + 1]].tolist()))
        for c in set(ref) | set(got):
            err = abs(got.get(c, 0.0) - float(ref.get(c, 0)))
            worst_e = max(worst_e, err / h3)
            assert err <= 1e-12 * h3, (t, c, got.get(c, 0.0), float(ref.get(c, 0)))
        exact = float(clip.tet_volume_exact(xyz[tets[t]]))
        assert abs(vol[t] - exact) <= 1e-13 * exact + ROW_ABS * h3
        s = float(np.sum(g[rowptr[t]:rowptr[t + 1]]))
        worst_s = max(worst_s, abs(s - exact) / h3)
        assert abs(s - exact) <= 1e-12 * exact + row_abs * h3, (t, s, exact)
    return worst_e, worst_s


@pytest.mark.parametrize("n", [16, 32])
def test_sliver_rows_match_exact_oracle(n):
    xyz, tets, target = sliver_tets(n, per_case=4, seed=11 + n)
    rows = clip.coupling_rows_exact(xyz, tets, n)
    assert min(len(r) for r in rows.values()) >= 2  # every sliver crosses a grid plane
    we, ws = _check_rows(xyz, tets, n, rows)
    print("slivers n=%d: max entry error %.2e h^3, max row-sum error %.2e h^3" % (n, we, ws))


@pytest.mark.parametrize("offsets,row_abs", [((0.0, 1e-13, -1e-13, 3e-14), 1e-12),
                                             ((2e-12, -5e-12, 1e-11, -3e-11, 1e-9), ROW_ABS)])
def test_plane_face_rows_match_exact_oracle(offsets, row_abs):
    """Faces on a grid plane or within 1e-13 h of it (moved onto it before
    clipping), and faces just beyond that (clipped as they are); caps as thin as
    1e-5 h, whose side faces are nearly parallel to the plane."""
    n = 16
    xyz, tets = plane_tets(n, offsets=offsets, heights=(0.8, 1e-3, 1e-5))
    rows = clip.coupling_rows_exact(xyz, tets, n)
    we, ws = _check_rows(xyz, tets, n, rows, row_abs=row_abs)
    print("plane faces %s: max entry error %.2e h^3, max row-sum error %.2e h^3" % (offsets, we, ws))


def test_headline_lprism_with_slivers_kept():
    """The 96^3-cube L-prism on the 128^3 grid with only inverted tets redrawn:
    its 40 thinnest tets and 300 others, row by row against the exact oracle."""
    n = 128
    xyz, tets = lprism_mesh(96, min_rel=0.0)
    p = xyz[tets]
    vol = np.einsum("ij,ij->i", np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), p[:, 3] - p[:, 0]) / 6.0
    thin = np.argsort(vol)[:40]
    assert vol[thin[0]] * n ** 3 < 1e-3  # the mesh holds slivers
    rng = np.random.default_rng(4)
    pick = np.unique(np.concatenate([thin, rng.choice(len(tets), 300, replace=False)]))
    rows = clip.coupling_rows_exact(xyz, tets, n, rows=pick)
    we, ws = _check_rows(xyz, tets, n, rows)
    print("L-prism 96^3 (min %.2e h^3): max entry error %.2e h^3, max row-sum error %.2e h^3"
          % (vol[thin[0]] * n ** 3, we, ws))
