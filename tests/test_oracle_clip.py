"""Pins of the oracle's intersection volumes, G and the projection (Sec. 5)."""
import numpy as np
import pytest

from oracle import clip, project
from synth import box_mesh

CORNER = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.float64)


def test_tet_inside_box_is_whole_tet():
    p = 0.1 + 0.2 * CORNER
    assert clip.tet_box_volume(p, [0, 0, 0], [1, 1, 1]) == pytest.approx(0.2 ** 3 / 6, rel=1e-13)


def test_disjoint_and_touching_are_zero():
    p = 2.0 + CORNER
    assert clip.tet_box_volume(p, [0, 0, 0], [1, 1, 1]) == 0.0
    # shares only the face x = 1 with the box
    q = CORNER + np.array([1.0, 0.0, 0.0])
    assert clip.tet_box_volume(q, [0, 0, 0], [1, 1, 1]) == pytest.approx(0.0, abs=1e-15)


@pytest.mark.parametrize("a", [0.25, 0.5, 0.8])
def test_corner_tet_cut_by_plane(a):
    # corner simplex {x,y,z >= 0, x+y+z <= 1} cut at x = a: the part x >= a is a
    # scaled simplex of volume (1-a)^3/6
    keep = clip.tet_box_volume(CORNER, [-1, -1, -1], [a, 2, 2])
    assert keep == pytest.approx(1 / 6 - (1 - a) ** 3 / 6, rel=1e-12)


def test_corner_tet_in_small_cube():
    # cube [0,a]^3 with a <= 1/3 lies inside the simplex
    assert clip.tet_box_volume(CORNER, [0, 0, 0], [0.3, 0.3, 0.3]) == pytest.approx(0.027, rel=1e-12)
    # cube [0,1/2]^3: the cube minus the corner region x+y+z > 1 (volume (1/2)^3/6)
    assert clip.tet_box_volume(CORNER, [0, 0, 0], [0.5, 0.5, 0.5]) == pytest.approx(
        0.125 - 0.125 / 6, rel=1e-12)


def test_kuhn_split_of_aligned_cube():
    # an unjittered mesh whose cubes are the grid cells: G = |tau| delta
    xyz, tets = box_mesh((0.0, 0.0, 0.0), (1.0, 1.0, 1.0), 4, jitter=0.0)
    rows = clip.coupling_rows(xyz, tets, 4)
    for t, row in rows.items():
        vol = clip.tet_volume(xyz[tets[t]])
        big = {c: v for c, v in row.items() if v > 1e-14}
        assert len(big) == 1
        cube = t // 6
        assert list(big) == [cube]
        assert big[cube] == pytest.approx(vol, rel=1e-12)
        assert vol == pytest.approx((1 / 4) ** 3 / 6, rel=1e-12)


def test_row_and_column_sums_of_jittered_box():
    """Rows sum to |tau| and columns to |c cap D| (D tiled exactly)."""
    lo, hi, n = 0.15, 0.85, 8
    xyz, tets = box_mesh((lo,) * 3, (hi,) * 3, 5)
    rows = clip.coupling_rows(xyz, tets, n)
    col = np.zeros(n ** 3)
    for t, row in rows.items():
        vol = clip.tet_volume(xyz[tets[t]])
        assert sum(row.values()) == pytest.approx(vol, rel=1e-12)
        for c, v in row.items():
            col[c] += v
    h = 1.0 / n
    e = np.arange(n) * h
    ov = np.clip(np.minimum(e + h, hi) - np.maximum(e, lo), 0.0, None)
    expect = (ov[None, None, :] * ov[None, :, None] * ov[:, None, None]).ravel()
    assert np.allclose(col, expect, rtol=1e-11, atol=1e-15)


def test_translation_by_one_cell_shifts_columns():
    xyz, tets = box_mesh((0.15,) * 3, (0.55,) * 3, 3)
    n = 8
    a = clip.coupling_rows(xyz, tets, n)
    b = clip.coupling_rows(xyz + np.array([1.0 / n, 0, 0]), tets, n)
    for t in a:
        shifted = {c + 1: v for c, v in a[t].items()}
        assert set(shifted) == set(b[t])
        for c in shifted:
            assert b[t][c] == pytest.approx(shifted[c], rel=1e-11, abs=1e-16)


def test_monte_carlo_point_sampling():
    rng = np.random.default_rng(3)
    xyz, tets = box_mesh((0.15,) * 3, (0.85,) * 3, 4)
    n = 6
    h = 1.0 / n
    for t in rng.choice(len(tets), 5, replace=False):
        p = xyz[tets[t]]
        row = clip.coupling_rows(xyz, tets, n, rows=[t])[t]
        m = 200000
        lam = rng.dirichlet(np.ones(4), size=m)  # uniform in the tet
        x = lam @ p
        cells = np.floor(x / h).astype(int)
        flat = cells[:, 0] + n * (cells[:, 1] + n * cells[:, 2])
        vol = clip.tet_volume(p)
        freq = np.bincount(flat, minlength=n ** 3) / m
        for c in set(row) | set(np.nonzero(freq)[0]):
            f = row.get(c, 0.0) / vol
            assert abs(freq[c] - f) < 5 * np.sqrt(f * (1 - f) / m) + 2e-5


def test_projection_preserves_constants_and_integrals():
    xyz, tets = box_mesh((0.15,) * 3, (0.85,) * 3, 4)
    n = 8
    rows = clip.coupling_rows(xyz, tets, n)
    ones = project.project_rows(xyz, tets, rows, np.ones(n ** 3))
    assert max(abs(v - 1.0) for v in ones.values()) < 1e-12
    rng = np.random.default_rng(0)
    th = rng.standard_normal(n ** 3)
    vals = project.project_rows(xyz, tets, rows, th)
    lhs = sum(clip.tet_volume(xyz[tets[t]]) * vals[t] for t in vals)
    col = np.zeros(n ** 3)
    for row in rows.values():
        for c, v in row.items():
            col[c] += v
    assert lhs == pytest.approx(col @ th, rel=1e-12)
    assert project.lognormal(np.array([0.0, 1.0]))[1] == pytest.approx(np.e)


def test_coincident_candidate_points():
    """Tet with a face on a box plane and an edge on another: the candidate
    vertex list holds exact duplicates (once a Qhull stall).  Checked against
    point sampling."""
    p = np.array([[0.11682211, 0.81982355, 0.9401086],
                  [0.115625, 0.81875, 0.95],
                  [0.125, 0.828125, 0.95],
                  [0.115625, 0.828125, 0.95]])
    h = 1.0 / 128
    lo = h * np.array([14, 105, 121])
    v = clip.tet_box_volume(p, lo, lo + h)
    rng = np.random.default_rng(5)
    lam = rng.dirichlet(np.ones(4), size=400000)
    x = lam @ p
    inside = np.all((x >= lo) & (x <= lo + h), axis=1).mean()
    f = v / clip.tet_volume(p)
    assert abs(inside - f) < 5 * np.sqrt(f * (1 - f) / len(x)) + 1e-4
    assert 0.0 < f < 1.0


# ---------------------------------------------------------------- exact statement
from fractions import Fraction  # noqa: E402

from synth.slivers import plane_tets, sliver_tets  # noqa: E402


def test_exact_corner_simplex_cut_by_plane():
    """Corner simplex cut at x = a keeps 1/6 - (1 - a)^3 / 6 on the side x <= a,
    exactly; the cube [0, 1/2]^3 holds 1/8 - (1/2)^3 / 6 of it, exactly."""
    for a in (Fraction(1, 4), Fraction(1, 2), Fraction(4, 5), Fraction(1, 3)):
        v = clip.tet_box_volume_exact(CORNER, [-1, -1, -1], [a, 2, 2])
        assert v == Fraction(1, 6) - (1 - a) ** 3 / 6
    assert clip.tet_box_volume_exact(CORNER, [0, 0, 0], [0.5, 0.5, 0.5]) == Fraction(1, 8) - Fraction(1, 48)
    assert clip.tet_box_volume_exact(CORNER, [0, 0, 0], [0.3, 0.3, 0.3]) == Fraction(0.3) ** 3
    assert clip.tet_box_volume_exact(2.0 + CORNER, [0, 0, 0], [1, 1, 1]) == 0


def test_exact_rows_sum_to_exact_tet_volume():
    """Every cell's piece is computed on its own, so a dropped piece, a wrong
    split or a sign slip shows up as an inexact row sum."""
    xyz, tets = box_mesh((0.15,) * 3, (0.85,) * 3, 4)
    rows = clip.coupling_rows_exact(xyz, tets, 7, rows=range(0, len(tets), 5))
    for t, row in rows.items():
        assert sum(row.values()) == clip.tet_volume_exact(xyz[tets[t]])
    sx, st, _ = sliver_tets(16, per_case=1)
    for t, row in clip.coupling_rows_exact(sx, st, 16).items():
        assert sum(row.values()) == clip.tet_volume_exact(sx[st[t]])
        assert len(row) > 1  # the sliver crosses grid planes


def test_exact_matches_hull_statement_on_jittered_tets():
    xyz, tets = box_mesh((0.15,) * 3, (0.85,) * 3, 5)
    n = 8
    ex = clip.coupling_rows_exact(xyz, tets, n, rows=range(0, len(tets), 9))
    hu = clip.coupling_rows(xyz, tets, n, rows=ex.keys())
    for t in ex:
        for c in set(ex[t]) | set(hu[t]):
            assert abs(float(ex[t].get(c, 0)) - hu[t].get(c, 0.0)) <= 1e-13 / n ** 3


def test_exact_aligned_kuhn_cube_is_diagonal():
    xyz, tets = box_mesh((0.0,) * 3, (1.0,) * 3, 4, jitter=0.0)
    for t, row in clip.coupling_rows_exact(xyz, tets, 4).items():
        assert list(row) == [t // 6]
        assert row[t // 6] == Fraction(1, 6 * 64)


@pytest.mark.parametrize("n", [8, 16])
def test_hull_statement_on_slivers_and_plane_faces(n):
    """The hull statement decides membership by signed distances to the face
    planes; barycentric coordinates of a flat tet lose digits and once dropped
    real vertices of the intersection (errors up to 1e-6 h^3)."""
    h = 1.0 / n
    for xyz, tets, bound in (sliver_tets(n, per_case=2)[:2] + (1e-15,), plane_tets(n) + (5e-13,)):
        ex = clip.coupling_rows_exact(xyz, tets, n)
        hu = clip.coupling_rows(xyz, tets, n)
        for t in ex:
            for c in set(ex[t]) | set(hu[t]):
                assert abs(float(ex[t].get(c, 0)) - hu[t].get(c, 0.0)) <= bound * h ** 3, (t, c)


def test_sliver_generator_volumes_and_placement():
    n = 16
    xyz, tets, target = sliver_tets(n)
    vol = np.array([clip.tet_volume(xyz[t]) for t in tets])
    assert np.allclose(vol, target, rtol=1e-6)
    assert xyz.min() > 0.0 and xyz.max() < 1.0
    span = (xyz[tets].max(axis=1) - xyz[tets].min(axis=1)) * n
    assert np.all(span.max(axis=1) > 1.0)  # every sliver is longer than a cell along some axis
    pxyz, ptets = plane_tets(n)
    for t in ptets:  # three vertices share one coordinate
        p = pxyz[t]
        assert any(p[0, a] == p[1, a] == p[2, a] for a in range(3))


# ---------------------------------------------------------------- C statement
from oracle import clip_c  # noqa: E402


def _rows_of(rp, col, val, t):
    return dict(zip(col[rp[t]:rp[t + 1]].tolist(), val[rp[t]:rp[t + 1]].tolist()))


def test_c_statement_matches_exact_on_slivers_and_plane_faces():
    n = 16
    h3 = (1.0 / n) ** 3
    for xyz, tets in (sliver_tets(n, per_case=2)[:2],
                      plane_tets(n, offsets=(0.0, 1e-13, 2e-12, 1e-9), heights=(0.8, 1e-5))):
        rp, col, val = clip_c.coupling_csr(xyz, tets, n)
        ex = clip.coupling_rows_exact(xyz, tets, n)
        for t in ex:
            got = _rows_of(rp, col, val, t)
            for c in set(got) | set(ex[t]):
                assert abs(got.get(c, 0.0) - float(ex[t].get(c, 0))) <= 1e-15 * h3, (t, c)


def test_c_statement_matches_hull_and_sums_rows_on_a_jittered_box():
    lo, hi, n, m = 0.15, 0.85, 8, 5
    xyz, tets = box_mesh((lo,) * 3, (hi,) * 3, m)
    rp, col, val = clip_c.coupling_csr(xyz, tets, n)
    hu = clip.coupling_rows(xyz, tets, n, rows=range(0, len(tets), 3))
    for t, ref in hu.items():
        got = _rows_of(rp, col, val, t)
        for c in set(got) | set(ref):
            assert abs(got.get(c, 0.0) - ref.get(c, 0.0)) <= 1e-13 / n ** 3
    vol = project.tet_volumes(xyz, tets)
    assert np.allclose(np.add.reduceat(val, rp[:-1]), vol, rtol=1e-12, atol=0)
    colsum = np.bincount(col, weights=val, minlength=n ** 3)
    e = np.arange(n) / n
    ov = np.clip(np.minimum(e + 1.0 / n, hi) - np.maximum(e, lo), 0.0, None)
    assert np.allclose(colsum, (ov[None, None, :] * ov[None, :, None] * ov[:, None, None]).ravel(),
                       rtol=1e-11, atol=1e-17)


def test_c_statement_aligned_cubes_and_box_grid():
    xyz, tets = box_mesh((0.0,) * 3, (1.0,) * 3, 4, jitter=0.0)
    rp, col, val = clip_c.coupling_csr(xyz, tets, 4)
    assert np.array_equal(np.diff(rp), np.ones(len(tets), dtype=np.int64))
    assert np.array_equal(col, np.arange(len(tets)) // 6)
    assert np.allclose(val, 1.0 / (6 * 64), rtol=1e-14)
    # a box grid with an offset origin: the same as the hull statement
    xyz, tets = box_mesh((0.3, 0.2, 0.25), (0.9, 0.55, 0.45), 3)
    dims, h, lo = (8, 4, 2), 0.125, (0.2, 0.1, 0.2)
    rp, col, val = clip_c.coupling_csr(xyz, tets, dims, lo=lo, h=h)
    hu = clip.coupling_rows(xyz, tets, dims, lo=lo, h=h)
    for t, ref in hu.items():
        got = _rows_of(rp, col, val, t)
        for c in set(got) | set(ref):
            assert abs(got.get(c, 0.0) - ref.get(c, 0.0)) <= 1e-13 * h ** 3


def test_csr_projection_matches_row_statement():
    xyz, tets = box_mesh((0.15,) * 3, (0.85,) * 3, 4)
    n = 8
    rp, col, val = clip_c.coupling_csr(xyz, tets, n)
    pi = project.projection_matrix(rp, col, val, project.tet_volumes(xyz, tets), n ** 3)
    th = np.random.default_rng(2).standard_normal((3, n ** 3))
    got = project.project_csr(pi, th)
    rows = clip.coupling_rows(xyz, tets, n)
    ref = project.project_rows(xyz, tets, rows, th)
    for t, v in ref.items():
        assert np.allclose(got[:, t], v, rtol=1e-12, atol=1e-12)
    assert np.allclose(project.project_csr(pi, np.ones(n ** 3)), 1.0, rtol=1e-12)
