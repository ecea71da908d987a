"""Pins of the oracle on box grids (n_x x n_y x n_z cubic cells; Sec. 7.2 embeds its
domain in a non-cubic bounding box).

Each pin compares the box oracle with something computed another way: the DCT
closed form against the SuperLU solve of the assembled system, the closed-form
spectrum against the assembled Schur complement, a permutation of the axes against
the unpermuted solve, a field that varies along one axis only against an
independent 1-D mixed solve, and the recursive V-cycle against its dense Kronecker
statement.
"""
import numpy as np
import pytest

from oracle import mixed, vcycle
from tests.test_oracle_mixed import _mixed_line


@pytest.mark.parametrize("dims", [(6, 4, 3), (4, 8, 2), (2, 3, 5), (8, 1, 1)])
def test_dct_equals_sparse_solve(dims):
    nx, ny, nz = dims
    h, kappa, sigma = 0.37, 2.5, 1.4
    ms = mixed.MixedSystem(dims, h=h)
    assert ms.Nt == nx * ny * nz and ms.Nu == (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1)
    xi = np.random.default_rng(sum(dims)).standard_normal(ms.Nt)
    _, th = ms.solve_sparse(kappa, sigma, xi)
    ref = mixed.solve_dct(dims, kappa, sigma, xi, h=h)
    assert np.linalg.norm(th - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("dims", [(4, 3, 2), (5, 2, 2)])
def test_spectrum_equals_assembled_schur(dims):
    h, kappa = 0.5, 1.7
    ms = mixed.MixedSystem(dims, h=h)
    M = ms.M.toarray()
    B = ms.B.toarray()
    S = kappa ** 2 * ms.W.toarray() + B @ np.linalg.solve(M, B.T)
    ev = np.sort(np.linalg.eigvalsh(S))
    lam = np.sort(mixed.schur_eigenvalues(dims, h, kappa).ravel())
    assert np.allclose(ev, lam, rtol=1e-12, atol=0)


def test_axis_permutation():
    """Swapping the x and z axes of the box (and of the noise) swaps them in the field: a
    transposed index or a misplaced extent in the assembly breaks this."""
    a, b, c = 5, 3, 2
    h, kappa = 0.4, 3.0
    xi = np.random.default_rng(5).standard_normal(a * b * c).reshape(c, b, a)  # [z, y, x] of box (a, b, c)
    _, t1 = mixed.MixedSystem((a, b, c), h=h).solve_sparse(kappa, 1.0, xi.ravel())
    xi2 = np.transpose(xi, (2, 1, 0))                                           # [z, y, x] of box (c, b, a)
    _, t2 = mixed.MixedSystem((c, b, a), h=h).solve_sparse(kappa, 1.0, xi2.ravel())
    assert np.allclose(np.transpose(t1.reshape(c, b, a), (2, 1, 0)), t2.reshape(a, b, c), rtol=1e-12, atol=0)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_noise_constant_across_lines_is_a_line_solve(axis):
    """Noise constant across two axes makes every line along the third an independent 1-D
    mixed problem with the line's own length."""
    dims = (6, 4, 3)
    h, kappa, sigma = 0.3, 2.0, 1.1
    m = dims[axis]
    eta = np.random.default_rng(axis).standard_normal(m)
    shape_zyx = dims[::-1]
    line_shape = [1, 1, 1]
    line_shape[2 - axis] = m
    xi = np.broadcast_to(eta.reshape(line_shape), shape_zyx).ravel()
    _, th = mixed.MixedSystem(dims, h=h).solve_sparse(kappa, sigma, xi)
    g = mixed.g_normaliser(kappa, sigma)
    ref = _mixed_line(np.full(m, kappa), np.full(m, g), eta, h)
    full = np.broadcast_to(ref.reshape(line_shape), shape_zyx).ravel()
    assert np.allclose(th, full, rtol=1e-11, atol=1e-14 * np.abs(ref).max())


@pytest.mark.parametrize("shape", [(2, 4, 8), (1, 2, 4), (4, 2, 1)])
def test_vcycle_box_recursive_equals_dense(shape):
    v = vcycle.VCycle(shape, 0.05, 1.0, 0.8)
    d = v.dense()
    b = np.random.default_rng(1).standard_normal(shape)
    assert np.allclose(v.apply(b).ravel(), d @ b.ravel(), rtol=1e-12, atol=1e-12)
    assert np.allclose(d, d.T, rtol=1e-12, atol=1e-14)
    assert np.linalg.eigvalsh(0.5 * (d + d.T)).min() > 0.0


def test_vcycle_box_level_factors():
    """The coarse operator reproduces the Galerkin one on constants, A_{l+1} 1 = R A_l P 1,
    at every level: the children factor of s_l is right whichever axes are coarsened."""
    v = vcycle.VCycle((2, 8, 16), 0.3, 1.0, 0.8)  # [z, y, x]: z stops coarsening first
    assert v.shapes[1] == (1, 4, 8) and v.shapes[2] == (1, 2, 4)
    for lvl in range(len(v.shapes) - 1):
        fine = np.ones(v.shapes[lvl])
        coarse = np.ones(v.shapes[lvl + 1])
        galerkin = vcycle.restrict(v.op(lvl, vcycle.prolong(coarse, fine.shape)))
        assert np.allclose(v.op(lvl + 1, coarse), galerkin, rtol=1e-13, atol=0)
    cube = vcycle.VCycle(8, 0.3)
    assert cube.s == [1.0, 2.0, 4.0, 8.0] and cube.q == [1.0, 4.0, 16.0, 64.0]


def test_cube_given_as_box_is_the_cube():
    n, h, kappa = 4, 0.25, 5.0
    a = mixed.MixedSystem(n, h=h)
    b = mixed.MixedSystem((n, n, n), h=h)
    assert (a.matrix(kappa) != b.matrix(kappa)).nnz == 0


def test_coupling_rows_on_a_box_grid():
    """A Kuhn mesh whose hexes are the grid's cells: every tet lies in its own hex, so its
    row is one entry, |tau|, at that hex's flat index i + nx (j + ny k)."""
    from oracle import clip
    from synth import cartesian_kuhn_mesh
    nx, ny, nz, h = 4, 3, 2, 0.5
    xyz, tets = cartesian_kuhn_mesh((0.0, 0.0, 0.0), (nx * h, ny * h, nz * h), (nx, ny, nz))
    rows = clip.coupling_rows(xyz, tets, (nx, ny, nz), lo=0.0, h=h)
    for t, row in rows.items():
        hexid = t // 6  # six tets per hex, hexes x fastest
        assert list(row) == [hexid]
        assert abs(row[hexid] - h ** 3 / 6.0) <= 1e-15


def test_restrict_noise_on_a_box():
    """Coupled sampling's coarse normals on a box: each coarse cell sums its 8 children,
    times (h_f / h_c)^{3/2} = 2^{-3/2}; checked by an explicit loop."""
    nx, ny, nz = 4, 2, 6
    xi = np.random.default_rng(3).standard_normal(nx * ny * nz)
    got = mixed.restrict_noise(xi, (nx, ny, nz))
    ref = np.zeros((nx // 2) * (ny // 2) * (nz // 2))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                ref[(i // 2) + (nx // 2) * ((j // 2) + (ny // 2) * (k // 2))] += xi[i + nx * (j + ny * k)]
    assert np.allclose(got, ref * 2.0 ** -1.5, rtol=1e-14, atol=0)


@pytest.mark.parametrize("dims", [(4, 3, 2), (2, 5, 3)])
def test_exact_covariance_on_a_box(dims):
    """The DCT statements of the exact covariance g^2 S^{-1} W S^{-1} (its diagonal and one
    column) equal the dense covariance of the assembled box system."""
    nx, ny, nz = dims
    h, kappa, sigma = 0.3, 2.2, 1.3
    ms = mixed.MixedSystem(dims, h=h)
    B = ms.B.toarray()
    W = ms.W.toarray()
    S = kappa ** 2 * W + B @ np.linalg.solve(ms.M.toarray(), B.T)
    Si = np.linalg.inv(S)
    cov = mixed.g_normaliser(kappa, sigma) ** 2 * Si @ W @ Si
    var = mixed.variance_exact(dims, kappa, sigma, h=h)
    assert var.shape == (nz, ny, nx)
    assert np.allclose(var.ravel(), np.diag(cov), rtol=1e-11, atol=0)
    cell = 1 + nx * (2 % ny + ny * (nz - 1))
    assert np.allclose(mixed.covariance_column(dims, kappa, sigma, cell, h=h), cov[:, cell], rtol=1e-10, atol=1e-14)
