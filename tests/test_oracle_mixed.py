"""Pins of the oracle's mixed RT0 x P0 system and its solves (Sec. 4)."""
import math

import numpy as np
import pytest

from oracle import mixed, philox


def _golden_g2():
    rows = []
    with open(__file__.replace("test_oracle_mixed.py", "golden/closed_forms.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                kappa, sigma, g2 = map(float, line.split())
                rows.append((kappa, sigma, g2))
    return rows


@pytest.mark.parametrize("kappa,sigma,g2", _golden_g2())
def test_g_closed_form(kappa, sigma, g2):
    assert mixed.g_normaliser(kappa, sigma) ** 2 == pytest.approx(g2, rel=1e-14)


def test_mass_matrix_closed_form():
    # 1-D RT0 mass per face line: h^3 (1/6, 2/3, 1/6), faces of other axes orthogonal
    n, h = 5, 0.3
    ms = mixed.MixedSystem(n, h)
    m = ms.M.toarray()
    # x-face (i=2, j=1, k=3): id (i-1) + (n-1)(j + n k)
    f = 1 + (n - 1) * (1 + n * 3)
    row = m[f]
    assert row[f] == pytest.approx(2 / 3 * h ** 3, rel=1e-14)
    assert row[f - 1] == pytest.approx(1 / 6 * h ** 3, rel=1e-14)
    assert row[f + 1] == pytest.approx(1 / 6 * h ** 3, rel=1e-14)
    assert np.count_nonzero(np.abs(row) > 1e-30) == 3


def test_divergence_is_face_flux():
    # b(phi_f, 1_c) = flux of phi_f out of cell c = +-h^2 (divergence theorem)
    n, h = 4, 0.25
    ms = mixed.MixedSystem(n, h)
    b = ms.B.toarray()
    assert set(np.round(np.unique(b[b != 0]) / h ** 2, 12)) == {-1.0, 1.0}
    # interior cell touches 6 interior faces, corner cell 3
    assert np.count_nonzero(b[1 + n * (1 + n * 1)]) == 6
    assert np.count_nonzero(b[0]) == 3
    # a constant field has zero discrete gradient: B^T 1 = 0
    assert np.abs(b.T @ np.ones(n ** 3)).max() < 1e-14


def test_constant_noise_closed_form():
    # xi = const => f in ker(B^T), S theta = kappa^2 h^3 theta = g h^{3/2} xi
    n, kappa, sigma = 4, 7.0, 1.3
    ms = mixed.MixedSystem(n)
    h = 1.0 / n
    xi = np.full(n ** 3, 0.7)
    u, th = ms.solve_sparse(kappa, sigma, xi)
    expect = mixed.g_normaliser(kappa, sigma) * h ** 1.5 * 0.7 / (kappa ** 2 * h ** 3)
    assert np.allclose(th, expect, rtol=1e-12)
    assert np.abs(u).max() < 1e-12 * abs(expect)


@pytest.mark.parametrize("n,kappa", [(3, 4.0), (4, 10.0)])
def test_dense_equals_sparse(n, kappa):
    ms = mixed.MixedSystem(n)
    xi = philox.normals(n ** 3, 1, 0)
    u1, t1 = ms.solve_sparse(kappa, 1.0, xi)
    u2, t2 = ms.solve_dense(kappa, 1.0, xi)
    assert np.linalg.norm(t1 - t2) <= 1e-13 * np.linalg.norm(t2)
    assert np.linalg.norm(u1 - u2) <= 1e-13 * np.linalg.norm(u2)


@pytest.mark.parametrize("n,kappa,sigma", [(4, 10.0, 1.0), (8, 20.0, 0.7), (16, 10.0, 1.0)])
def test_dct_closed_form_equals_sparse_direct(n, kappa, sigma):
    ms = mixed.MixedSystem(n)
    xi = philox.normals(n ** 3, 1, 3)
    _, t_sp = ms.solve_sparse(kappa, sigma, xi)
    t_dct = mixed.solve_dct(n, kappa, sigma, xi)
    assert np.linalg.norm(t_sp - t_dct) <= 1e-12 * np.linalg.norm(t_sp)


def test_schur_spectrum_matches_assembly():
    n, kappa = 4, 3.0
    ms = mixed.MixedSystem(n)
    h = 1.0 / n
    m = ms.M.toarray()
    b = ms.B.toarray()
    s = kappa ** 2 * h ** 3 * np.eye(n ** 3) + b @ np.linalg.solve(m, b.T)
    ev = np.sort(np.linalg.eigvalsh(s))
    lam = np.sort(mixed.schur_eigenvalues(n, h, kappa).ravel())
    assert np.allclose(ev, lam, rtol=1e-12, atol=1e-15)


def test_variance_closed_form_matches_dense_covariance():
    n, kappa, sigma = 4, 5.0, 1.1
    ms = mixed.MixedSystem(n)
    h = 1.0 / n
    m = ms.M.toarray()
    b = ms.B.toarray()
    s = kappa ** 2 * h ** 3 * np.eye(n ** 3) + b @ np.linalg.solve(m, b.T)
    sinv = np.linalg.inv(s)
    cov = mixed.g_normaliser(kappa, sigma) ** 2 * sinv @ (h ** 3 * np.eye(n ** 3)) @ sinv
    var = mixed.variance_exact(n, kappa, sigma)
    assert np.allclose(var.ravel(), np.diag(cov), rtol=1e-12)
    col = mixed.covariance_column(n, kappa, sigma, 21)
    assert np.allclose(col, cov[:, 21], rtol=1e-11, atol=1e-14)


def _centre_variance(n, kappa, sigma):
    h = 1.0 / n
    lam = mixed.schur_eigenvalues(n, h, kappa)
    k = np.arange(n)
    i = n // 2
    q = np.sqrt(2.0 / n) * np.cos(np.pi * k * (2 * i + 1) / (2 * n))
    q[0] /= math.sqrt(2.0)
    q2 = q ** 2
    return mixed.g_normaliser(kappa, sigma) ** 2 * h ** 3 * np.einsum("a,b,c,abc->", q2, q2, q2, 1 / lam ** 2)


@pytest.mark.parametrize("kappa", [10.0, 20.0])
def test_marginal_variance_tends_to_sigma2(kappa):
    """Sec. 4: g makes the marginal variance sigma^2.

    The cell-average variance converges at first order in kappa h, so the
    Richardson extrapolation of the box-centre variance from 256^3 and 512^3
    must match the continuum value (Neumann images included) closely.
    """
    sigma = 1.0
    v256 = _centre_variance(256, kappa, sigma)
    v512 = _centre_variance(512, kappa, sigma)
    extrap = 2 * v512 - v256
    target = mixed.neumann_image_variance([0.5 + 0.5 / 512] * 3, kappa, sigma)
    assert abs(extrap - target) < 5e-3
    assert v256 < v512 < target


def test_wall_variance_inflation():
    # Sec. 4.1: the no-flux boundary inflates the variance along the boundary
    var = mixed.variance_exact(32, 10.0, 1.0)
    assert var[16, 16, 0] > 1.3 * var[16, 16, 16]
    assert var[0, 0, 0] > var[16, 16, 0]


def test_sample_variance_matches_exact_covariance():
    n, kappa, sigma, ns = 8, 6.0, 1.0, 4000
    xi = philox.normals_batch(n ** 3, 5, 0, ns)
    th = mixed.solve_dct(n, kappa, sigma, xi)
    var = mixed.variance_exact(n, kappa, sigma).ravel()
    emp = th.var(axis=0)
    z = (emp - var) / (var * math.sqrt(2.0 / ns))
    assert np.abs(z).max() < 5.0
    assert abs(np.mean(z)) < 5.0 / math.sqrt(n ** 3) * 4
    col = mixed.covariance_column(n, kappa, sigma, 100)
    emp_col = (th * th[:, 100:101]).mean(axis=0)
    assert np.abs(emp_col - col).max() < 5 * math.sqrt(2.0 / ns) * var.max()


def test_restricted_noise_has_the_coarse_covariance():
    """Sec. 6.2: P^T W_f P ... the restricted right-hand side P^T W_f^{1/2} xi has
    covariance P^T W_f P = W_c exactly (each coarse cell sums 8 disjoint fine cells)."""
    n_f = 4
    r = mixed.restriction_matrix(n_f)
    wf = np.eye(n_f ** 3) * (1.0 / n_f) ** 3
    wc = np.eye((n_f // 2) ** 3) * (2.0 / n_f) ** 3
    assert np.allclose(r @ wf @ r.T, wc, rtol=1e-14, atol=0)
    xi = philox.normals(n_f ** 3, 3, 1)
    xc = mixed.restrict_noise(xi, n_f)
    # same as W_c^{-1/2} P^T W_f^{1/2} xi written with the dense matrices
    assert np.allclose(xc, np.sqrt(np.diag(wc)) ** -1 * (r @ (np.sqrt(np.diag(wf)) * xi)), rtol=1e-14)


def test_restricted_noise_is_standard_normal():
    from scipy import stats
    xi = philox.normals(64 ** 3, 9, 2)
    xc = mixed.restrict_noise(xi, 64)
    assert stats.kstest(xc, "norm").pvalue > 1e-3
    assert abs(np.corrcoef(xc[:-1], xc[1:])[0, 1]) < 5 / np.sqrt(len(xc))


# ------------------------------------------------ cell-wise kappa(x), sigma(x)
def _mixed_line(kappa_line, g_line, eta, h):
    """The mixed RT0 x P0 method on one line of n cells, written from scratch for a
    field that does not vary across the line: x-face mass h^3 tridiag(1/6, 2/3, 1/6)
    over the n-1 inner faces; the integral of the divergence of the face-f function
    is +h^2 over cell f and -h^2 over cell f+1 (matrix h^2 D); reaction block
    h^3 diag(kappa^2); right-hand side -g h^{3/2} eta.  Solved densely."""
    n = len(kappa_line)
    T = np.diag(np.full(n - 1, 2.0 / 3.0)) + np.diag(np.full(n - 2, 1.0 / 6.0), 1) + np.diag(np.full(n - 2, 1.0 / 6.0), -1)
    D = np.zeros((n, n - 1))
    for f in range(n - 1):
        D[f, f] = 1.0       # face f is the right face of cell f (outward normal +x)
        D[f + 1, f] = -1.0  # and the left face of cell f + 1
    A = np.block([[h ** 3 * T, h ** 2 * D.T], [h ** 2 * D, -h ** 3 * np.diag(np.asarray(kappa_line) ** 2)]])
    b = np.concatenate([np.zeros(n - 1), -np.asarray(g_line) * h ** 1.5 * eta])
    return np.linalg.solve(A, b)[n - 1:]


def test_fields_constant_arrays_equal_scalar():
    n = 4
    ms = mixed.MixedSystem(n)
    xi = np.random.default_rng(11).standard_normal(n ** 3)
    _, t1 = ms.solve_sparse(20.0, 1.3, xi)
    _, t2 = ms.solve_sparse(np.full(n ** 3, 20.0), np.full(n ** 3, 1.3), xi)
    assert np.array_equal(t1, t2)


@pytest.mark.parametrize("n", [4, 8])
def test_fields_sigma_only_is_rescaled_noise(n):
    """With kappa constant, a cell-wise sigma only rescales the noise cell by cell, so the
    DCT closed form of the constant-kappa Schur complement gives the exact field."""
    rng = np.random.default_rng(n)
    sig = rng.uniform(0.5, 2.0, n ** 3)
    xi = rng.standard_normal(n ** 3)
    _, th = mixed.MixedSystem(n).solve_sparse(20.0, sig, xi)
    ref = mixed.solve_dct(n, 20.0, 1.0, sig * xi)
    assert np.linalg.norm(th - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("axis", [0, 2])
def test_fields_layered_kappa_reduces_to_one_line(axis):
    """kappa and the noise vary along one axis only: the 3-D field is constant across
    the other two axes and equals the 1-D mixed solution on every line."""
    n, h = 8, 1.0 / 8
    rng = np.random.default_rng(3 + axis)
    k_line = rng.uniform(5.0, 40.0, n)
    s_line = rng.uniform(0.5, 2.0, n)
    eta = rng.standard_normal(n)
    idx = np.indices((n, n, n))  # [0] = k (z), [1] = j (y), [2] = i (x) in the C-order flat index i + n (j + n k)
    pos = idx[2] if axis == 0 else idx[0]
    kap, sig, xi = k_line[pos].ravel(), s_line[pos].ravel(), eta[pos].ravel()
    _, th = mixed.MixedSystem(n).solve_sparse(kap, sig, xi)
    th = th.reshape(n, n, n)
    line = th[0, 0, :] if axis == 0 else th[:, 0, 0]
    g_line = np.array([mixed.g_normaliser(k, s) for k, s in zip(k_line, s_line)])
    ref = _mixed_line(k_line, g_line, eta, h)
    assert np.allclose(line, ref, rtol=1e-11, atol=1e-14 * np.abs(ref).max())
    # constant across the other two axes
    full = np.broadcast_to(line[None, None, :] if axis == 0 else line[:, None, None], (n, n, n))
    assert np.allclose(th, full, rtol=1e-11, atol=1e-14 * np.abs(ref).max())
