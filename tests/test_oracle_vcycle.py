"""Pins of the oracle's multigrid preconditioner statement."""
import numpy as np
import pytest

from oracle import vcycle


@pytest.mark.parametrize("n,kh2,c,omega", [(2, 0.5, 1.0, 0.8), (4, 0.05, 1.0, 0.8), (8, 0.3, 1.5, 0.7)])
def test_recursive_equals_dense(n, kh2, c, omega):
    v = vcycle.VCycle(n, kh2, c, omega)
    b = np.random.default_rng(1).standard_normal((n, n, n))
    assert np.allclose(v.apply(b).ravel(), v.dense() @ b.ravel(), rtol=1e-12, atol=1e-14)


def test_symmetric_positive_definite_and_convergent():
    v = vcycle.VCycle(8, 0.02, 1.0, 0.8)
    bm = v.dense()
    assert np.abs(bm - bm.T).max() < 1e-13 * np.abs(bm).max()
    assert np.linalg.eigvalsh(0.5 * (bm + bm.T)).min() > 0
    a = v.dense_operator(0, 8)
    rho = max(abs(np.linalg.eigvals(np.eye(512) - bm @ a)))
    assert rho < 0.6


def test_one_cell_is_exact_inverse():
    v = vcycle.VCycle(1, 0.7, 1.0, 0.8)
    assert v.apply(np.array([[[2.1]]]))[0, 0, 0] == pytest.approx(2.1 / 0.7)


def test_prolongation_reproduces_linear_functions():
    nc = 8
    xc = (np.arange(nc) + 0.5) / nc
    xf = (np.arange(2 * nc) + 0.5) / (2 * nc)
    p = vcycle.prolong_matrix_1d(nc)
    lin = p @ (3 * xc - 1)
    assert np.allclose(lin[1:-1], 3 * xf[1:-1] - 1, atol=1e-14)
    assert np.allclose(p @ np.ones(nc), 1.0)
    # 3-D: constants preserved, restriction sums to 8 x
    e = np.ones((4, 4, 4))
    assert np.allclose(vcycle.prolong(e), 1.0)
    assert np.allclose(vcycle.restrict(np.ones((8, 8, 8))), 8.0)


def test_laplacian_is_graph_laplacian():
    n = 5
    x = np.random.default_rng(2).standard_normal((n, n, n))
    lx = vcycle.laplacian(x)
    assert abs(lx.sum()) < 1e-12
    i, j, k = 2, 1, 3
    nb = [x[i + 1, j, k], x[i - 1, j, k], x[i, j + 1, k], x[i, j - 1, k], x[i, j, k + 1], x[i, j, k - 1]]
    assert lx[i, j, k] == pytest.approx(6 * x[i, j, k] - sum(nb))
    assert vcycle.neighbour_count(n)[0, 0, 0] == 3
