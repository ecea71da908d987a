"""Full-size configurations, checked on sampled outputs the oracle computes
one by one (the exact DCT solve per sample, the oracle's clipping per tet),
and the Matern second moments over a large batch.

Tolerances: solved fields 1e-6 relative L2 (solver tolerance 1e-8 there);
projected FP32 fields 1e-6 relative; moments within Monte Carlo error.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1712_06758_gb300 as pkg  # noqa: E402
from oracle import clip, mixed, philox, project  # noqa: E402
from synth import lprism_mesh  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1712_06758_gb300 import build
    build.build()
    pkg.lib()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _check_level(smp, lvl, n, xyz, tets, kappa, sigma, seed, ns, picks, ntet_check=40):
    """Whole batch (lognormal on tets), then sampled samples/tets against the oracle."""
    out = smp.sample(lvl, ns, kappa, sigma, seed, 0, pkg.SPDE_OUT_LOGNORMAL)
    assert smp.stats()["max_rel_residual"] <= 1e-8
    logn = out.cpu().numpy()
    del out
    assert np.all(np.isfinite(logn)) and np.all(logn > 0)
    rng = np.random.default_rng(lvl)
    tsel = rng.choice(len(tets), ntet_check, replace=False)
    rows = clip.coupling_rows(xyz, tets, n, rows=tsel)
    for s in picks:
        grid = smp.sample(lvl, 1, kappa, sigma, seed, s, pkg.SPDE_OUT_GRID_GAUSSIAN | pkg.SPDE_OUT_F64)
        ref = mixed.solve_dct(n, kappa, sigma, philox.normals(n ** 3, seed, s))
        assert rel(grid.cpu().numpy()[0], ref) <= 1e-6
        pr = project.project_rows(xyz, tets, rows, ref)
        want = np.exp(np.array([pr[t] for t in tsel]))
        assert rel(logn[s, tsel], want) <= 1e-6


@pytest.mark.parametrize("lvl,n,m,ns", [(0, 32, 24, 4096), (1, 64, 48, 1024), (2, 128, 96, 256), (3, 256, 192, 64)])
def test_mlmc_hierarchy_level(lvl, n, m, ns):
    """4-level MLMC batch: grids 32..256^3, L-prism meshes 24..192^3 cubes, kappa 20, tol 1e-8."""
    xyz, tets = lprism_mesh(m)
    smp = pkg.Sampler(pkg.SPDE_PREC_MIXED, tol=1e-8)
    smp.add_level(lvl, n)
    smp.attach_mesh(lvl, xyz, tets)
    _check_level(smp, lvl, n, xyz, tets, 20.0, 1.0, 1, ns, picks=(0, ns - 1))
    smp.close()
    torch.cuda.empty_cache()


def test_matern_moments_from_gpu_samples():
    """Empirical variance of 4096 GPU samples vs the exact discrete variance
    g^2 diag(S^-1 W S^-1), and a covariance column at lags 1..4 cells."""
    n, kappa, sigma, ns = 32, 20.0, 1.0, 4096
    smp = pkg.Sampler(pkg.SPDE_PREC_MIXED, tol=1e-8)
    smp.add_level(0, n)
    th = smp.sample(0, ns, kappa, sigma, 11, 0, pkg.SPDE_OUT_GRID_GAUSSIAN).double()
    var_emp = th.var(dim=0, unbiased=True).cpu().numpy()
    mean_emp = th.mean(dim=0).cpu().numpy()
    var = mixed.variance_exact(n, kappa, sigma).ravel()
    z = (var_emp - var) / (var * math.sqrt(2.0 / (ns - 1)))
    assert np.abs(z).max() < 5.5
    assert abs(z.mean()) < 0.1  # 32768 cells, correlated: loose bound on the average
    assert np.abs(mean_emp / np.sqrt(var)).max() < 5.5 / math.sqrt(ns) * 1.2
    c = 16 + n * (16 + n * 16)
    col = mixed.covariance_column(n, kappa, sigma, c)
    centred = th - th.mean(dim=0, keepdim=True)
    emp = (centred * centred[:, c:c + 1]).sum(dim=0).cpu().numpy() / (ns - 1)
    for lag in range(1, 5):
        cc = c + lag
        sd = math.sqrt((var[c] * var[cc] + col[cc] ** 2) / ns)
        assert abs(emp[cc] - col[cc]) < 5 * sd
    smp.close()


def test_large_single_level_512():
    """512^3 grid (134M cells), kappa 40, 2 samples, L-prism 160^3 cubes, tol 1e-8, lognormal."""
    n, m = 512, 160
    xyz, tets = lprism_mesh(m)
    smp = pkg.Sampler(pkg.SPDE_PREC_MIXED, tol=1e-8)
    smp.add_level(0, n)
    smp.attach_mesh(0, xyz, tets)
    _check_level(smp, 0, n, xyz, tets, 40.0, 1.0, 1, 2, picks=(1,), ntet_check=30)
    smp.close()
    torch.cuda.empty_cache()
