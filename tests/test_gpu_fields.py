"""GPU parity for cell-wise kappa(x), sigma(x) (spde_level_set_fields /
spde_sample_fields) against the oracle's variable-coefficient system.

Tolerances as in test_gpu_parity: solved fields 1e-8 relative L2 (solver
tolerance 1e-10 times the conditioning of the scaled system), projected FP32
fields 1e-6.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1712_06758_gb300 as pkg  # noqa: E402
from oracle import clip, mixed, philox, project  # noqa: E402
from synth import box_mesh  # noqa: E402

DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1712_06758_gb300 import build
    build.build()
    pkg.lib()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def fields(n, kind="smooth"):
    """Cell-wise kappa, sigma on [0, 1]^3 (cell centres, x fastest)."""
    c = (np.arange(n) + 0.5) / n
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    if kind == "smooth":
        kap = 10.0 + 30.0 * x + 8.0 * np.sin(2 * np.pi * z)
        sig = 0.5 + 1.5 * y
    elif kind == "jump":  # a layer with 6x the inverse correlation length
        kap = np.where((z > 0.3) & (z < 0.6), 60.0, 10.0)
        sig = np.where(x < 0.5, 0.7, 1.4)
    else:
        raise ValueError(kind)
    return kap.ravel(), sig.ravel()


@pytest.mark.parametrize("prec", [pkg.SPDE_PREC_MIXED, pkg.SPDE_PREC_FP64])
@pytest.mark.parametrize("n,kind", [(8, "smooth"), (16, "smooth"), (16, "jump")])
def test_fields_solve_matches_oracle(prec, n, kind):
    ns, seed, first = 2, 5, 3
    kap, sig = fields(n, kind)
    smp = pkg.Sampler(prec)
    smp.add_level(0, n)
    smp.set_fields(0, kap, sig)
    got = smp.sample_fields(0, ns, seed, first, pkg.SPDE_OUT_GRID_GAUSSIAN | pkg.SPDE_OUT_F64).cpu().numpy()
    assert smp.stats()["max_rel_residual"] <= 1e-10
    xi = philox.normals_batch(n ** 3, seed, first, ns)
    ms = mixed.MixedSystem(n)
    for s in range(ns):
        _, ref = ms.solve_sparse(kap, sig, xi[s])
        assert rel(got[s], ref) <= 1e-8
    smp.close()


@pytest.mark.parametrize("n", [32, 64])
def test_fields_sigma_only_matches_closed_form(n):
    """Constant kappa with a cell-wise sigma: the exact field is the DCT solve of the
    cell-rescaled noise."""
    ns = 3
    _, sig = fields(n, "jump")
    smp = pkg.Sampler()
    smp.add_level(0, n)
    smp.set_fields(0, np.full(n ** 3, 20.0), sig)
    got = smp.sample_fields(0, ns, 9, 0, pkg.SPDE_OUT_GRID_GAUSSIAN | pkg.SPDE_OUT_F64).cpu().numpy()
    xi = philox.normals_batch(n ** 3, 9, 0, ns)
    assert rel(got, mixed.solve_dct(n, 20.0, 1.0, xi * sig[None, :])) <= 1e-8
    smp.close()


def test_constant_fields_reproduce_scalar_path():
    """Constant fields give the scalar path's field to the solver tolerance (the two paths use
    different preconditioner arithmetic, so their iterates differ in the last bits)."""
    n, ns = 64, 2
    smp = pkg.Sampler()
    smp.add_level(0, n)
    a = smp.sample(0, ns, 20.0, 1.3, 4, 0, pkg.SPDE_OUT_GRID_GAUSSIAN | pkg.SPDE_OUT_F64).cpu().numpy()
    smp.set_fields(0, np.full(n ** 3, 20.0), np.full(n ** 3, 1.3))
    b = smp.sample_fields(0, ns, 4, 0, pkg.SPDE_OUT_GRID_GAUSSIAN | pkg.SPDE_OUT_F64).cpu().numpy()
    assert rel(b, a) <= 1e-9
    smp.set_fields(0, None, None)  # cleared: the fields entry point refuses again
    with pytest.raises(pkg.SpdeError):
        smp.sample_fields(0, 1, 4, 0, pkg.SPDE_OUT_GRID_GAUSSIAN)
    smp.close()


def test_fields_lognormal_on_tets():
    n, ns = 16, 2
    kap, sig = fields(n, "smooth")
    xyz, tets = box_mesh((0.15,) * 3, (0.85,) * 3, 8)
    smp = pkg.Sampler()
    smp.add_level(0, n)
    smp.attach_mesh(0, xyz, tets)
    smp.set_fields(0, kap, sig)
    got = smp.sample_fields(0, ns, 2, 0, pkg.SPDE_OUT_LOGNORMAL).cpu().numpy().astype(np.float64)
    xi = philox.normals_batch(n ** 3, 2, 0, ns)
    ms = mixed.MixedSystem(n)
    th = np.stack([ms.solve_sparse(kap, sig, xi[s])[1] for s in range(ns)])
    rows = clip.coupling_rows(xyz, tets, n, rows=range(0, len(tets), 29))
    ref = project.project_rows(xyz, tets, rows, th)
    idx = np.array(sorted(ref))
    assert rel(got[:, idx], np.exp(np.stack([ref[t] for t in idx], axis=1))) <= 1e-6
    smp.close()


def test_fields_argument_errors():
    n = 8
    kap, sig = fields(n)
    smp = pkg.Sampler()
    smp.add_level(0, n)
    with pytest.raises(pkg.SpdeError):  # no fields yet
        smp.sample_fields(0, 1, 1, 0, pkg.SPDE_OUT_GRID_GAUSSIAN)
    bad = kap.copy()
    bad[17] = 0.0
    with pytest.raises(pkg.SpdeError):
        smp.set_fields(0, bad, sig)
    bad = sig.copy()
    bad[3] = np.nan
    with pytest.raises(pkg.SpdeError):
        smp.set_fields(0, kap, bad)
    with pytest.raises(pkg.SpdeError):
        pkg.spde_level_set_fields(smp.ctx, 0, kap, None)
    smp.close()
    sch = pkg.Sampler(pkg.SPDE_PREC_MIXED, solver=pkg.SPDE_SOLVER_SCHUR_CG)
    sch.add_level(0, n)
    sch.set_fields(0, kap, sig)
    with pytest.raises(pkg.SpdeError):  # fields need the MINRES solver
        sch.sample_fields(0, 1, 1, 0, pkg.SPDE_OUT_GRID_GAUSSIAN)
    sch.close()
