"""GPU parity on box grids (n_x x n_y x n_z cubic cells, each extent a power of two).

Sec. 7.2 embeds its domain in a 1600 x 2420 x 240 ft bounding box; a box grid
covers such a box without the cells a cube would waste.  Every step is checked
against the oracle on boxes whose multigrid hierarchy takes both kernel paths:
tiled levels (extents multiples of 32 x 16 x 8) and the one-CTA coarse levels,
including levels where an extent has reached 1 and is no longer coarsened.
Tolerances as in test_gpu_parity.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1712_06758_gb300 as pkg  # noqa: E402
from oracle import clip, mixed, philox, project, vcycle  # noqa: E402
from synth import spe10_mesh  # noqa: E402
from tests.layout import oracle_eq_to_lib, oracle_to_lib, wall_mask  # noqa: E402

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


@pytest.mark.parametrize("dims", [(8, 4, 16), (32, 16, 8), (4, 64, 4)])
@pytest.mark.parametrize("prec", [pkg.SPDE_PREC_FP64, pkg.SPDE_PREC_MIXED])
def test_apply_box_matches_assembled_operator(dims, prec):
    h, kappa, ns = 0.05, 13.0, 2
    ms = mixed.MixedSystem(dims, h=h)
    rng = np.random.default_rng(sum(dims))
    xs, refs = [], []
    for _ in range(ns):
        u = rng.standard_normal(ms.Nu)
        th = rng.standard_normal(ms.Nt)
        xs.append(oracle_to_lib(u, th, dims, h))
        yu, yt = ms.apply(kappa, u, th)
        refs.append(oracle_eq_to_lib(yu, yt, dims, h))
    dt = torch.float64 if prec == pkg.SPDE_PREC_FP64 else torch.float32
    x = torch.tensor(np.stack(xs), dtype=dt, device=DEV)
    y = torch.full_like(x, float("nan"))
    pkg.spde_apply_box(dims, h, kappa, ns, prec, x, y)
    got = y.cpu().numpy().astype(np.float64)
    assert np.all(got[:, wall_mask(dims)] == 0.0)
    assert rel(got, np.stack(refs)) <= (1e-13 if prec == pkg.SPDE_PREC_FP64 else 1e-6)


# (64, 32, 16): two tiled levels, then 16x8x4 .. 1 on the coarse kernel (z reaches 1 first);
# (32, 32, 4): coarse kernel only (4096 cells), z stops halving after two levels;
# (128, 128, 16): the SPE10 shape's path (tiled 128x128x16 and 64x64x8, coarse from 32x32x4)
@pytest.mark.parametrize("dims", [(64, 32, 16), (32, 32, 4), (128, 128, 16)])
@pytest.mark.parametrize("prec", [pkg.SPDE_PREC_FP64, pkg.SPDE_PREC_MIXED])
def test_precond_box_matches_oracle_vcycle(dims, prec):
    nx, ny, nz = dims
    h, kappa, ns = 1.0 / 64, 20.0, 2
    o = pkg.spde_opts_init()
    rng = np.random.default_rng(7)
    n3 = nx * ny * nz
    r = rng.standard_normal((ns, 4 * n3))
    r[:, wall_mask(dims)] = 0.0
    dt = torch.float64 if prec == pkg.SPDE_PREC_FP64 else torch.float32
    rt = torch.tensor(r, dtype=dt, device=DEV)
    z = torch.full_like(rt, float("nan"))
    pkg.spde_precond_box(dims, h, kappa, ns, prec, rt, z, opts=o)
    got = z.cpu().numpy().astype(np.float64)
    vc = vcycle.VCycle((nz, ny, nx), (kappa * h) ** 2, o.schur_c, o.omega)
    tol = 1e-12 if prec == pkg.SPDE_PREC_FP64 else 2e-6
    for s in range(ns):
        ref_t = vc.apply(r[s, 3 * n3:].reshape(nz, ny, nx)).ravel()
        assert rel(got[s, 3 * n3:], ref_t) <= tol
        assert np.allclose(got[s, :3 * n3], o.flux_diag * r[s, :3 * n3], rtol=1e-6, atol=0)


@pytest.mark.parametrize("dims", [(64, 32, 16), (32, 32, 4), (32, 64, 8)])
@pytest.mark.parametrize("prec", [pkg.SPDE_PREC_MIXED, pkg.SPDE_PREC_FP64])
def test_box_sample_matches_closed_form(dims, prec):
    nx, ny, nz = dims
    h, kappa, sigma, ns = 1.0 / 32, 20.0, 1.2, 2
    smp = pkg.Sampler(prec)
    smp.add_level(0, dims, (0.0, 0.0, 0.0), (nx * h, ny * h, nz * h))
    got = smp.sample(0, ns, kappa, sigma, 3, 5, pkg.SPDE_OUT_GRID_GAUSSIAN | pkg.SPDE_OUT_F64).cpu().numpy()
    st = smp.stats()
    assert st["max_rel_residual"] <= 1e-10
    xi = philox.normals_batch(nx * ny * nz, 3, 5, ns)
    ref = mixed.solve_dct(dims, kappa, sigma, xi, h=h)
    for s in range(ns):
        assert rel(got[s], ref[s]) <= 1e-8
    smp.close()


def test_box_fields_match_sparse_solve():
    dims = (32, 16, 8)
    nx, ny, nz = dims
    h = 1.0 / 32
    zc, yc, xc = np.meshgrid((np.arange(nz) + 0.5) * h, (np.arange(ny) + 0.5) * h, (np.arange(nx) + 0.5) * h,
                             indexing="ij")
    kap = (10.0 + 30.0 * xc + 8.0 * np.sin(8 * np.pi * zc)).ravel()
    sig = (0.5 + 1.5 * yc / (ny * h)).ravel()
    smp = pkg.Sampler()
    smp.add_level(0, dims, (0.0, 0.0, 0.0), (nx * h, ny * h, nz * h))
    smp.set_fields(0, kap, sig)
    got = smp.sample_fields(0, 2, 4, 0, pkg.SPDE_OUT_GRID_GAUSSIAN | pkg.SPDE_OUT_F64).cpu().numpy()
    assert smp.stats()["max_rel_residual"] <= 1e-10
    xi = philox.normals_batch(nx * ny * nz, 4, 0, 2)
    ms = mixed.MixedSystem(dims, h=h)
    for s in range(2):
        _, ref = ms.solve_sparse(kap, sig, xi[s])
        assert rel(got[s], ref) <= 1e-8
    smp.close()


def test_spe10_box_lognormal_matches_oracle():
    """The SPE10 stand-in on a box grid that covers the paper's bounding box."""
    dims, h = (64, 64, 8), 38.0  # 2432 x 2432 x 304 ft, around the 1600 x 2420 x 240 ft box
    nx, ny, nz = dims
    xyz, tets = spe10_mesh(counts=(6, 22, 9))
    smp = pkg.Sampler()
    smp.add_level(0, dims, (0.0, 0.0, 0.0), (nx * h, ny * h, nz * h))
    smp.attach_mesh(0, xyz, tets)
    got = smp.sample(0, 2, 0.02, 1.0, 8, 0, pkg.SPDE_OUT_LOGNORMAL).cpu().numpy().astype(np.float64)
    th = mixed.solve_dct(dims, 0.02, 1.0, philox.normals_batch(nx * ny * nz, 8, 0, 2), h=h)
    rows = clip.coupling_rows(xyz, tets, dims, lo=0.0, h=h, rows=range(0, len(tets), 17))
    ref = project.project_rows(xyz, tets, rows, th)
    idx = np.array(sorted(ref))
    refm = np.exp(np.stack([ref[t] for t in idx], axis=1))
    assert np.linalg.norm(got[:, idx] - refm) <= 1e-6 * np.linalg.norm(refm)
    smp.close()


def test_box_argument_errors():
    smp = pkg.Sampler()
    with pytest.raises(pkg.SpdeError):  # 128 x 128 x 4 cells on the first untiled level
        smp.add_level(0, (512, 512, 16), (0.0,) * 3, (1.0, 1.0, 1.0 / 32))
    with pytest.raises(pkg.SpdeError):  # not cubic cells
        smp.add_level(0, (64, 32, 16), (0.0,) * 3, (1.0, 1.0, 0.25))
    with pytest.raises(pkg.SpdeError):  # not a power of two
        smp.add_level(0, (48, 32, 16), (0.0,) * 3, (1.5, 1.0, 0.5))
    with pytest.raises(pkg.SpdeError):  # more than 2^29 cells
        smp.add_level(0, 1024)
    with pytest.raises(pkg.SpdeError):
        smp.add_level(0, (1024, 1024, 1024), (0.0,) * 3, (1.0, 1.0, 1.0))
    smp.add_level(0, (1024, 1024, 512), (0.0,) * 3, (1.0, 1.0, 0.5))  # 2^29 cells: accepted (nothing allocated)
    smp.close()
    sch = pkg.Sampler(pkg.SPDE_PREC_MIXED, solver=pkg.SPDE_SOLVER_SCHUR_CG)
    sch.add_level(0, (64, 32, 16), (0.0,) * 3, (2.0, 1.0, 0.5))
    with pytest.raises(pkg.SpdeError):  # the Schur-CG option needs a cube
        sch.sample(0, 1, 20.0, 1.0, 1, 0, pkg.SPDE_OUT_GRID_GAUSSIAN)
    sch.close()


def test_box_coupled_two_level_sample():
    """Sec. 6.2's coupled pair on box grids: the coarse level halves every extent."""
    fdims, cdims = (64, 32, 16), (32, 16, 8)
    h, kappa, sigma, ns, seed = 1.0 / 32, 20.0, 1.0, 2, 9
    smp = pkg.Sampler(pkg.SPDE_PREC_MIXED)
    hi = (fdims[0] * h, fdims[1] * h, fdims[2] * h)
    smp.add_level(0, fdims, (0.0, 0.0, 0.0), hi)
    smp.add_level(1, cdims, (0.0, 0.0, 0.0), hi)
    kind = pkg.SPDE_OUT_GRID_GAUSSIAN | pkg.SPDE_OUT_F64
    nf, nc = int(np.prod(fdims)), int(np.prod(cdims))
    fine = torch.zeros((ns, nf), dtype=torch.float64, device=DEV)
    coarse = torch.zeros((ns, nc), dtype=torch.float64, device=DEV)
    pkg.spde_sample_coupled(smp.ctx, 0, 1, ns, kappa, sigma, seed, 0, kind, fine, coarse)
    xi = philox.normals_batch(nf, seed, 0, ns)
    ref_f = mixed.solve_dct(fdims, kappa, sigma, xi, h=h)
    ref_c = mixed.solve_dct(cdims, kappa, sigma, np.stack([mixed.restrict_noise(x, fdims) for x in xi]), h=2 * h)
    assert rel(fine.cpu().numpy(), ref_f) <= 1e-8
    assert rel(coarse.cpu().numpy(), ref_c) <= 1e-8
    smp.close()


def test_box_serving_matches_sample():
    """Requests on a box level through the serving engine equal spde_sample bit for bit."""
    dims, h = (64, 32, 16), 1.0 / 32
    smp = pkg.Sampler(pkg.SPDE_PREC_MIXED, serve_max_batch=4)
    smp.add_level(0, dims, (0.0, 0.0, 0.0), tuple(h * v for v in dims))
    kind = pkg.SPDE_OUT_GRID_GAUSSIAN
    outs = []
    for k, ns in enumerate((3, 5, 1)):
        out = torch.full((ns, int(np.prod(dims))), float("nan"), dtype=torch.float32, device=DEV)
        rid = pkg.spde_submit(smp.ctx, 0, ns, 20.0, 1.0 + 0.25 * k, 40 + k, 3 * k, kind, out)
        outs.append((rid, ns, k, out))
    import time
    pending = {o[0] for o in outs}
    t0 = time.time()
    while pending and time.time() - t0 < 120:
        for rid in list(pending):
            done, _, st = pkg.spde_poll(smp.ctx, rid)
            if done:
                assert st == pkg.SPDE_OK
                pending.discard(rid)
        time.sleep(0.002)
    assert not pending
    for rid, ns, k, out in outs:
        alone = torch.full_like(out, float("nan"))
        pkg.spde_sample(smp.ctx, 0, ns, 20.0, 1.0 + 0.25 * k, 40 + k, 3 * k, kind, alone)
        assert torch.equal(out, alone)
    smp.close()
