"""GPU parity: every step of the path, through the C ABI, against the oracle.

Tolerances: integers bit-exact; FP64 normals within 16 ulp per element and
1e-15 relative L2; FP64 operator applications to rounding (1e-13 relative);
FP32 steps to 1e-6 relative; solved fields to 1e-8 relative L2 (the solver
tolerance 1e-10 times the conditioning of the scaled system); projected
fields in FP32 to 1e-6 relative L2, which is the field tolerance the
sampler targets.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1712_06758_gb300 as pkg  # noqa: E402
from oracle import clip, mixed, philox, project, vcycle  # noqa: E402
from synth import box_mesh, lprism_mesh  # noqa: E402
from tests.layout import lib_to_oracle, oracle_to_lib, oracle_eq_to_lib, wall_mask  # noqa: E402

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


# ---------------------------------------------------------------- noise (K1)
@pytest.mark.parametrize("seed,sample", [(1, 0), (0xDEADBEEF12345678, 2 ** 32 - 1), (7, 2 ** 40 + 3)])
def test_philox_words_bit_exact(seed, sample):
    npairs = 5000
    out = torch.zeros(npairs * 4, dtype=torch.int32, device=DEV)
    pkg.spde_noise_words(npairs, seed, sample, out)
    got = out.cpu().numpy().view(np.uint32).reshape(npairs, 4)
    ref = philox.noise_words(2 * npairs, seed, sample).astype(np.uint32)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("ncells,ns,first", [(4097, 3, 0), (2 * 16 ** 3, 2, 2 ** 32 - 1), (1, 1, 5)])
def test_normals_match(ncells, ns, first):
    out = torch.zeros((ns, ncells), dtype=torch.float64, device=DEV)
    pkg.spde_noise(ncells, ns, 1, first, 1.0, out)
    got = out.cpu().numpy()
    ref = philox.normals_batch(ncells, 1, first, ns)
    tol = 16 * 2.0 ** -52 * np.maximum(1.0, np.abs(ref))
    assert np.all(np.abs(got - ref) <= tol)
    assert rel(got, ref) <= 1e-15
    scaled = torch.zeros_like(out)
    pkg.spde_noise(ncells, ns, 1, first, -2.5, scaled)
    assert np.allclose(scaled.cpu().numpy(), -2.5 * got, rtol=1e-15, atol=0)


# --------------------------------------------------------------- operator (K2)
@pytest.mark.parametrize("n", [4, 8, 16, 32, 64])
@pytest.mark.parametrize("prec", [pkg.SPDE_PREC_FP64, pkg.SPDE_PREC_MIXED])
def test_apply_matches_assembled_operator(n, prec):
    h, kappa, ns = 1.0 / n, 13.0, 2
    ms = mixed.MixedSystem(n)
    rng = np.random.default_rng(n)
    xs, refs = [], []
    for _ in range(ns):
        u = rng.standard_normal(ms.Nu)
        th = rng.standard_normal(ms.Nt)
        xs.append(oracle_to_lib(u, th, n, h))
        yu, yt = ms.apply(kappa, u, th)
        refs.append(oracle_eq_to_lib(yu, yt, n, h))
    dt = torch.float64 if prec == pkg.SPDE_PREC_FP64 else torch.float32
    x = torch.tensor(np.stack(xs), dtype=dt, device=DEV)
    y = torch.full_like(x, float("nan"))
    pkg.spde_apply(n, h, kappa, ns, prec, x, y)
    got = y.cpu().numpy().astype(np.float64)
    ref = np.stack(refs)
    assert np.all(got[:, wall_mask(n)] == 0.0)
    assert rel(got, ref) <= (1e-13 if prec == pkg.SPDE_PREC_FP64 else 1e-6)


# ---------------------------------------------------------- preconditioner (K3)
@pytest.mark.parametrize("n", [4, 8, 16, 32, 64, 128])
@pytest.mark.parametrize("prec", [pkg.SPDE_PREC_FP64, pkg.SPDE_PREC_MIXED])
def test_precond_matches_oracle_vcycle(n, prec):
    h, kappa, ns = 1.0 / n, 20.0, 2
    o = pkg.spde_opts_init()
    rng = np.random.default_rng(3)
    r = rng.standard_normal((ns, 4 * n ** 3))
    r[:, wall_mask(n)] = 0.0
    dt = torch.float64 if prec == pkg.SPDE_PREC_FP64 else torch.float32
    rt = torch.tensor(r, dtype=dt, device=DEV)
    z = torch.full_like(rt, float("nan"))
    pkg.spde_precond(n, h, kappa, ns, prec, rt, z, opts=o)
    got = z.cpu().numpy().astype(np.float64)
    vc = vcycle.VCycle(n, (kappa * h) ** 2, o.schur_c, o.omega)
    n3 = n ** 3
    for s in range(ns):
        ref_t = vc.apply(r[s, 3 * n3:].reshape(n, n, n)).ravel()
        tol = 1e-12 if prec == pkg.SPDE_PREC_FP64 else 2e-6
        assert rel(got[s, 3 * n3:], ref_t) <= tol
        assert np.allclose(got[s, :3 * n3], o.flux_diag * r[s, :3 * n3], rtol=1e-6, atol=0)


# ------------------------------------------------------ solve (K4 + K5, a4/a5)
def _rhs(n, kappa, sigma, seed, first, ns):
    h = 1.0 / n
    xi = philox.normals_batch(n ** 3, seed, first, ns)
    return xi, -mixed.g_normaliser(kappa, sigma) * h * xi


@pytest.mark.parametrize("prec", [pkg.SPDE_PREC_MIXED, pkg.SPDE_PREC_FP64])
@pytest.mark.parametrize("n,ns", [(4, 2), (16, 3), (64, 2)])
def test_solve_matches_closed_form(prec, n, ns):
    kappa, sigma = 20.0, 1.0
    h = 1.0 / n
    smp = pkg.Sampler(prec)
    smp.add_level(0, n)
    xi, rhs = _rhs(n, kappa, sigma, 1, 0, ns)
    x = torch.zeros((ns, 4 * n ** 3), dtype=torch.float64, device=DEV)
    pkg.spde_solve(smp.ctx, 0, ns, kappa, torch.tensor(rhs, device=DEV), x)
    st = smp.stats()
    assert st["max_rel_residual"] <= 1e-10
    got = x.cpu().numpy()
    ref = mixed.solve_dct(n, kappa, sigma, xi)
    for s in range(ns):
        _, th = lib_to_oracle(got[s], n, h)
        assert rel(th, ref[s]) <= 1e-8
    assert np.all(got[:, wall_mask(n)] == 0.0)
    smp.close()


def test_solve_flux_matches_sparse_direct():
    n, kappa, sigma = 8, 10.0, 1.3
    h = 1.0 / n
    smp = pkg.Sampler(pkg.SPDE_PREC_MIXED)
    smp.add_level(0, n)
    xi, rhs = _rhs(n, kappa, sigma, 4, 9, 1)
    x = torch.zeros((1, 4 * n ** 3), dtype=torch.float64, device=DEV)
    pkg.spde_solve(smp.ctx, 0, 1, kappa, torch.tensor(rhs, device=DEV), x)
    u, th = lib_to_oracle(x.cpu().numpy()[0], n, h)
    u_ref, th_ref = mixed.MixedSystem(n).solve_sparse(kappa, sigma, xi[0])
    assert rel(th, th_ref) <= 1e-8
    assert rel(u, u_ref) <= 1e-8
    smp.close()


# ------------------------------------------------------------- clipping (K6)
def _gpu_rows(smp, level):
    rowptr, col, g, vol = pkg.spde_mesh_copy_csr(smp.ctx, level)
    return rowptr, col, g, vol


@pytest.mark.parametrize("case", ["box12_n16", "lprism24_n32", "aligned"])
def test_clip_matches_oracle(case):
    if case == "box12_n16":
        n, (xyz, tets) = 16, box_mesh((0.15,) * 3, (0.85,) * 3, 12)
    elif case == "lprism24_n32":
        n, (xyz, tets) = 32, lprism_mesh(24)
    else:
        n, (xyz, tets) = 8, box_mesh((0.0,) * 3, (1.0,) * 3, 8, jitter=0.0)
    h = 1.0 / n
    smp = pkg.Sampler()
    smp.add_level(0, n)
    smp.attach_mesh(0, xyz, tets)
    rowptr, col, g, vol = _gpu_rows(smp, 0)
    vref = np.array([clip.tet_volume(xyz[t]) for t in tets])
    assert np.allclose(vol, vref, rtol=1e-13)
    # every row sums to its tet volume
    rs = np.add.reduceat(g, rowptr[:-1]) if len(g) else np.zeros(len(vol))
    assert np.allclose(rs, vol, rtol=1e-11, atol=0)
    # sampled rows entry by entry
    step = 1 if case == "aligned" else 23
    rows = clip.coupling_rows(xyz, tets, n, rows=range(0, len(tets), step))
    for t, ref in rows.items():
        got = dict(zip(col[rowptr[t]:rowptr[t + 1]].tolist(), g[rowptr[t]:rowptr[t + 1]].tolist()))
        for c in set(ref) | set(got):
            assert abs(got.get(c, 0.0) - ref.get(c, 0.0)) <= 1e-12 * h ** 3, (t, c)
    if case == "aligned":
        assert len(g) == len(tets)
    smp.close()


# Tets of the jittered 192^3-cube L-prism (seed 1) around tet 15898757, whose
# vertices lie within rounding of the 256^3 grid planes z = 0.5 and x = 0.05
# (on the outer face): a configuration where inconsistent tolerances in the
# clipping once left a sliver of the intersection surface open.
NEAR_PLANE_XYZ = [[0.4964294809383716, 0.7293650418560711, 0.49456028756468584], [0.05, 0.734375, 0.4953125],
                  [0.05355736155541837, 0.734459848836528, 0.4948498762023506],
                  [0.05852057207050046, 0.7353840591258433, 0.4954273461282783], [0.05, 0.7390625000000001, 0.4953125],
                  [0.05509514229698885, 0.7382908577087337, 0.495951502032792],
                  [0.05909978334196638, 0.7388096298173595, 0.49416448731158635],
                  [0.4950461197617592, 0.7305617978133694, 0.5007409101409984], [0.05, 0.734375, 0.49999999999999994],
                  [0.055500692284403796, 0.7355042826276564, 0.5008434084846913],
                  [0.05916945957529681, 0.7348260817433576, 0.5003229827332125],
                  [0.4943341457401298, 0.7350223236231647, 0.5009075124864458],
                  [0.49999999999999994, 0.734375, 0.49999999999999994],
                  [0.05, 0.7390625000000001, 0.49999999999999994],
                  [0.054071817109563554, 0.7392692841949706, 0.500000417513931],
                  [0.05925084593838861, 0.7401303576354158, 0.4994870852676509]]
NEAR_PLANE_TETS = [[1, 2, 5, 14], [1, 2, 14, 9], [1, 4, 14, 5], [1, 4, 13, 14], [1, 8, 9, 14], [1, 8, 14, 13],
                   [2, 3, 6, 15], [2, 3, 15, 10], [2, 5, 15, 6], [2, 5, 14, 15], [2, 9, 10, 15]]


def test_clip_vertices_near_grid_planes():
    n = 256
    xyz = np.array(NEAR_PLANE_XYZ)
    tets = np.array(NEAR_PLANE_TETS, dtype=np.int32)
    smp = pkg.Sampler()
    smp.add_level(0, n)
    smp.attach_mesh(0, xyz, tets)  # the library checks every row sum to 1e-10
    rowptr, col, g, vol = _gpu_rows(smp, 0)
    rs = np.add.reduceat(g, rowptr[:-1])
    assert np.allclose(rs, vol, rtol=1e-13, atol=0)
    rows = clip.coupling_rows(xyz, tets, n)
    for t, ref in rows.items():
        got = dict(zip(col[rowptr[t]:rowptr[t + 1]].tolist(), g[rowptr[t]:rowptr[t + 1]].tolist()))
        for c in set(ref) | set(got):
            assert abs(got.get(c, 0.0) - ref.get(c, 0.0)) <= 1e-12 / n ** 3, (t, c)
    smp.close()


def test_clip_column_sums_match_domain_overlap():
    """Sum over tets of G[tau][c] = |c cap D| for the box domain D (closed form)."""
    lo, hi, n = 0.15, 0.85, 16
    xyz, tets = box_mesh((lo,) * 3, (hi,) * 3, 12)
    smp = pkg.Sampler()
    smp.add_level(0, n)
    smp.attach_mesh(0, xyz, tets)
    rowptr, col, g, vol = _gpu_rows(smp, 0)
    colsum = np.bincount(col, weights=g, minlength=n ** 3)
    h = 1.0 / n
    e = np.arange(n) * h
    ov = np.clip(np.minimum(e + h, hi) - np.maximum(e, lo), 0.0, None)
    expect = (ov[None, None, :] * ov[None, :, None] * ov[:, None, None]).ravel()
    assert np.allclose(colsum, expect, rtol=1e-11, atol=1e-17)
    smp.close()


def test_mesh_orientation_and_rejections():
    n = 16
    xyz, tets = box_mesh((0.15,) * 3, (0.85,) * 3, 4)
    smp = pkg.Sampler()
    smp.add_level(0, n)
    smp.attach_mesh(0, xyz, tets)
    a = _gpu_rows(smp, 0)
    flipped = tets.copy()
    flipped[::3, [2, 3]] = flipped[::3, [3, 2]]
    smp.attach_mesh(0, xyz, flipped)
    b = _gpu_rows(smp, 0)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])  # same sparsity
    h = 1.0 / n
    assert np.allclose(a[2], b[2], rtol=0, atol=1e-15 * h ** 3)  # same volumes up to rounding
    assert np.allclose(a[3], b[3], rtol=1e-15, atol=0)
    bad = xyz.copy()
    bad[tets[5, 0]] = [1.2, 0.5, 0.5]  # drags tet 5 (and others) outside the box
    with pytest.raises(pkg.SpdeError) as ei:
        smp.attach_mesh(0, bad, tets)
    assert ei.value.status == pkg.SPDE_EMESH
    flat = tets.copy()
    flat[7] = [tets[7, 0], tets[7, 0], tets[7, 1], tets[7, 2]]
    with pytest.raises(pkg.SpdeError) as ei:
        smp.attach_mesh(0, xyz, flat)
    assert ei.value.status == pkg.SPDE_EMESH and "tet 7" in str(ei.value)
    smp.close()


# ----------------------------------------------------------- projection (K7)
@pytest.mark.parametrize("ns", [1, 3, 8, 9, 10, 40, 64])
@pytest.mark.parametrize("kind", [pkg.SPDE_OUT_GAUSSIAN, pkg.SPDE_OUT_LOGNORMAL,
                                  pkg.SPDE_OUT_LOGNORMAL | pkg.SPDE_OUT_F64])
def test_project_matches_oracle(ns, kind):
    n = 16
    xyz, tets = box_mesh((0.15,) * 3, (0.85,) * 3, 12)
    smp = pkg.Sampler()
    smp.add_level(0, n)
    smp.attach_mesh(0, xyz, tets)
    th = np.random.default_rng(ns).standard_normal((ns, n ** 3)) * 0.7
    dt = torch.float64 if kind & pkg.SPDE_OUT_F64 else torch.float32
    out = torch.full((ns, len(tets)), float("nan"), dtype=dt, device=DEV)
    pkg.spde_project(smp.ctx, 0, ns, torch.tensor(th, device=DEV), kind, out)
    got = out.cpu().numpy().astype(np.float64)
    rows = clip.coupling_rows(xyz, tets, n, rows=range(0, len(tets), 41))
    ref = project.project_rows(xyz, tets, rows, th)
    idx = np.array(sorted(ref))
    refm = np.stack([ref[t] for t in idx], axis=1)
    if (kind & 15) == pkg.SPDE_OUT_LOGNORMAL:
        refm = np.exp(refm)
    assert rel(got[:, idx], refm) <= 1e-6
    smp.close()


# ------------------------------------------------------------- end to end
@pytest.mark.parametrize("prec", [pkg.SPDE_PREC_MIXED, pkg.SPDE_PREC_FP64])
def test_sample_config1_matches_oracle(prec):
    """16^3 grid, kappa 10, box mesh 12^3 x 6 tets, seed 1, samples 0..3."""
    n, kappa, sigma, seed, ns = 16, 10.0, 1.0, 1, 4
    xyz, tets = box_mesh((0.15,) * 3, (0.85,) * 3, 12)
    smp = pkg.Sampler(prec)
    smp.add_level(0, n)
    smp.attach_mesh(0, xyz, tets)
    grid = smp.sample(0, ns, kappa, sigma, seed, 0, pkg.SPDE_OUT_GRID_GAUSSIAN | pkg.SPDE_OUT_F64)
    gauss = smp.sample(0, ns, kappa, sigma, seed, 0, pkg.SPDE_OUT_GAUSSIAN)
    logn = smp.sample(0, ns, kappa, sigma, seed, 0, pkg.SPDE_OUT_LOGNORMAL)
    xi = philox.normals_batch(n ** 3, seed, 0, ns)
    ref = mixed.solve_dct(n, kappa, sigma, xi)
    assert rel(grid.cpu().numpy(), ref) <= 1e-8
    rows = clip.coupling_rows(xyz, tets, n, rows=range(0, len(tets), 37))
    pr = project.project_rows(xyz, tets, rows, ref)
    idx = np.array(sorted(pr))
    refm = np.stack([pr[t] for t in idx], axis=1)
    assert rel(gauss.cpu().numpy()[:, idx], refm) <= 1e-6
    assert rel(logn.cpu().numpy()[:, idx], np.exp(refm)) <= 1e-6
    smp.close()


def test_plain_and_mixed_paths_agree():
    n, kappa, ns = 32, 20.0, 3
    fields = []
    for prec in (pkg.SPDE_PREC_FP64, pkg.SPDE_PREC_MIXED):
        smp = pkg.Sampler(prec)
        smp.add_level(0, n)
        fields.append(smp.sample(0, ns, kappa, 1.0, 9, 100, pkg.SPDE_OUT_GRID_GAUSSIAN | pkg.SPDE_OUT_F64).cpu().numpy())
        smp.close()
    assert rel(fields[1], fields[0]) <= 1e-8


def test_sample_alone_equals_sample_in_batch():
    """A column's result does not depend on the batch it runs in (bitwise)."""
    n, kappa = 32, 20.0
    smp = pkg.Sampler(pkg.SPDE_PREC_MIXED)
    smp.add_level(0, n)
    batch = smp.sample(0, 8, kappa, 1.0, 3, 10, pkg.SPDE_OUT_GRID_GAUSSIAN | pkg.SPDE_OUT_F64).cpu().numpy()
    for i in (0, 5):
        alone = smp.sample(0, 1, kappa, 1.0, 3, 10 + i, pkg.SPDE_OUT_GRID_GAUSSIAN | pkg.SPDE_OUT_F64).cpu().numpy()
        assert np.array_equal(alone[0], batch[i])
    smp.close()


def test_host_output_equals_device_output():
    n = 16
    xyz, tets = box_mesh((0.15,) * 3, (0.85,) * 3, 6)
    smp = pkg.Sampler()
    smp.add_level(0, n)
    smp.attach_mesh(0, xyz, tets)
    dev = smp.sample(0, 3, 10.0, 1.0, 1, 0).cpu().numpy()
    host = np.zeros((3, len(tets)), dtype=np.float32)
    pkg.spde_sample(smp.ctx, 0, 3, 10.0, 1.0, 1, 0, pkg.SPDE_OUT_LOGNORMAL, host)
    assert np.array_equal(host, dev)
    smp.close()


def test_argument_errors_and_empty_batch():
    smp = pkg.Sampler()
    smp.add_level(0, 8)
    out = torch.zeros((1, 8 ** 3), device=DEV)
    for bad in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(pkg.SpdeError) as ei:
            pkg.spde_sample(smp.ctx, 0, 1, bad, 1.0, 1, 0, pkg.SPDE_OUT_GRID_GAUSSIAN, out)
        assert ei.value.status == pkg.SPDE_EINVAL
    with pytest.raises(pkg.SpdeError):
        pkg.spde_sample(smp.ctx, 3, 1, 1.0, 1.0, 1, 0, pkg.SPDE_OUT_GRID_GAUSSIAN, out)
    with pytest.raises(pkg.SpdeError):  # no mesh on this level
        pkg.spde_sample(smp.ctx, 0, 1, 1.0, 1.0, 1, 0, pkg.SPDE_OUT_LOGNORMAL, out)
    pkg.spde_sample(smp.ctx, 0, 0, 1.0, 1.0, 1, 0, pkg.SPDE_OUT_GRID_GAUSSIAN, out)  # no-op
    for bad_n in (12, 2, 2048):
        with pytest.raises(pkg.SpdeError):
            smp.add_level(1, bad_n)
    smp.close()


def test_iteration_cap_reports_enoconv():
    smp = pkg.Sampler(pkg.SPDE_PREC_MIXED, max_iter=2, max_outer=1)
    smp.add_level(0, 16)
    with pytest.raises(pkg.SpdeError) as ei:
        smp.sample(0, 1, 10.0, 1.0, 1, 0, pkg.SPDE_OUT_GRID_GAUSSIAN)
    assert ei.value.status == pkg.SPDE_ENOCONV
    assert smp.stats()["max_rel_residual"] > 1e-10
    smp.close()


@pytest.mark.parametrize("nf", [32, 64])
def test_coupled_two_level_sample(nf):
    """Sec. 6.2 coupled pair: fine field from the fine noise, coarse field from the
    restricted noise, fine solve warm-started from the coarse field."""
    nc, kappa, sigma, ns, seed = nf // 2, 20.0, 1.0, 3, 5
    smp = pkg.Sampler(pkg.SPDE_PREC_MIXED)
    smp.add_level(0, nf)
    smp.add_level(1, nc)
    kind = pkg.SPDE_OUT_GRID_GAUSSIAN | pkg.SPDE_OUT_F64
    fine = torch.zeros((ns, nf ** 3), dtype=torch.float64, device=DEV)
    coarse = torch.zeros((ns, nc ** 3), dtype=torch.float64, device=DEV)
    pkg.spde_sample_coupled(smp.ctx, 0, 1, ns, kappa, sigma, seed, 4, kind, fine, coarse)
    warm_iters = smp.stats()["inner_iters"]
    xi = philox.normals_batch(nf ** 3, seed, 4, ns)
    ref_f = mixed.solve_dct(nf, kappa, sigma, xi)
    ref_c = mixed.solve_dct(nc, kappa, sigma, np.stack([mixed.restrict_noise(x, nf) for x in xi]))
    assert rel(fine.cpu().numpy(), ref_f) <= 1e-8
    assert rel(coarse.cpu().numpy(), ref_c) <= 1e-8
    alone = smp.sample(0, ns, kappa, sigma, seed, 4, kind)
    assert rel(fine.cpu().numpy(), alone.cpu().numpy()) <= 1e-8
    assert warm_iters <= smp.stats()["inner_iters"]  # the coarse field is a useful start
    smp.close()


# ------------------------------------------------ Schur-complement variant
@pytest.mark.parametrize("n", [4, 8, 32, 128])
@pytest.mark.parametrize("prec", [pkg.SPDE_PREC_FP64, pkg.SPDE_PREC_MIXED])
def test_schur_apply_matches_closed_form(n, prec):
    """Scaled S = h^{-1} S_unscaled is diagonal in the DCT-II basis with eigenvalues Lambda / h."""
    import scipy.fft
    h, kappa, ns = 1.0 / n, 20.0, 2
    x = np.random.default_rng(n).standard_normal((ns, n ** 3))
    lam = mixed.schur_eigenvalues(n, h, kappa) / h
    ref = np.stack([scipy.fft.idctn(scipy.fft.dctn(v.reshape(n, n, n), norm="ortho") * lam, norm="ortho").ravel()
                    for v in x])
    dt = torch.float64 if prec == pkg.SPDE_PREC_FP64 else torch.float32
    xt = torch.tensor(x, dtype=dt, device=DEV)
    yt = torch.full_like(xt, float("nan"))
    pkg.spde_schur_apply(n, h, kappa, ns, prec, xt, yt)
    assert rel(yt.cpu().numpy().astype(np.float64), ref) <= (1e-12 if prec == pkg.SPDE_PREC_FP64 else 2e-6)


@pytest.mark.parametrize("prec", [pkg.SPDE_PREC_MIXED, pkg.SPDE_PREC_FP64])
@pytest.mark.parametrize("n,ns", [(16, 3), (64, 2), (128, 2)])
def test_schur_cg_solver_matches_closed_form(prec, n, ns):
    kappa, sigma = 20.0, 1.0
    smp = pkg.Sampler(prec, solver=pkg.SPDE_SOLVER_SCHUR_CG)
    smp.add_level(0, n)
    grid = smp.sample(0, ns, kappa, sigma, 1, 0, pkg.SPDE_OUT_GRID_GAUSSIAN | pkg.SPDE_OUT_F64)
    assert smp.stats()["max_rel_residual"] <= 1e-10
    xi = philox.normals_batch(n ** 3, 1, 0, ns)
    assert rel(grid.cpu().numpy(), mixed.solve_dct(n, kappa, sigma, xi)) <= 1e-8
    smp.close()
