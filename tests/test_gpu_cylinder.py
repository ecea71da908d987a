"""GPU parity on the quarter-cylinder mesh (stand-in for the paper's crooked pipe, Sec. 7.1):
strongly stretched tets, a curved boundary, embedded in a cubic box of side 8."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1712_06758_gb300 as pkg  # noqa: E402
from oracle import clip, mixed, philox, project  # noqa: E402
from synth import quarter_cylinder_mesh  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1712_06758_gb300 import build
    build.build()
    pkg.lib()


@pytest.mark.parametrize("n", [32, 64])
def test_cylinder_lognormal_matches_oracle(n):
    ns, kappa, h = 2, 2.0, 8.0 / n
    xyz, tets = quarter_cylinder_mesh(8, 12, 14)
    smp = pkg.Sampler()
    smp.add_level(0, n, (0.0, 0.0, 0.0), (8.0, 8.0, 8.0))
    smp.attach_mesh(0, xyz, tets)  # rejects any row whose intersections miss the tet volume
    assert smp.ntets(0) == len(tets)
    got = smp.sample(0, ns, kappa, 1.0, 6, 0, pkg.SPDE_OUT_LOGNORMAL).cpu().numpy().astype(np.float64)
    th = mixed.solve_dct(n, kappa, 1.0, philox.normals_batch(n ** 3, 6, 0, ns), h=h)
    rows = clip.coupling_rows(xyz, tets, n, lo=0.0, h=h, rows=range(0, len(tets), 23))
    ref = project.project_rows(xyz, tets, rows, th)
    idx = np.array(sorted(ref))
    refm = np.exp(np.stack([ref[t] for t in idx], axis=1))
    assert np.linalg.norm(got[:, idx] - refm) <= 1e-6 * np.linalg.norm(refm)
    smp.close()


def test_cylinder_on_a_box_grid_matches_oracle():
    """The same mesh turned so that its axis runs along x ((x, y, z) -> (z, x, y), a rotation),
    on a 32 x 16 x 16 box grid of spacing 1/4: the box [0,8] x [0,4] x [0,4] around it."""
    dims, h, ns, kappa = (32, 16, 16), 0.25, 2, 2.0
    xyz, tets = quarter_cylinder_mesh(8, 12, 14)
    xyz = np.ascontiguousarray(xyz[:, [2, 0, 1]])
    smp = pkg.Sampler()
    smp.add_level(0, dims, (0.0, 0.0, 0.0), tuple(h * v for v in dims))
    smp.attach_mesh(0, xyz, tets)
    assert smp.ntets(0) == len(tets)
    got = smp.sample(0, ns, kappa, 1.0, 6, 0, pkg.SPDE_OUT_LOGNORMAL).cpu().numpy().astype(np.float64)
    th = mixed.solve_dct(dims, kappa, 1.0, philox.normals_batch(int(np.prod(dims)), 6, 0, ns), h=h)
    rows = clip.coupling_rows(xyz, tets, dims, lo=0.0, h=h, rows=range(0, len(tets), 23))
    ref = project.project_rows(xyz, tets, rows, th)
    idx = np.array(sorted(ref))
    refm = np.exp(np.stack([ref[t] for t in idx], axis=1))
    assert np.linalg.norm(got[:, idx] - refm) <= 1e-6 * np.linalg.norm(refm)
    smp.close()
