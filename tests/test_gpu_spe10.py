"""GPU parity on the SPE10-sized box (Sec. 7.2's second domain): stretched Cartesian hexes split
into tets, the 1600 x 2420 x 240 ft bounding box at the corner of a cubic embedding grid."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1712_06758_gb300 as pkg  # noqa: E402
from oracle import clip, mixed, philox, project  # noqa: E402
from synth import spe10_mesh  # noqa: E402

SIDE = 2432.0  # cube side in ft, at least the bounding box's 2420 ft


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1712_06758_gb300 import build
    build.build()
    pkg.lib()


@pytest.mark.parametrize("n", [32, 64])
def test_spe10_lognormal_matches_oracle(n):
    ns, kappa, h = 2, 0.02, SIDE / n  # correlation length 1 / kappa = 50 ft
    xyz, tets = spe10_mesh(counts=(6, 22, 9))
    smp = pkg.Sampler()
    smp.add_level(0, n, (0.0, 0.0, 0.0), (SIDE, SIDE, SIDE))
    smp.attach_mesh(0, xyz, tets)
    assert smp.ntets(0) == len(tets)
    got = smp.sample(0, ns, kappa, 1.0, 8, 0, pkg.SPDE_OUT_LOGNORMAL).cpu().numpy().astype(np.float64)
    th = mixed.solve_dct(n, kappa, 1.0, philox.normals_batch(n ** 3, 8, 0, ns), h=h)
    rows = clip.coupling_rows(xyz, tets, n, lo=0.0, h=h, rows=range(0, len(tets), 17))
    ref = project.project_rows(xyz, tets, rows, th)
    idx = np.array(sorted(ref))
    refm = np.exp(np.stack([ref[t] for t in idx], axis=1))
    assert np.linalg.norm(got[:, idx] - refm) <= 1e-6 * np.linalg.norm(refm)
    smp.close()
