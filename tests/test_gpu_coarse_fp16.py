"""FP16 storage of the coarse multigrid levels (opts.coarse_fp16).

The levels held by the one-CTA coarse kernel (at most 4096 cells) may be
stored in FP16, each column scaled by its largest value, with FP32
arithmetic.  The preconditioner then differs from the FP32 one by FP16
rounding only, and the refined field still meets the tolerance against the
oracle's exact solve, in about as many iterations.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1712_06758_gb300 as pkg  # noqa: E402
from oracle import mixed, philox  # noqa: E402
from tests.layout import wall_mask  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1712_06758_gb300 import build
    build.build()
    pkg.lib()


@pytest.mark.parametrize("n,scale", [(16, 1.0), (16, 1e-6), (8, 3e4)])
def test_fp16_coarse_preconditioner_is_the_fp32_one_to_rounding(n, scale):
    """Every level of these grids is held by the coarse kernel; the column scaling
    keeps tiny and large inputs within FP16 range."""
    ns = 3
    r = np.random.default_rng(n).standard_normal((ns, 4 * n ** 3)) * scale
    r[:, wall_mask(n)] = 0.0
    rr = torch.tensor(r, dtype=torch.float32, device="cuda")
    z32, z16 = torch.empty_like(rr), torch.empty_like(rr)
    o16 = pkg.spde_opts_init()
    o16.coarse_fp16 = 1
    pkg.spde_precond(n, 1.0 / n, 20.0, ns, pkg.SPDE_PREC_MIXED, rr, z32)
    pkg.spde_precond(n, 1.0 / n, 20.0, ns, pkg.SPDE_PREC_MIXED, rr, z16, opts=o16)
    torch.cuda.synchronize()
    a, b = z16.double().cpu().numpy(), z32.double().cpu().numpy()
    assert np.all(np.isfinite(a))
    rel = np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)
    assert rel.max() <= 5e-3 and rel.max() > 0.0


@pytest.mark.parametrize("n", [32, 64])
def test_fp16_coarse_sampling_meets_the_tolerance(n):
    ns, kappa, sigma, seed = 4, 20.0, 1.0, 6
    kind = pkg.SPDE_OUT_GRID_GAUSSIAN | pkg.SPDE_OUT_F64
    ref = mixed.solve_dct(n, kappa, sigma, philox.normals_batch(n ** 3, seed, 0, ns))
    its = {}
    for fp16 in (0, 1):
        smp = pkg.Sampler(pkg.SPDE_PREC_MIXED, coarse_fp16=fp16)
        smp.add_level(0, n)
        got = smp.sample(0, ns, kappa, sigma, seed, 0, kind).cpu().numpy()
        st = smp.stats()
        assert np.linalg.norm(got - ref) <= 1e-8 * np.linalg.norm(ref)
        assert st["max_rel_residual"] <= 1e-10
        its[fp16] = (st["outer_iters"], st["inner_iters"])
        smp.close()
    print("n=%d: FP32 coarse %s, FP16 coarse %s (outer, inner iterations)" % (n, its[0], its[1]))
    assert its[1][0] <= its[0][0] + 1
