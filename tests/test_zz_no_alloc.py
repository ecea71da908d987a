"""The allocation-free preconditioner entry point (spde_precond_noalloc).

It serves callers that cannot allocate device memory (memory owned by
another allocator, or loops that cannot afford cudaMalloc's device
synchronisation).  Through the C ABI, two calls in a row must match the
allocating entry point spde_precond within the preconditioner tolerances
used elsewhere in the suite; a request that needs more than the static
scratch must be rejected before any work.  Kept in a file of its own that
pytest collects last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1712_06758_gb300 as pkg  # noqa: E402
from tests.layout import wall_mask  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1712_06758_gb300 import build
    build.build()
    pkg.lib()


def _rand(n, ns, seed, dt):
    r = np.random.default_rng(seed).standard_normal((ns, 4 * n ** 3))
    r[:, wall_mask(n)] = 0.0
    return torch.tensor(r, dtype=dt, device="cuda")


@pytest.mark.parametrize("n,ns,prec", [(64, 3, pkg.SPDE_PREC_FP64), (128, 2, pkg.SPDE_PREC_MIXED),
                                       (32, 5, pkg.SPDE_PREC_MIXED), (16, 2, pkg.SPDE_PREC_FP64)])
def test_noalloc_matches_allocating_entry_point(n, ns, prec):
    h, kappa = 1.0 / n, 20.0
    dt = torch.float64 if prec == pkg.SPDE_PREC_FP64 else torch.float32
    tol = 1e-12 if prec == pkg.SPDE_PREC_FP64 else 2e-6
    for call, seed in enumerate((11, 12)):  # two calls in a row share the static scratch
        r = _rand(n, ns, seed + n, dt)
        ref = torch.full_like(r, float("nan"))
        got = torch.full_like(r, float("nan"))
        pkg.spde_precond(n, h, kappa, ns, prec, r, ref)
        pkg.spde_precond_noalloc(n, h, kappa, ns, prec, r, got)
        torch.cuda.synchronize()
        a = got.cpu().numpy().astype(np.float64)
        b = ref.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(a)), call
        assert np.linalg.norm(a - b) <= tol * np.linalg.norm(b), call


def test_noalloc_rejects_requests_beyond_the_static_scratch():
    n = 256
    r = torch.zeros(4, device="cuda")  # never touched: the size check comes first
    with pytest.raises(pkg.SpdeError) as ei:
        pkg.spde_precond_noalloc(n, 1.0 / n, 20.0, 4, pkg.SPDE_PREC_FP64, r, r)
    assert ei.value.status == pkg.SPDE_EINVAL
    assert "static scratch" in str(ei.value)
