"""The allocation-free preconditioner entry point (spde_precond_noalloc).

It serves callers that cannot allocate device memory (memory owned by
another allocator, or loops that cannot afford cudaMalloc's device
synchronisation).  Through the C ABI, two calls in a row must give exactly
what the allocating entry point spde_precond gives (same kernels, same plan,
only the scratch lives elsewhere); a call on a shape never seen before must
leave the device's free memory unchanged; a request that needs more than the
static scratch, or a grid beyond the library's limit, must be rejected
before any work.  Kept in a file of its own that pytest collects last.
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
    for call, seed in enumerate((11, 12)):  # two calls in a row share the static scratch
        r = _rand(n, ns, seed + n, dt)
        ref = torch.full_like(r, float("nan"))
        got = torch.full_like(r, float("nan"))
        pkg.spde_precond(n, h, kappa, ns, prec, r, ref)
        pkg.spde_precond_noalloc(n, h, kappa, ns, prec, r, got)
        torch.cuda.synchronize()
        assert torch.isfinite(got).all(), call
        assert torch.equal(got, ref), call  # the same kernels on the same plan: bitwise equal
    pkg.spde_precond_status()  # neither call's sweeps gave up


def test_noalloc_allocates_no_device_memory():
    n, ns, prec = 64, 6, pkg.SPDE_PREC_MIXED  # a shape no other call in this file uses
    r = _rand(n, ns, 5, torch.float32)
    z1 = torch.empty_like(r)
    z2 = torch.empty_like(r)
    warm = _rand(16, 1, 6, torch.float32)  # loads the kernels (module loading is lazy)
    pkg.spde_precond_noalloc(16, 1.0 / 16, 20.0, 1, prec, warm, torch.empty_like(warm))
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    pkg.spde_precond_noalloc(n, 1.0 / n, 20.0, ns, prec, r, z1)
    pkg.spde_precond_noalloc(n, 1.0 / n, 20.0, ns, prec, r, z2)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.equal(z1, z2) and torch.isfinite(z1).all()


def test_noalloc_rejects_requests_beyond_the_static_scratch():
    n = 256
    r = torch.zeros(4, device="cuda")  # never touched: the size check comes first
    with pytest.raises(pkg.SpdeError) as ei:
        pkg.spde_precond_noalloc(n, 1.0 / n, 20.0, 4, pkg.SPDE_PREC_FP64, r, r)
    assert ei.value.status == pkg.SPDE_EINVAL
    assert "static scratch" in str(ei.value)
    with pytest.raises(pkg.SpdeError) as ei:  # beyond the grid limit of every entry point
        pkg.spde_precond_noalloc(1024, 1.0 / 1024, 20.0, 1, pkg.SPDE_PREC_MIXED, r, r)
    assert ei.value.status == pkg.SPDE_EINVAL
    assert "static scratch" not in str(ei.value)
