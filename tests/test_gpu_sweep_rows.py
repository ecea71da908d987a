"""The whole-row sweep tiles (k_mg_down_rows / k_mg_up_rows) against the 32 x 16 tiles.

Levels 32, 64 or 128 cells wide run their FP32 V-cycle sweeps on tiles of
whole x rows (sweep_rows = 1, the default).  Every cell takes the same
arithmetic in the same order on both tilings (the sums of products are
written as explicit fused multiply-adds), so the preconditioner must give the
same bits with either; sampling differs only through the grouping of the
b.y partial sums that MINRES reads, so its results agree to the solve's
tolerance.  The oracle V-cycle tests (test_gpu_parity, test_gpu_box) run the
default, i.e. these tiles.
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


def _opts(rows):
    o = pkg.spde_opts_init()
    o.sweep_rows = rows
    return o


def _rand(dims, ns, seed):
    r = np.random.default_rng(seed).standard_normal((ns, 4 * int(np.prod(dims))))
    r[:, wall_mask(dims)] = 0.0
    return torch.tensor(r, dtype=torch.float32, device="cuda")


@pytest.mark.parametrize("n,ns", [(32, 5), (64, 3), (128, 2), (256, 1)])
def test_rows_give_the_same_vcycle_bits(n, ns):
    r = _rand((n, n, n), ns, n)
    z = [torch.full_like(r, float("nan")) for _ in range(2)]
    for rows in (0, 1):
        pkg.spde_precond(n, 1.0 / n, 20.0, ns, pkg.SPDE_PREC_MIXED, r, z[rows], _opts(rows))
    torch.cuda.synchronize()
    assert torch.isfinite(z[1]).all()
    assert torch.equal(z[0], z[1])
    pkg.spde_precond_status()


@pytest.mark.parametrize("dims", [(64, 32, 16), (128, 64, 32), (32, 64, 16), (64, 16, 32)])
def test_rows_give_the_same_bits_on_boxes(dims):
    """Boxes: rows only where the level's y extent is a multiple of the tile's rows
    (16, or 32 on 32-wide levels); other levels keep the 32 x 16 tiles."""
    ns = 2
    r = _rand(dims, ns, sum(dims))
    z = [torch.full_like(r, float("nan")) for _ in range(2)]
    for rows in (0, 1):
        pkg.spde_precond_box(dims, 0.02, 13.0, ns, pkg.SPDE_PREC_MIXED, r, z[rows], _opts(rows))
    torch.cuda.synchronize()
    assert torch.isfinite(z[1]).all()
    assert torch.equal(z[0], z[1])
    pkg.spde_precond_status()


@pytest.mark.parametrize("n,planes", [(64, 8), (64, 16), (64, 32), (64, 64), (128, 64)])
def test_rows_with_each_march_length(n, planes):
    """The z extent per CTA (sweep_planes) changes the tiling, not a bit of the V-cycle."""
    ns = 3
    r = _rand((n, n, n), ns, 7)
    ref = torch.full_like(r, float("nan"))
    pkg.spde_precond(n, 1.0 / n, 20.0, ns, pkg.SPDE_PREC_MIXED, r, ref, _opts(0))
    o = _opts(1)
    o.sweep_planes = planes
    got = torch.full_like(r, float("nan"))
    pkg.spde_precond(n, 1.0 / n, 20.0, ns, pkg.SPDE_PREC_MIXED, r, got, o)
    torch.cuda.synchronize()
    assert torch.equal(ref, got)


def test_rows_sample_agrees_with_tiles():
    n, S = 128, 8
    kind = pkg.SPDE_OUT_GRID_GAUSSIAN | pkg.SPDE_OUT_F64
    outs = []
    for rows in (0, 1):
        smp = pkg.Sampler(pkg.SPDE_PREC_MIXED, tol=1e-10, sweep_rows=rows)
        smp.add_level(0, n)
        outs.append(smp.sample(0, S, 20.0, 1.0, 5, 0, kind))
        st = smp.stats()
        assert st["max_rel_residual"] <= 1e-10
        smp.close()
    a, b = outs
    assert float((a - b).norm() / a.norm()) <= 1e-8


def test_rows_serving_lane_per_column_kappa():
    """A serving lane carries one kappa per column (the sweep coefficients come from a
    per-column table): each request equals spde_sample of its own kappa, bit for bit,
    and the 32 x 16 tiles to the solve's tolerance."""
    import time
    n, ns = 64, 2
    kind = pkg.SPDE_OUT_GRID_GAUSSIAN | pkg.SPDE_OUT_F64
    got = {}
    for rows in (0, 1):
        smp = pkg.Sampler(pkg.SPDE_PREC_MIXED, tol=1e-10, serve_max_batch=8, sweep_rows=rows)
        smp.add_level(0, n)
        reqs = []
        for k, kappa in enumerate((10.0, 20.0, 40.0, 15.0)):
            out = torch.full((ns, n ** 3), float("nan"), dtype=torch.float64, device="cuda")
            reqs.append((pkg.spde_submit(smp.ctx, 0, ns, kappa, 1.0, 30 + k, 0, kind, out), kappa, k, out))
        t0 = time.time()
        pending = {r[0] for r in reqs}
        while pending:
            for rid in list(pending):
                done, _, st = pkg.spde_poll(smp.ctx, rid)
                if done:
                    assert st == pkg.SPDE_OK
                    pending.discard(rid)
            assert time.time() - t0 < 120.0
            time.sleep(0.002)
        for rid, kappa, k, out in reqs:
            alone = smp.sample(0, ns, kappa, 1.0, 30 + k, 0, kind)
            assert torch.equal(out, alone), (rows, kappa)
            got[(rows, k)] = out
        smp.close()
    for k in range(4):
        a, b = got[(0, k)], got[(1, k)]
        assert float((a - b).norm() / a.norm()) <= 1e-8
