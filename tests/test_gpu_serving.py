"""Serving path (spde_submit / spde_poll / spde_cancel): continuous batching.

Each result must be the same alone (spde_sample) and in a mix of requests
for several levels, kappas, sigmas and sizes submitted together; tolerance:
bitwise, since a column follows exactly the per-column arithmetic of the
batched path.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1712_06758_gb300 as pkg  # noqa: E402
from synth import box_mesh, lprism_mesh  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1712_06758_gb300 import build
    build.build()
    pkg.lib()


def _hierarchy(smp):
    meshes = {0: (16, box_mesh((0.15,) * 3, (0.85,) * 3, 8)), 1: (32, lprism_mesh(24))}
    for lvl, (n, (xyz, tets)) in meshes.items():
        smp.add_level(lvl, n)
        smp.attach_mesh(lvl, xyz, tets)
    return meshes


def _wait(smp, ids, timeout=120.0):
    res = {}
    t0 = time.time()
    while len(res) < len(ids):
        for i in ids:
            if i in res:
                continue
            done, lat, st = pkg.spde_poll(smp.ctx, i)
            if done:
                res[i] = (lat, st)
        assert time.time() - t0 < timeout, "requests did not finish"
        time.sleep(0.002)
    return res


def test_mixed_stream_matches_alone():
    smp = pkg.Sampler(pkg.SPDE_PREC_MIXED, serve_max_batch=6)
    meshes = _hierarchy(smp)
    rng = np.random.default_rng(4)
    reqs = []
    for k in range(14):
        lvl = int(rng.integers(0, 2))
        kappa = [10.0, 20.0, 40.0][int(rng.integers(0, 3))]  # kappas share a level's lane
        sigma = float(rng.uniform(0.5, 2.0))
        ns = int(rng.integers(1, 9))
        kind = [pkg.SPDE_OUT_LOGNORMAL, pkg.SPDE_OUT_GAUSSIAN | pkg.SPDE_OUT_F64,
                pkg.SPDE_OUT_GRID_GAUSSIAN][k % 3]
        n = meshes[lvl][0]
        per = n ** 3 if (kind & 15) == pkg.SPDE_OUT_GRID_GAUSSIAN else len(meshes[lvl][1][1])
        dt = torch.float64 if kind & pkg.SPDE_OUT_F64 else torch.float32
        out = torch.full((ns, per), float("nan"), dtype=dt, device="cuda")
        seed, first = 1000 + k, 7 * k
        rid = pkg.spde_submit(smp.ctx, lvl, ns, kappa, sigma, seed, first, kind, out)
        reqs.append((rid, lvl, ns, kappa, sigma, seed, first, kind, out))
    res = _wait(smp, [r[0] for r in reqs])
    for rid, lvl, ns, kappa, sigma, seed, first, kind, out in reqs:
        lat, st = res[rid]
        assert st == pkg.SPDE_OK and lat > 0
        alone = torch.full_like(out, float("nan"))
        pkg.spde_sample(smp.ctx, lvl, ns, kappa, sigma, seed, first, kind, alone)
        assert torch.equal(out, alone), (rid, lvl, ns, kappa)
    smp.close()


def test_cancel_and_errors():
    smp = pkg.Sampler(pkg.SPDE_PREC_MIXED, serve_max_batch=2)
    _hierarchy(smp)
    out = torch.zeros((40, 32 ** 3), dtype=torch.float32, device="cuda")
    rid = pkg.spde_submit(smp.ctx, 1, 40, 20.0, 1.0, 3, 0, pkg.SPDE_OUT_GRID_GAUSSIAN, out)
    with pytest.raises(pkg.SpdeError) as ei:  # grids cannot change while requests are in flight
        smp.add_level(1, 32)
    assert ei.value.status == pkg.SPDE_EBUSY
    pkg.spde_cancel(smp.ctx, rid)
    lat, st = _wait(smp, [rid])[rid]
    assert st == pkg.SPDE_ECANCELED
    with pytest.raises(pkg.SpdeError):
        pkg.spde_poll(smp.ctx, rid)  # reported once, then forgotten
    with pytest.raises(pkg.SpdeError):
        pkg.spde_cancel(smp.ctx, 12345)
    host = np.zeros((1, 16 ** 3), dtype=np.float32)
    with pytest.raises(pkg.SpdeError) as ei:
        pkg.spde_submit(smp.ctx, 0, 1, 10.0, 1.0, 1, 0, pkg.SPDE_OUT_GRID_GAUSSIAN, host)
    assert ei.value.status == pkg.SPDE_EINVAL
    smp.close()
    plain = pkg.Sampler(pkg.SPDE_PREC_FP64)
    plain.add_level(0, 16)
    with pytest.raises(pkg.SpdeError):
        pkg.spde_submit(plain.ctx, 0, 1, 10.0, 1.0, 1, 0, pkg.SPDE_OUT_GRID_GAUSSIAN,
                        torch.zeros((1, 16 ** 3), device="cuda"))
    plain.close()


def test_admission_under_a_small_budget():
    """A budget that holds one lane at a time: lanes take turns, results stay exact."""
    smp = pkg.Sampler(pkg.SPDE_PREC_MIXED, serve_max_batch=4)
    smp.add_level(0, 16)
    smp.add_level(1, 32)
    need = pkg.spde_query_footprint(smp.ctx, 1, 4)
    smp.close()
    smp = pkg.Sampler(pkg.SPDE_PREC_MIXED, serve_max_batch=4, serve_budget_bytes=int(need * 1.2))
    smp.add_level(0, 16)
    smp.add_level(1, 32)
    outs, ids = [], []
    for k, (lvl, kappa) in enumerate([(1, 20.0), (0, 10.0), (1, 10.0), (0, 20.0)]):
        n = [16, 32][lvl]
        out = torch.full((3, n ** 3), float("nan"), device="cuda")
        ids.append(pkg.spde_submit(smp.ctx, lvl, 3, kappa, 1.0, 50 + k, 0, pkg.SPDE_OUT_GRID_GAUSSIAN, out))
        outs.append((lvl, kappa, k, out))
    res = _wait(smp, ids)
    assert all(st == pkg.SPDE_OK for _, st in res.values())
    for lvl, kappa, k, out in outs:
        alone = torch.full_like(out, float("nan"))
        pkg.spde_sample(smp.ctx, lvl, 3, kappa, 1.0, 50 + k, 0, pkg.SPDE_OUT_GRID_GAUSSIAN, alone)
        assert torch.equal(out, alone)
    smp.close()


def test_batch_size_does_not_change_a_column():
    """A column's bits do not depend on how many columns share its batch: the same
    samples drawn 3 at a time, 64 at a time and through a serving lane (64^3, where
    the sweeps' tiling could depend on the batch size)."""
    n, kind = 64, pkg.SPDE_OUT_GRID_GAUSSIAN | pkg.SPDE_OUT_F64
    smp = pkg.Sampler(pkg.SPDE_PREC_MIXED)
    smp.add_level(0, n)
    big = smp.sample(0, 64, 20.0, 1.0, 8, 0, kind)
    small = smp.sample(0, 3, 20.0, 1.0, 8, 5, kind)
    torch.cuda.synchronize()
    assert torch.equal(big[5:8], small)
    out = torch.empty((3, n ** 3), dtype=torch.float64, device="cuda")
    rid = pkg.spde_submit(smp.ctx, 0, 3, 20.0, 1.0, 8, 5, kind, out)
    _, st = _wait(smp, [rid])[rid]
    assert st == pkg.SPDE_OK
    assert torch.equal(out, small)
    smp.close()
