"""The asynchronous, graph-driven sampling path (spde_sample with use_graphs = 1).

Each refinement solve runs as one captured CUDA graph whose conditional
while-nodes take the refinement steps and MINRES iterations, every
convergence test made on the device; spde_sample returns once noise, graph
and projection are enqueued.  The graph launches the kernels of the
synchronous path in the same order with the same arguments, so results must
be the same bits; two calls on two streams must return at once (host time far
below device time) and give the same bits as the blocking path.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1712_06758_gb300 as pkg  # noqa: E402
from oracle import mixed, philox  # noqa: E402
from synth import box_mesh, lprism_mesh  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1712_06758_gb300 import build
    build.build()
    pkg.lib()


def _pair(prec=pkg.SPDE_PREC_MIXED, **kw):
    return pkg.Sampler(prec, use_graphs=1, **kw), pkg.Sampler(prec, use_graphs=0, **kw)


@pytest.mark.parametrize("prec,n,ns", [(pkg.SPDE_PREC_MIXED, 32, 7), (pkg.SPDE_PREC_MIXED, 64, 16),
                                       (pkg.SPDE_PREC_FP64, 16, 2)])
def test_graph_path_is_bitwise_the_synchronous_path(prec, n, ns):
    xyz, tets = lprism_mesh(n * 3 // 4) if n >= 32 else box_mesh((0.15,) * 3, (0.85,) * 3, 12)
    a, b = _pair(prec)
    for smp in (a, b):
        smp.add_level(0, n)
        smp.attach_mesh(0, xyz, tets)
    for kind in (pkg.SPDE_OUT_GRID_GAUSSIAN | pkg.SPDE_OUT_F64, pkg.SPDE_OUT_LOGNORMAL):
        for kappa in (20.0, 35.0):  # a second kappa re-captures the graph
            ga = a.sample(0, ns, kappa, 1.3, 5, 11, kind)
            gb = b.sample(0, ns, kappa, 1.3, 5, 11, kind)
            torch.cuda.synchronize()
            assert torch.equal(ga, gb), (kind, kappa)
    sa, sb = a.stats(), b.stats()
    assert sa["outer_iters"] == sb["outer_iters"] and sa["max_rel_residual"] == sb["max_rel_residual"]
    assert sa["max_rel_residual"] <= 1e-10
    a.close()
    b.close()


def test_graph_path_fields_and_coupled_pairs():
    n = 32
    c = (np.arange(n) + 0.5) / n
    fz, fy, fx = np.meshgrid(c, c, c, indexing="ij")
    kap = (10.0 + 30.0 * fx + 8.0 * np.sin(2 * np.pi * fz)).ravel()
    sig = (0.5 + 1.5 * fy).ravel()
    a, b = _pair()
    kind = pkg.SPDE_OUT_GRID_GAUSSIAN | pkg.SPDE_OUT_F64
    for smp in (a, b):
        smp.add_level(0, n)
        smp.add_level(1, n // 2)
        smp.set_fields(0, kap, sig)
    fa = a.sample_fields(0, 5, 3, 0, kind)
    fb = b.sample_fields(0, 5, 3, 0, kind)
    torch.cuda.synchronize()
    assert torch.equal(fa, fb)
    outs = []
    for smp in (a, b):
        fine = torch.empty((4, n ** 3), dtype=torch.float64, device="cuda")
        coarse = torch.empty((4, (n // 2) ** 3), dtype=torch.float64, device="cuda")
        smp.set_fields(0, None, None)
        pkg.spde_sample_coupled(smp.ctx, 0, 1, 4, 20.0, 1.0, 9, 2, kind, fine, coarse)
        pkg.spde_wait(smp.ctx)
        outs.append((fine, coarse))
    torch.cuda.synchronize()
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    a.close()
    b.close()


def test_iteration_cap_is_reported_by_wait():
    a, b = _pair(max_iter=2, max_outer=1)
    for smp in (a, b):
        smp.add_level(0, 16)
    out = torch.empty((1, 16 ** 3), dtype=torch.float64, device="cuda")
    pkg.spde_sample(a.ctx, 0, 1, 10.0, 1.0, 1, 0, pkg.SPDE_OUT_GRID_GAUSSIAN | pkg.SPDE_OUT_F64, out)  # returns
    with pytest.raises(pkg.SpdeError) as ei:
        pkg.spde_wait(a.ctx)
    assert ei.value.status == pkg.SPDE_ENOCONV
    pkg.spde_wait(a.ctx)  # reported once
    with pytest.raises(pkg.SpdeError) as ei:
        ref = b.sample(0, 1, 10.0, 1.0, 1, 0, pkg.SPDE_OUT_GRID_GAUSSIAN | pkg.SPDE_OUT_F64)
    assert ei.value.status == pkg.SPDE_ENOCONV
    ref = torch.empty_like(out)
    with pytest.raises(pkg.SpdeError):
        pkg.spde_sample(b.ctx, 0, 1, 10.0, 1.0, 1, 0, pkg.SPDE_OUT_GRID_GAUSSIAN | pkg.SPDE_OUT_F64, ref)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)  # the same last iterate
    assert a.stats()["max_rel_residual"] == b.stats()["max_rel_residual"] > 1e-10
    a.close()
    b.close()


def test_two_streams_return_at_once_and_match_the_blocking_path():
    n, ns, kappa, sigma, seed = 128, 32, 20.0, 1.0, 7
    kind = pkg.SPDE_OUT_GRID_GAUSSIAN
    smp = pkg.Sampler(pkg.SPDE_PREC_MIXED, use_graphs=1)
    smp.add_level(0, n)
    warm = torch.empty((ns, n ** 3), dtype=torch.float32, device="cuda")
    smp.sample(0, ns, kappa, sigma, seed, 1000, kind, warm)  # captures the graph
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    o1 = torch.empty((ns, n ** 3), dtype=torch.float32, device="cuda")
    o2 = torch.empty_like(o1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s1)
    t0 = time.perf_counter()
    pkg.spde_sample(smp.ctx, 0, ns, kappa, sigma, seed, 0, kind, o1, s1)
    pkg.spde_sample(smp.ctx, 0, ns, kappa, sigma, seed, ns, kind, o2, s2)
    host_ms = 1000.0 * (time.perf_counter() - t0)
    e1.record(s2)
    torch.cuda.synchronize()
    dev_ms = e0.elapsed_time(e1)
    pkg.spde_wait(smp.ctx)
    assert host_ms < 0.25 * dev_ms, (host_ms, dev_ms)  # no host synchronisation inside the calls
    blk = pkg.Sampler(pkg.SPDE_PREC_MIXED, use_graphs=0)
    blk.add_level(0, n)
    r1 = blk.sample(0, ns, kappa, sigma, seed, 0, kind)
    r2 = blk.sample(0, ns, kappa, sigma, seed, ns, kind)
    torch.cuda.synchronize()
    assert torch.equal(o1, r1) and torch.equal(o2, r2)
    # and the field is the one the oracle's exact solve gives
    ref = mixed.solve_dct(n, kappa, sigma, philox.normals_batch(n ** 3, seed, 0, 2))
    got = o1[:2].double().cpu().numpy()
    assert np.linalg.norm(got - ref) <= 1e-6 * np.linalg.norm(ref)
    print("two async calls: host %.2f ms, device %.1f ms" % (host_ms, dev_ms))
    smp.close()
    blk.close()
