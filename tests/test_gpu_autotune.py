"""The autotuner (spde_autotune) and stored schedules (spde_level_set_tuning).

A tuned level must still give the exact field (oracle DCT solve within the
solver tolerance), the schedule must be no slower than the context's default
on the timed call, serving must follow the level's schedule bit for bit, and
clearing the schedule must give back the untuned bits.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1712_06758_gb300 as pkg  # noqa: E402
from oracle import mixed, philox  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1712_06758_gb300 import build
    build.build()
    pkg.lib()


def test_autotune_keeps_the_field_and_serving_follows():
    n, ns, kappa, sigma = 64, 8, 20.0, 1.0
    kind = pkg.SPDE_OUT_GRID_GAUSSIAN | pkg.SPDE_OUT_F64
    smp = pkg.Sampler(pkg.SPDE_PREC_MIXED)
    smp.add_level(0, n)
    untuned = smp.sample(0, ns, kappa, sigma, 4, 0, kind)
    t = pkg.spde_autotune(smp.ctx, 0, ns, kappa, sigma)
    assert t["evaluated"] >= 8
    assert t["ms_per_call"] <= t["default_ms"]
    assert 0.0 < t["omega"] < 1.0 and t["sweep_planes"] in (0, 8, 16, 32, 64)
    got = smp.sample(0, ns, kappa, sigma, 4, 0, kind)
    ref = mixed.solve_dct(n, kappa, sigma, philox.normals_batch(n ** 3, 4, 0, ns))
    g = got.cpu().numpy()
    assert np.linalg.norm(g - ref) <= 1e-8 * np.linalg.norm(ref)
    assert smp.stats()["max_rel_residual"] <= 1e-10
    # serving runs the level's schedule: same bits as spde_sample
    out = torch.empty_like(got)
    rid = pkg.spde_submit(smp.ctx, 0, ns, kappa, sigma, 4, 0, kind, out)
    import time
    t0 = time.time()
    while True:
        done, _, st = pkg.spde_poll(smp.ctx, rid)
        if done:
            break
        assert time.time() - t0 < 60
        time.sleep(0.002)
    assert st == pkg.SPDE_OK
    torch.cuda.synchronize()
    assert torch.equal(out, got)
    # a stored schedule applied to a fresh context gives the same bits; clearing it gives the untuned ones
    other = pkg.Sampler(pkg.SPDE_PREC_MIXED)
    other.add_level(0, n)
    pkg.spde_level_set_tuning(other.ctx, 0, t)
    assert torch.equal(other.sample(0, ns, kappa, sigma, 4, 0, kind), got)
    pkg.spde_level_set_tuning(other.ctx, 0, None)
    assert torch.equal(other.sample(0, ns, kappa, sigma, 4, 0, kind), untuned)
    with pytest.raises(pkg.SpdeError):
        pkg.spde_level_set_tuning(other.ctx, 0, dict(t, omega=1.5))
    other.close()
    smp.close()
