"""The bounded device waits give up and report, without faulting or hanging the GPU.

The multigrid sweeps wait on mbarriers for their TMA plane copies.  Each wait
is limited to about one second; a wait that runs out raises a device fault
word that the host turns into SPDE_ETIMEOUT.  spde_check_wait_limit runs one
CTA whose barrier never completes (no arrival is ever made), so its wait must
run out; afterwards the context must still solve correctly.
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


def test_wait_runs_out_and_context_stays_usable():
    ms = pkg.spde_check_wait_limit(0)
    assert 900.0 <= ms <= 5000.0
    n, ns = 32, 2
    smp = pkg.Sampler()
    smp.add_level(0, n)
    got = smp.sample(0, ns, 20.0, 1.0, 3, 0, pkg.SPDE_OUT_GRID_GAUSSIAN | pkg.SPDE_OUT_F64).cpu().numpy()
    ref = mixed.solve_dct(n, 20.0, 1.0, philox.normals_batch(n ** 3, 3, 0, ns))
    assert np.linalg.norm(got - ref) <= 1e-8 * np.linalg.norm(ref)
    smp.close()


def test_probe_does_not_disturb_a_running_lane():
    """The probe raises a fault word of its own: a serving lane whose sweeps run
    before, while and after the probe's wait gives up (about 1.3 s of work)
    keeps its own word clear, finishes with SPDE_OK and gives the same bits as
    spde_sample."""
    import time
    n, ns, chunk = 128, 320, 64
    kind = pkg.SPDE_OUT_GRID_GAUSSIAN | pkg.SPDE_OUT_F64
    smp = pkg.Sampler(pkg.SPDE_PREC_MIXED, tol=1e-10)
    smp.add_level(0, n)
    out = torch.empty((ns, n ** 3), dtype=torch.float64, device="cuda")
    rid = pkg.spde_submit(smp.ctx, 0, ns, 20.0, 1.0, 9, 0, kind, out)
    ms = pkg.spde_check_wait_limit(0)  # runs while the lane works
    assert 900.0 <= ms <= 5000.0
    t0 = time.time()
    while True:
        done, _, st = pkg.spde_poll(smp.ctx, rid)
        if done:
            break
        assert time.time() - t0 < 120.0
        time.sleep(0.005)
    assert st == pkg.SPDE_OK
    for k in range(0, ns, chunk):
        ref = smp.sample(0, chunk, 20.0, 1.0, 9, k, kind)
        torch.cuda.synchronize()
        assert torch.equal(out[k:k + chunk], ref), k
    pkg.spde_precond_status()  # the step-level preconditioner words stay clear too
    smp.close()
