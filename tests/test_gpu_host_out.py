"""Outputs in host memory: spde_sample and spde_sample_fields with a host buffer.

Pinned host memory of the sampling device is written by the output kernels
directly (it is mapped into the device's address space); other host memory
is staged on the device and copied.  Either way the call returns once the
host buffer holds the result, and the values are the same bits as those of a
device output of the same draw.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1712_06758_gb300 as pkg  # noqa: E402
from synth import lprism_mesh  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1712_06758_gb300 import build
    build.build()
    pkg.lib()


N, S = 32, 8


def _sampler(graphs):
    smp = pkg.Sampler(pkg.SPDE_PREC_MIXED, tol=1e-10, use_graphs=graphs)
    smp.add_level(0, N)
    xyz, tets = lprism_mesh(3 * N // 4)
    smp.attach_mesh(0, xyz, tets)
    return smp


def _host_buffers(shape, dtype):
    pinned = torch.empty(shape, dtype=dtype, pin_memory=True).numpy()
    pageable = np.empty(shape, dtype=np.float64 if dtype == torch.float64 else np.float32)
    return pinned, pageable


@pytest.mark.parametrize("graphs", [1, 0])
@pytest.mark.parametrize("kind", [pkg.SPDE_OUT_LOGNORMAL, pkg.SPDE_OUT_GRID_GAUSSIAN | pkg.SPDE_OUT_F64])
def test_host_outputs_are_the_device_bits(graphs, kind):
    smp = _sampler(graphs)
    per = N ** 3 if (kind & 15) == pkg.SPDE_OUT_GRID_GAUSSIAN else smp.ntets(0)
    dtype = torch.float64 if kind & pkg.SPDE_OUT_F64 else torch.float32
    dev = torch.empty((S, per), dtype=dtype, device="cuda")
    stream = torch.cuda.current_stream()
    pkg.spde_sample(smp.ctx, 0, S, 20.0, 1.3, 9, 40, kind, dev, stream)
    pkg.spde_wait(smp.ctx)
    torch.cuda.synchronize()
    ref = dev.cpu().numpy()
    assert np.isfinite(ref).all()
    for host in _host_buffers((S, per), dtype):
        host[...] = np.nan
        pkg.spde_sample(smp.ctx, 0, S, 20.0, 1.3, 9, 40, kind, host, stream)  # returns with host written
        assert np.array_equal(host, ref)
    smp.close()


def test_fields_into_pinned_host_memory():
    smp = _sampler(1)
    c = (np.arange(N) + 0.5) / N
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    smp.set_fields(0, (10.0 + 20.0 * x).ravel(), (0.5 + y).ravel())
    nt = smp.ntets(0)
    dev = torch.empty((S, nt), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    smp.sample_fields(0, S, 3, 0, pkg.SPDE_OUT_LOGNORMAL, dev, stream)
    torch.cuda.synchronize()
    pinned, _ = _host_buffers((S, nt), torch.float32)
    smp.sample_fields(0, S, 3, 0, pkg.SPDE_OUT_LOGNORMAL, pinned, stream)
    assert np.array_equal(pinned, dev.cpu().numpy())
    smp.close()
