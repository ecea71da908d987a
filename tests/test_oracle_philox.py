"""Pins of the oracle's Philox4x32-10 and white-noise mapping (Sec. 4.2)."""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest
from scipy import stats

from oracle import philox


def test_two_statements_agree():
    rng = np.random.default_rng(7)
    ctr = rng.integers(0, 2 ** 32, size=(500, 4), dtype=np.uint64)
    key = rng.integers(0, 2 ** 32, size=(500, 2), dtype=np.uint64)
    vec = philox.philox4x32_10(ctr[:, 0], ctr[:, 1], ctr[:, 2], ctr[:, 3], key[:, 0], key[:, 1])
    vec = np.stack(vec, axis=1)
    for i in range(len(ctr)):
        assert tuple(int(v) for v in vec[i]) == philox.philox4x32_10_int(ctr[i], key[i])


TRITON_SCRIPT = textwrap.dedent("""
    import os, sys
    os.environ["TRITON_INTERPRET"] = "1"
    import numpy as np, torch, triton, triton.language as tl

    @triton.jit
    def k(ctr_ptr, out_ptr, seed, N: tl.constexpr):
        offs = tl.arange(0, N)
        c0 = tl.load(ctr_ptr + offs * 4 + 0).to(tl.uint32, bitcast=True)
        c1 = tl.load(ctr_ptr + offs * 4 + 1).to(tl.uint32, bitcast=True)
        c2 = tl.load(ctr_ptr + offs * 4 + 2).to(tl.uint32, bitcast=True)
        c3 = tl.load(ctr_ptr + offs * 4 + 3).to(tl.uint32, bitcast=True)
        a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
        tl.store(out_ptr + offs * 4 + 0, a.to(tl.int32, bitcast=True))
        tl.store(out_ptr + offs * 4 + 1, b.to(tl.int32, bitcast=True))
        tl.store(out_ptr + offs * 4 + 2, c.to(tl.int32, bitcast=True))
        tl.store(out_ptr + offs * 4 + 3, d.to(tl.int32, bitcast=True))

    rng = np.random.default_rng(11)
    rows = []
    for seed in (1, 0x123456789ABCDEF, 2**63 - 25):
        ctr = rng.integers(0, 2**32, size=(64, 4), dtype=np.uint64).astype(np.uint32)
        ctr[0] = 0
        out = torch.zeros(64 * 4, dtype=torch.int32)
        k[(1,)](torch.from_numpy(ctr.view(np.int32).reshape(-1).copy()), out, seed, N=64)
        w = out.numpy().view(np.uint32).reshape(64, 4)
        for i in range(64):
            rows.append([seed] + [int(x) for x in ctr[i]] + [int(x) for x in w[i]])
    np.save(sys.argv[1], np.array(rows, dtype=object), allow_pickle=True)
""")


def test_matches_triton_library_statement(tmp_path):
    """Triton ships its own Philox4x32-10 (run here by its CPU interpreter)."""
    pytest.importorskip("triton")
    script = tmp_path / "tri.py"
    script.write_text(TRITON_SCRIPT)
    out = tmp_path / "rows.npy"
    env = dict(os.environ, TRITON_INTERPRET="1", CUDA_VISIBLE_DEVICES="")
    res = subprocess.run([sys.executable, str(script), str(out)], env=env, capture_output=True,
                         text=True, timeout=600)
    if res.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + res.stderr[-300:])
    rows = np.load(out, allow_pickle=True)
    for seed, c0, c1, c2, c3, *w in rows:
        mine = philox.philox4x32_10(c0, c1, c2, c3, seed & 0xFFFFFFFF, seed >> 32)
        assert [int(v) for v in mine] == [int(v) for v in w]


def test_uniforms_range_and_distribution():
    w = philox.noise_words(200000, seed=1, sample=0)
    u1, u2 = philox.uniforms(w)
    assert u1.min() > 0.0 and u1.max() <= 1.0
    assert u2.min() >= 0.0 and u2.max() < 1.0
    assert stats.kstest(u1, "uniform").pvalue > 1e-3
    assert stats.kstest(u2, "uniform").pvalue > 1e-3
    # every output byte uniform over 256 values
    bytes_ = w.astype(np.uint32).view(np.uint8).ravel()
    counts = np.bincount(bytes_, minlength=256)
    assert stats.chisquare(counts).pvalue > 1e-4


def test_normals_moments_and_independence():
    xi = philox.normals(400000, seed=3, sample=11)
    assert abs(xi.mean()) < 5 / np.sqrt(len(xi))
    assert abs(xi.var() - 1.0) < 5 * np.sqrt(2.0 / len(xi))
    assert stats.kstest(xi, "norm").pvalue > 1e-3
    # the two members of a Box-Muller pair are uncorrelated
    c = np.corrcoef(xi[0::2], xi[1::2])[0, 1]
    assert abs(c) < 5 / np.sqrt(len(xi) / 2)


def test_streams_differ_by_sample_and_seed():
    a = philox.normals(1000, 1, 0)
    b = philox.normals(1000, 1, 1)
    c = philox.normals(1000, 2, 0)
    d = philox.normals(1000, 1, 2 ** 32)  # high word of the sample index
    for other in (b, c, d):
        assert abs(np.corrcoef(a, other)[0, 1]) < 0.2
    assert np.array_equal(a, philox.normals(1000, 1, 0))


def test_odd_cell_count_is_prefix():
    a = philox.normals(1001, 5, 9)
    b = philox.normals(1002, 5, 9)
    assert np.array_equal(a, b[:1001])
