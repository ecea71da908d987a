"""Host-side checks of the C ABI library (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    src = open(os.path.join(ROOT, "include", "spde.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(spde_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def built():
    from paper_1712_06758_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built)
    names = _header_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol(built):
    import paper_1712_06758_gb300 as pkg
    assert sorted(pkg.EXPORTED) == _header_functions()
    for name in _header_functions():
        assert callable(getattr(pkg, name))


def test_opts_defaults_and_argument_errors(built):
    import paper_1712_06758_gb300 as pkg
    o = pkg.spde_opts_init()
    assert o.precision == pkg.SPDE_PREC_MIXED and o.tol == 1e-10 and 0 < o.omega < 1
    # argument validation happens before any device work
    lib = pkg.lib()
    assert lib.spde_noise(-1, 1, 1, 0, 1.0, None, None) == pkg.SPDE_EINVAL
    assert lib.spde_apply(1, 0.1, 1.0, 1, 0, None, None, None) == pkg.SPDE_EINVAL
    assert lib.spde_apply(2, 0.1, 1.0, 1, 0, None, None, None) == pkg.SPDE_EINVAL
    assert lib.spde_precond(12, 0.1, 1.0, 1, 0, None, None, None, None) == pkg.SPDE_EINVAL
    assert lib.spde_sample(None, 0, 1, 1.0, 1.0, 1, 0, 0, None, None) == pkg.SPDE_EINVAL
    assert "context" in pkg.spde_last_error()
    assert lib.spde_opts_init(None) == pkg.SPDE_EINVAL
    assert lib.spde_destroy(None) == pkg.SPDE_OK


def test_no_cpu_fallback_when_library_missing(tmp_path, monkeypatch):
    import paper_1712_06758_gb300 as pkg
    monkeypatch.setattr(pkg, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(pkg, "_lib", None)
    with pytest.raises(ImportError):
        pkg.lib()


def test_layout_round_trip():
    from tests.layout import lib_to_oracle, oracle_to_lib, wall_mask
    n, h = 5, 0.2
    rng = np.random.default_rng(0)
    u = rng.standard_normal(3 * (n - 1) * n * n)
    th = rng.standard_normal(n ** 3)
    v = oracle_to_lib(u, th, n, h)
    assert np.all(v[wall_mask(n)] == 0)
    u2, th2 = lib_to_oracle(v, n, h)
    assert np.allclose(u, u2) and np.allclose(th, th2)
