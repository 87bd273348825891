"""The C-ABI library loads and exports every entry point include/dd4d.h declares.

CPU only: no compute call is made (there may be no GPU here).
"""

import os
import re

import pytest

from paper_2211_06902_gb300 import dd4d

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "dd4d.h")).read()
    return sorted(set(re.findall(r"\b(dd_[a-z_0-9A-Z]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(dd4d.LIB_PATH):
        from paper_2211_06902_gb300 import build
        build.build()
    return dd4d.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "dd_solve_blocks" in names and "dd_multiboson_action" in names
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(dd4d.exported_symbols()) == names


def test_strerror_and_roots_without_gpu(lib):
    assert lib.dd_strerror(0) == b"ok"
    assert lib.dd_strerror(3) == b"solver did not converge"
    import numpy as np
    from oracle.dd import field_roots
    for N, c in [(8, 0.5), (4, 0.5), (24, 0.3), (6, 0.0)]:
        # the library's roots equal the oracle's (pinned by the Chebyshev identity)
        assert np.allclose(dd4d.roots(N, c), field_roots(N, c), rtol=0, atol=1e-15)
    with pytest.raises(dd4d.DDError):
        dd4d.roots(5, 0.5)


def test_hop_variant_names_distinct():
    """Every compiled stencil launch form has its own description, per precision."""
    for prec in ("f64", "f32", "bf16"):
        n = dd4d.lib().dd_hop_variants(dd4d.PREC[prec])
        names = [dd4d.hop_variant_name(prec, v) for v in range(n)]
        assert all(names), (prec, names)
        assert len(set(names)) == n, (prec, names)
        assert dd4d.hop_variant_name(prec, n) is None and dd4d.hop_variant_name(prec, -1) is None
