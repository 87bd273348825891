"""The library's decomposition of the benchmark lattices (paper Sec. 2) reports
the stored set sizes of the closed form (32^4, uneven 64x32^3, 48^4)."""

import pytest

from paper_2211_06902_gb300 import dd4d

from test_oracle_geometry import BENCH_GEOMETRIES

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", list(BENCH_GEOMETRIES))
def test_benchmark_geometry_counts(name):
    L, cores, ref, omegas = BENCH_GEOMETRIES[name]
    ctx = dd4d.Context(L, 0.13)
    info = ctx.set_geometry(cores)
    got = (info["nblocks"], info["n_lambda1"], info["n_dpi"], info["n_B"], info["n_C"], info["n_E"],
           info["n_A"])
    assert got == ref
    assert info["max_omega"] == max(omegas or {10000})
    ctx.close()
