"""Failure detection without faulting the GPU: every failure is made on the
host (bad inputs, impossible sizes, a too-small iteration budget) and must
come back as a status code with the context still usable."""

import numpy as np
import pytest

from paper_2211_06902_gb300 import dd4d, synth

from gpu_common import make_case
from oracle.geometry import uniform_cores

pytestmark = pytest.mark.gpu


def test_nan_gauge_field_reports_enan_and_context_survives():
    L = (8,) * 4
    U, ctx, info, geo = make_case(L, 0.13, 0.3, 1, uniform_cores(L, 3, 1))
    n = len(ctx.geom_sites(dd4d.SET_OMEGA, 0))
    b = synth.complex_gaussian(1, synth.TAG_RHS, (2, 1, n, 12))
    bad = U.copy()
    bad[0, 0, 0, 0, 1, 0, 0] = np.nan
    ctx.gauge_upload(bad)
    x = np.zeros_like(b)
    with pytest.raises(dd4d.DDError) as e:
        ctx.solve_blocks("omega", [0, 1], 1, b, x, dd4d.params(1e-10, inner_prec="f32"))
    assert e.value.status == dd4d.DD_ENAN
    # the same context recovers with a valid field
    ctx.gauge_upload(U)
    st = ctx.solve_blocks("omega", [0, 1], 1, b, x, dd4d.params(1e-10, inner_prec="f32"))
    assert st["status"] == 0 and st["max_relres"] <= 1e-10


def test_out_of_memory_is_reported():
    with pytest.raises(dd4d.DDError) as e:
        dd4d.Context((256, 256, 128, 128), 0.13)      # 2^30 sites: 618 GB of links
    assert e.value.status == dd4d.DD_ENOMEM


def test_invalid_geometry_and_sizes():
    L = (8,) * 4
    ctx = dd4d.Context(L, 0.13)
    with pytest.raises(dd4d.DDError):
        ctx.set_geometry([[(0, 6)]] + [[(0, 2), (4, 6)]] * 3)      # one core in x0
    with pytest.raises(dd4d.DDError):
        ctx.set_geometry([[(0, 2), (3, 6)]] + [[(0, 2), (4, 6)]] * 3)   # no frame
    with pytest.raises(dd4d.DDError):
        dd4d.Context((7, 8, 8, 8), 0.13)                              # odd extent
    ctx.gauge_upload(synth.gauge_field(L, 0.3, 1))
    info = ctx.set_geometry(uniform_cores(L, 3, 1))
    with pytest.raises(dd4d.DDError):
        ctx.solve_blocks("omega", [0], 70000, np.zeros(24), np.zeros(24), dd4d.params())


def test_bounded_wait_gives_up_and_context_survives():
    """The bundle stencil's bounded mbarrier wait, made to give up through the test
    hook dd_debug_wait_fault (one CTA arms a barrier without issuing its copy, so
    nothing is in flight, and waits about 64 us), comes back as DD_ETIMEOUT; with
    the hook off, the same context computes the stencil (checked against the
    oracle) and solves to 1e-10."""
    from oracle.lattice import apply_D_restricted
    from gpu_common import from_field, relerr, to_field
    L = (8,) * 4
    U, ctx, info, geo = make_case(L, 0.13, 0.3, 1, uniform_cores(L, 3, 1))
    v = next(k for k in range(64) if (dd4d.hop_variant_name("f32", k) or "").startswith("k_hop_lb"))
    ctx.set_hop_variant("f32", v)
    ids = list(range(info["nblocks"]))
    sites = [ctx.geom_sites(dd4d.SET_OMEGA, b) for b in ids]
    psi = synth.complex_gaussian(3, synth.TAG_RHS, (len(ids), 2, len(sites[0]), 12))
    out = np.zeros_like(psi)
    ctx.debug_wait_fault(True)
    with pytest.raises(dd4d.DDError) as e:
        ctx.apply_D_block("omega", ids, 2, psi, out, "f32")       # host buffers: synchronising
    assert e.value.status == dd4d.DD_ETIMEOUT
    ctx.debug_wait_fault(False)
    out[:] = 0
    ctx.apply_D_block("omega", ids, 2, psi, out, "f32")
    for b in ids:
        for r in range(2):
            f = to_field(L, sites[b], psi[b, r])
            want = from_field(L, sites[b], apply_D_restricted(U, f, 0.13, geo.omega_mask[b]))
            assert relerr(out[b, r], want) < 2e-6
    x = np.zeros_like(psi)
    st = ctx.solve_blocks("omega", ids, 2, psi, x, dd4d.params(1e-10, inner_prec="f32"))
    assert st["status"] == 0 and st["max_relres"] <= 1e-10
