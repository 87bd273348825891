"""GPU path on the one-dimensional decomposition in thick time slices (paper
Sec. 3, Fig. 1dDD; only x0 decomposed, domains wrap around in space): site
sets, restricted stencils, w, block and frame solves against the oracle, and
the dense check of the 1D determinant formula
det D = det W_1 prod_a det D_Omega^a / det D_Lambda1."""

import numpy as np
import pytest

from paper_2211_06902_gb300 import dd4d, synth
from oracle.dd import Oracle
from oracle.lattice import apply_D_restricted

from gpu_common import from_field, make_case, relerr, to_field

pytestmark = pytest.mark.gpu

L = (8, 4, 4, 2)
CORES = [[(0, 1), (4, 5)], [], [], []]


@pytest.fixture(scope="module")
def case():
    return make_case(L, 0.13, 0.4, 6, CORES)


def test_sets_and_counts(case):
    U, ctx, info, geo = case
    assert info["nblocks"] == 2 and info["n_C"] == 0
    assert np.array_equal(ctx.geom_sites(dd4d.SET_DPI), geo.sites(geo.dPi))
    assert np.array_equal(ctx.geom_sites(dd4d.SET_LAMBDA1), geo.sites(geo.Lambda1))
    for b in range(2):
        assert np.array_equal(np.sort(ctx.geom_sites(dd4d.SET_OMEGA, b)), geo.sites(geo.omega_mask[b]))
        assert np.array_equal(np.sort(ctx.geom_sites(dd4d.SET_PHI, b)), geo.sites(geo.phi_mask[b]))


@pytest.mark.parametrize("kind,set_id,masks", [("omega", dd4d.SET_OMEGA, "omega_mask"),
                                               ("phi", dd4d.SET_PHI, "phi_mask")])
def test_wrapping_block_stencils(case, kind, set_id, masks):
    U, ctx, info, geo = case
    sites = [ctx.geom_sites(set_id, b) for b in range(2)]
    psi = synth.complex_gaussian(3, synth.TAG_RHS, (2, 2, len(sites[0]), 12))
    out = np.zeros_like(psi)
    ctx.apply_D_block(kind, [0, 1], 2, psi, out, "f64")
    for b in range(2):
        for r in range(2):
            f = to_field(L, sites[b], psi[b, r])
            ref = from_field(L, sites[b], apply_D_restricted(U, f, 0.13, getattr(geo, masks)[b]))
            assert relerr(out[b, r], ref) < 1e-12


@pytest.mark.parametrize("inner", ["f64", "f32"])
def test_w_and_solves(case, inner):
    U, ctx, info, geo = case
    o = Oracle(U, 0.13, geo)
    dpi = ctx.geom_sites(dd4d.SET_DPI)
    V = int(np.prod(L))
    chis = [synth.complex_gaussian(4, synth.TAG_CHI + k, L + (4, 3)) * geo.dPi[..., None, None]
            for k in range(2)]
    vec = np.stack([c.reshape(V, 12)[dpi] for c in chis])
    out = np.zeros_like(vec)
    assert ctx.apply_w(2, vec, out, dd4d.params(1e-11, inner_prec=inner)) == 0
    for k in range(2):
        assert relerr(out[k], o.apply_w(chis[k]).reshape(V, 12)[dpi]) < 1e-8


def test_one_dimensional_det_formula(case):
    U, ctx, info, geo = case
    rep = ctx.logdet_check(dd4d.params(1e-13, maxiter=5000))
    assert abs(rep["residual"]) < 1e-9, rep
    f = Oracle(U, 0.13, geo).logdet_factors()
    assert abs(rep["logabs_D"] - f["D"][1]) < 1e-9
    assert abs(rep["logabs_W1"] - f["W1"][1]) < 1e-8
    one_d = rep["logabs_W1"] + float(np.sum(rep["logabs_omega"])) - rep["logabs_Lambda1"]
    assert abs(rep["logabs_D"] - one_d) < 1e-8
    assert abs(float(np.sum(rep["logabs_phi"])) - 2 * rep["logabs_Lambda1"]) < 1e-9


def test_two_dimensional_decomposition_identity():
    """Time and x1 decomposed (corners: dPi1 not empty), x2 and x3 wrapping:
    the dense check of Eq. (detD) against the oracle."""
    L2 = (8, 8, 2, 2)
    cores = [[(0, 1), (4, 5)], [(0, 1), (4, 5)], [], []]
    U, ctx, info, geo = make_case(L2, 0.13, 0.4, 7, cores)
    assert info["nblocks"] == 4 and info["n_C"] > 0
    rep = ctx.logdet_check(dd4d.params(1e-13, maxiter=5000))
    assert abs(rep["residual"]) < 1e-9, rep
    f = Oracle(U, 0.13, geo).logdet_factors()
    assert abs(rep["logabs_D"] - f["D"][1]) < 1e-9
    assert abs(rep["logabs_W1"] - f["W1"][1]) < 1e-8
