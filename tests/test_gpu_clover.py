"""GPU clover term (the site-local term the paper admits in D, Sec. 1) against the
oracle: D_X = A - kappa H restricted (FP64 stencil, 1e-12), block and frame
solves (left-preconditioned by A^{-1}, FP64 and the mixed forms with FP32 or
BF16-storage inner solves and a double-float residual, at tol 1e-10: the true
residual with the oracle's own operator |b - D_X x| <= 1e-10 |b| and the
oracle's solution to 1e-8), w and the
multi-boson action (1e-8 / 1e-9, FP64 and FP32 inner), the dense check of
Eq. (detD) with the clover term, the rebuild of A on a new gauge field and
kappa, and the calls that refuse the term."""

import numpy as np
import pytest

from paper_2211_06902_gb300 import dd4d, synth
from oracle.dd import Oracle, field_roots
from oracle.geometry import uniform_cores
from oracle.lattice import apply_D, apply_D_restricted

from gpu_common import from_field, make_case, relerr, to_field

pytestmark = pytest.mark.gpu

CSW = 1.2
CASES = {
    "8^4": lambda: make_case((8,) * 4, 0.13, 0.4, 2, uniform_cores((8,) * 4, 3, 1)),
    "1D 8x4x4x2": lambda: make_case((8, 4, 4, 2), 0.13, 0.4, 6, [[(0, 1), (4, 5)], [], [], []]),
}


def _clover_case(name):
    U, ctx, info, geo = CASES[name]()
    ctx.set_clover(CSW)
    return U, ctx, info, geo


@pytest.mark.parametrize("name", list(CASES))
def test_stencil(name):
    U, ctx, info, geo = _clover_case(name)
    L = geo.L
    V = int(np.prod(L))
    psi = synth.complex_gaussian(1, synth.TAG_RHS, (2, V, 12))
    out = np.zeros_like(psi)
    ctx.apply_D_block("full", None, 2, psi, out, "f64")
    for r in range(2):
        ref = apply_D(U, psi[r].reshape(L + (4, 3)), 0.13, csw=CSW).reshape(V, 12)
        assert relerr(out[r], ref) < 1e-12
    ids = list(range(info["nblocks"]))
    for kind, set_id, masks in [("omega", dd4d.SET_OMEGA, geo.omega_mask), ("phi", dd4d.SET_PHI, geo.phi_mask)]:
        sites = [ctx.geom_sites(set_id, b) for b in ids]
        n = len(sites[0])
        psi = synth.complex_gaussian(2, synth.TAG_RHS, (len(ids), 2, n, 12))
        out = np.zeros_like(psi)
        ctx.apply_D_block(kind, ids, 2, psi, out, "f64")
        for b in ids[:4]:
            for r in range(2):
                f = to_field(L, sites[b], psi[b, r])
                ref = from_field(L, sites[b], apply_D_restricted(U, f, 0.13, masks[b], csw=CSW))
                assert relerr(out[b, r], ref) < 1e-12


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("name", list(CASES))
def test_block_and_frame_solves(name, prec):
    U, ctx, info, geo = _clover_case(name)
    o = Oracle(U, 0.13, geo, csw=CSW)
    L = geo.L
    ids = list(range(info["nblocks"]))
    sites = [ctx.geom_sites(dd4d.SET_OMEGA, b) for b in ids]
    b = synth.complex_gaussian(3, synth.TAG_RHS, (len(ids), 2, len(sites[0]), 12))
    x = np.zeros_like(b)
    prm = dd4d.params(1e-10, inner_prec=prec, inner_tol=1e-3 if prec == "bf16" else 3e-6,
                      autotune=prec != "f64")
    st = ctx.solve_blocks("omega", ids, 2, b, x, prm)
    assert st["status"] == dd4d.DD_OK, st
    for k in ids[:4]:
        for r in range(2):
            f = to_field(L, sites[k], b[k, r])
            xf = to_field(L, sites[k], x[k, r])
            res = f - apply_D_restricted(U, xf, 0.13, geo.omega_mask[k], csw=CSW)
            # the true residual, although the solver tests the preconditioned one
            assert np.linalg.norm(res) <= 1e-10 * np.linalg.norm(f)
            assert relerr(x[k, r], from_field(L, sites[k], o.omega_solver(k).solve_field(f))) < 1e-8
    fs = ctx.geom_sites(dd4d.SET_LAMBDA1)
    bf = synth.complex_gaussian(4, synth.TAG_RHS, (1, 1, len(fs), 12))
    xf = np.zeros_like(bf)
    assert ctx.solve_blocks("lambda1", None, 1, bf, xf, prm)["status"] == 0
    f = to_field(L, fs, bf[0, 0])
    assert relerr(xf[0, 0], from_field(L, fs, o.frame_solver().solve_field(f))) < 1e-8


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("name", list(CASES))
def test_w_and_action(name, prec):
    U, ctx, info, geo = _clover_case(name)
    o = Oracle(U, 0.13, geo, csw=CSW)
    dpi = ctx.geom_sites(dd4d.SET_DPI)
    V = int(np.prod(geo.L))
    chis = [synth.complex_gaussian(5, synth.TAG_CHI + k, geo.L + (4, 3)) * geo.dPi[..., None, None]
            for k in range(2)]
    vec = np.stack([c.reshape(V, 12)[dpi] for c in chis])
    out = np.zeros_like(vec)
    prm = dd4d.params(1e-11, inner_prec=prec)
    assert ctx.apply_w(2, vec, out, prm) == 0
    for k in range(2):
        assert relerr(out[k], o.apply_w(chis[k]).reshape(V, 12)[dpi]) < 1e-8
    u = field_roots(4, 0.5)
    S, Sb, Sr, st = ctx.multiboson_action(u, vec, prm)
    S0, Sb0, Sr0 = o.multiboson_action(u, chis)
    assert st == 0 and abs(S - S0) <= 1e-9 * S0 and abs(Sr - Sr0) <= 1e-9 * S0


def test_logdet_identity_with_clover():
    L = (4,) * 4
    U, ctx, info, geo = make_case(L, 0.13, 0.4, 5, uniform_cores(L, 1, 1))
    ctx.set_clover(1.0)
    rep = ctx.logdet_check(dd4d.params(1e-13, maxiter=5000))
    assert abs(rep["residual"]) < 1e-9, rep
    f = Oracle(U, 0.13, geo, csw=1.0).logdet_factors()
    assert abs(rep["logabs_D"] - f["D"][1]) < 1e-9
    assert abs(rep["logabs_W1"] - f["W1"][1]) < 1e-8


def test_rebuild_on_new_links_and_kappa_and_switch_off():
    L = (8, 4, 4, 2)
    U, ctx, info, geo = CASES["1D 8x4x4x2"]()
    V = int(np.prod(L))
    psi = synth.complex_gaussian(7, synth.TAG_RHS, (1, V, 12))
    out = np.zeros_like(psi)
    ctx.apply_D_block("full", None, 1, psi, out, "f64")
    wilson = out.copy()
    ctx.set_clover(CSW)
    U2 = synth.gauge_field(L, 0.5, 9)
    ctx.gauge_upload(U2)
    ctx.set_kappa(0.12)
    ctx.apply_D_block("full", None, 1, psi, out, "f64")
    ref = apply_D(U2, psi[0].reshape(L + (4, 3)), 0.12, csw=CSW).reshape(V, 12)
    assert relerr(out[0], ref) < 1e-12
    ctx.set_clover(0.0)
    ctx.gauge_upload(U)
    ctx.set_kappa(0.13)
    ctx.apply_D_block("full", None, 1, psi, out, "f64")
    assert np.array_equal(out, wilson)


def test_refusals():
    U, ctx, info, geo = _clover_case("1D 8x4x4x2")
    V = int(np.prod(geo.L))
    psi = synth.complex_gaussian(8, synth.TAG_RHS, (1, V, 12))
    out = np.zeros_like(psi)
    with pytest.raises(dd4d.DDError):
        ctx.apply_D_block("full", None, 1, psi, out, "f32")
    ids = list(range(info["nblocks"]))
    n = len(ctx.geom_sites(dd4d.SET_OMEGA, 0))
    b = synth.complex_gaussian(8, synth.TAG_RHS, (len(ids), 1, n, 12))
    with pytest.raises(dd4d.DDError):
        ctx.solve_blocks("omega", ids, 1, b, np.zeros_like(b), dd4d.params(1e-10, inner_prec="f32",
                                                                            net_guess=True))
    dpi = ctx.geom_sites(dd4d.SET_DPI)
    chi = synth.complex_gaussian(8, synth.TAG_CHI, (1, len(dpi), 12))
    with pytest.raises(dd4d.DDError):
        ctx.mb_force([0.5 + 0.5j], chi)


def test_condition_bound():
    """c_A bounds cond_2(A) from above (checked against the oracle's A, site by site),
    is 1 without the term, and follows A when kappa changes."""
    from oracle.lattice import clover_term
    U, ctx, info, geo = _clover_case("1D 8x4x4x2")
    cA = ctx.clover_cond()
    A = clover_term(U, 0.13, CSW).reshape(-1, 12, 12)
    s = np.linalg.svd(A, compute_uv=False)
    assert cA >= s[:, 0].max() / s[:, -1].min() * (1 - 1e-12) and cA < 10
    ctx.set_kappa(0.12)
    assert ctx.clover_cond() != cA
    ctx.set_clover(0.0)
    assert ctx.clover_cond() == 1.0


def test_mixed_matches_f64_and_rebuilds_tables():
    """The mixed solve with the clover term agrees with the FP64 one (both to
    1e-11, so within 1e-8), also after A changes with a new kappa (the packed
    tables follow the FP64 one)."""
    U, ctx, info, geo = _clover_case("8^4")
    ids = list(range(info["nblocks"]))
    n = len(ctx.geom_sites(dd4d.SET_OMEGA, 0))
    b = synth.complex_gaussian(9, synth.TAG_RHS, (len(ids), 3, n, 12))
    for kappa in (0.13, 0.125):
        ctx.set_kappa(kappa)
        x64 = np.zeros_like(b)
        x32 = np.zeros_like(b)
        assert ctx.solve_blocks("omega", ids, 3, b, x64, dd4d.params(1e-11, inner_prec="f64"))["status"] == 0
        st = ctx.solve_blocks("omega", ids, 3, b, x32, dd4d.params(1e-11, inner_prec="f32"))
        assert st["status"] == 0 and st["max_relres"] <= 1e-11
        assert relerr(x32, x64) < 1e-8
