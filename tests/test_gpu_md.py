"""GPU block-local molecular dynamics (dd_pf_heatbath, dd_md_trajectory) against the
oracle's leapfrog (oracle/md.py): the pseudofermion fields (1e-12), the links and
momenta after a trajectory, and H at both ends, on a 1D and a 2D decomposition
(frame corners); FP64 and FP32-inner solves; time reversibility on the GPU;
momenta off the active links returned as zero; refusals."""

import numpy as np
import pytest

from paper_2211_06902_gb300 import dd4d, synth
from oracle import md
from oracle.dd import Oracle, field_roots

from gpu_common import from_field, make_case, relerr, to_field

pytestmark = pytest.mark.gpu

KAPPA = 0.13
CASES = {
    "1D": ((4, 2, 2, 2), [[(0, 0), (2, 2)], [], [], []]),
    "2D": ((8, 8, 2, 2), [[(0, 1), (4, 5)], [(0, 1), (4, 5)], [], []]),
}


def _setup(name, seed=3):
    L, cores = CASES[name]
    U, ctx, info, geo = make_case(L, KAPPA, 0.4, seed, cores)
    o = Oracle(U, KAPPA, geo)
    V = int(np.prod(L))
    dpi = ctx.geom_sites(dd4d.SET_DPI)
    u = field_roots(4, 0.5)
    chis = [synth.complex_gaussian(4, synth.TAG_CHI + k, L + (4, 3)) * geo.dPi[..., None, None]
            for k in range(len(u))]
    chi = np.stack([c.reshape(V, 12)[dpi] for c in chis])
    sites = [ctx.geom_sites(dd4d.SET_OMEGA, b) for b in range(info["nblocks"])]
    etas = [synth.complex_gaussian(5, synth.TAG_RHS + a, L + (4, 3)) * geo.omega_mask[a][..., None, None]
            for a in range(info["nblocks"])]
    eta = np.stack([from_field(L, sites[a], etas[a])[None] for a in range(info["nblocks"])])
    P = synth.momenta(L, 6)
    return L, U, ctx, info, geo, o, u, chis, chi, sites, etas, eta, P


@pytest.mark.parametrize("name", list(CASES))
def test_pf_heatbath_matches_the_oracle(name):
    L, U, ctx, info, geo, o, u, chis, chi, sites, etas, eta, P = _setup(name)
    phi = np.zeros_like(eta)
    ctx.pf_heatbath(eta, phi)
    ref = md.pf_heatbath(o, etas)
    for a in range(info["nblocks"]):
        assert relerr(phi[a, 0], from_field(L, sites[a], ref[a])) < 1e-12


@pytest.mark.parametrize("prec,tol_u", [("f64", 1e-9), ("f32", 1e-8)])
@pytest.mark.parametrize("name", list(CASES))
def test_trajectory_matches_the_oracle(name, prec, tol_u):
    L, U, ctx, info, geo, o, u, chis, chi, sites, etas, eta, P = _setup(name)
    phi = np.zeros_like(eta)
    ctx.pf_heatbath(eta, phi)
    phis = [to_field(L, sites[a], phi[a, 0]) for a in range(info["nblocks"])]
    tau, n = 0.3, 3
    prm = dd4d.params(1e-12, inner_prec=prec)
    Pg = P.copy()
    st = ctx.md_trajectory(u, chi, phi, Pg, tau, n, prm)
    assert st["status"] == 0 and st["force_evals"] == n + 1 and st["steps"] == n
    act = md.active_mask(geo)
    h0 = md.hamiltonian(U, KAPPA, geo, u, chis, phis, P * act[..., None])
    U1, P1 = md.leapfrog(U, P, KAPPA, geo, u, chis, phis, tau, n)
    h1 = md.hamiltonian(U1, KAPPA, geo, u, chis, phis, P1)
    Ug = ctx.gauge_download()
    assert np.abs(Ug - U1).max() < tol_u
    assert np.array_equal(Ug[~act], U[~act])
    assert np.abs(Pg - P1).max() < 100 * tol_u * np.abs(P1).max()
    assert np.all(Pg[~act] == 0)
    for k, ref in (("kinetic0", h0["kinetic"]), ("s_mb0", h0["s_mb"]), ("s_pf0", h0["s_pf"]),
                   ("kinetic1", h1["kinetic"]), ("s_mb1", h1["s_mb"]), ("s_pf1", h1["s_pf"])):
        assert abs(st[k] - ref) <= 1e-9 * abs(ref), (k, st[k], ref)
    dH, dH_ref = st["H1"] - st["H0"], h1["H"] - h0["H"]
    assert abs(dH - dH_ref) < 1e-6 * max(1.0, abs(dH_ref)) + 1e-9 * h0["H"], (dH, dH_ref)


def test_trajectory_is_reversible_on_the_gpu():
    L, U, ctx, info, geo, o, u, chis, chi, sites, etas, eta, P = _setup("2D", seed=7)
    phi = np.zeros_like(eta)
    ctx.pf_heatbath(eta, phi)
    prm = dd4d.params(1e-12, inner_prec="f64")
    Pg = P * md.active_mask(geo)[..., None]
    P0 = Pg.copy()
    st1 = ctx.md_trajectory(u, chi, phi, Pg, 0.4, 4, prm)
    Pg *= -1
    st2 = ctx.md_trajectory(u, chi, phi, Pg, 0.4, 4, prm)
    assert np.abs(ctx.gauge_download() - U).max() < 1e-10
    assert np.abs(-Pg - P0).max() < 1e-9 * np.abs(P0).max()
    assert abs(st2["H1"] - st1["H0"]) < 1e-8 * st1["H0"]


def test_single_terms_and_refusals():
    L, U, ctx, info, geo, o, u, chis, chi, sites, etas, eta, P = _setup("1D")
    phi = np.zeros_like(eta)
    ctx.pf_heatbath(eta, phi)
    phis = [to_field(L, sites[a], phi[a, 0]) for a in range(info["nblocks"])]
    prm = dd4d.params(1e-12, inner_prec="f64")
    # pseudofermions only
    Pg = P.copy()
    st = ctx.md_trajectory(None, None, phi, Pg, 0.2, 2, prm)
    U1, P1 = md.leapfrog(U, P, KAPPA, geo, [], [], phis, 0.2, 2)
    assert st["s_mb0"] == 0.0 and abs(st["s_pf0"] - np.vdot(eta, eta).real) < 1e-10 * st["s_pf0"]
    assert np.abs(ctx.gauge_download() - U1).max() < 1e-9
    # multi-boson fields only, from the new links
    Pg2 = P.copy()
    st = ctx.md_trajectory(u, chi, None, Pg2, 0.2, 2, prm)
    U2, _ = md.leapfrog(U1, P, KAPPA, geo, u, chis, None, 0.2, 2)
    assert st["s_pf0"] == 0.0 and np.abs(ctx.gauge_download() - U2).max() < 1e-9
    with pytest.raises(dd4d.DDError):
        ctx.md_trajectory(None, None, None, P.copy(), 0.2, 2, prm)
    with pytest.raises(dd4d.DDError):
        ctx.md_trajectory(u, chi, phi, P.copy(), 0.2, 0, prm)
    ctx.set_clover(1.0)
    with pytest.raises(dd4d.DDError):
        ctx.md_trajectory(u, chi, phi, P.copy(), 0.2, 1, prm)
