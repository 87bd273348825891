"""GPU force of the factorized multi-boson action on the active links (paper Sec. 4,
Eq. localMB): F[x, mu, t] = dS/d eps at U_mu(x) -> exp(i eps lambda_t/2) U_mu(x)
against the oracle (explicit adjoint block solves; pinned by finite differences
of the total action).  Block solves to 1e-12 (FP64) or 1e-11 (FP32 inner with
double-float defect correction): every entry within 1e-8 (FP64) / 1e-7 (FP32)
of the largest force, exactly zero off the active links."""

import numpy as np
import pytest
import torch

from paper_2211_06902_gb300 import dd4d, synth
from oracle.dd import Oracle, field_roots
from oracle.geometry import uniform_cores

from gpu_common import config1, make_case

pytestmark = pytest.mark.gpu

CASES = {
    "1D 8x4x4x2": lambda: make_case((8, 4, 4, 2), 0.13, 0.4, 6, [[(0, 1), (4, 5)], [], [], []]),
    "time undecomposed 4x8x2x2": lambda: make_case((4, 8, 2, 2), 0.13, 0.3, 5,
                                                   [[], [(0, 1), (4, 5)], [], []]),
    "8^4": config1,
}


def _fields(geo, ctx, n_f, seed):
    dpi = ctx.geom_sites(dd4d.SET_DPI)
    V = int(np.prod(geo.L))
    chis = [synth.complex_gaussian(seed, synth.TAG_CHI + k, geo.L + (4, 3)) * geo.dPi[..., None, None]
            for k in range(n_f)]
    return chis, np.stack([c.reshape(V, 12)[dpi] for c in chis])


def _active(o, geo):
    act = np.zeros(tuple(geo.L) + (4,), dtype=bool)
    for a in range(geo.nblocks):
        for x, mu in o.active_links(a):
            act[x + (mu,)] = True
    return act


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("inner", ["f64", "f32"])
def test_force_matches_oracle(name, inner):
    U, ctx, info, geo = CASES[name]()
    u = field_roots(4, 0.5)
    chis, vec = _fields(geo, ctx, len(u), 3)
    tol = 1e-12 if inner == "f64" else 1e-11
    F, st = ctx.mb_force(u, vec, prm=dd4d.params(tol, inner_prec=inner))
    assert st == 0
    o = Oracle(U, 0.13, geo)
    ref = o.mb_force(u, chis)
    act = _active(o, geo)
    assert act.any() and np.all(F[~act] == 0)
    scale = np.abs(ref).max()
    assert scale > 0
    assert np.abs(F - ref).max() <= (1e-8 if inner == "f64" else 1e-7) * scale


def test_device_output_matches_host_output():
    U, ctx, info, geo = CASES["1D 8x4x4x2"]()
    u = field_roots(2, 0.5)
    chis, vec = _fields(geo, ctx, len(u), 4)
    prm = dd4d.params(1e-12)
    Fh, _ = ctx.mb_force(u, vec, prm=prm)
    dF = torch.zeros(tuple(geo.L) + (4, 8), dtype=torch.float64, device="cuda")
    _, st = ctx.mb_force(u, torch.from_numpy(vec.view(np.float64)).cuda(), F=dF, prm=prm)
    assert st == 0
    assert np.array_equal(dF.cpu().numpy(), Fh)


@pytest.mark.parametrize("name", ["1D 8x4x4x2", "8^4"])
@pytest.mark.parametrize("inner", ["f64", "f32"])
def test_logdet_force_matches_oracle(name, inner):
    """Noise estimate of d ln|det D_Omega0^a| / d eps (Eq. SFeffN) with the same noise
    vectors on both sides (passed in): every entry within 1e-8 (FP64) / 1e-7 (FP32 inner)
    of the largest value, exactly zero off the active links; the oracle's estimator is
    pinned against the dense trace (test_oracle_dd)."""
    U, ctx, info, geo = CASES[name]()
    n = 4
    ids = list(range(info["nblocks"]))
    sites = [ctx.geom_sites(dd4d.SET_OMEGA, b) for b in ids]
    V = int(np.prod(geo.L))
    fields = [[synth.complex_gaussian(13, 700 + 50 * b + k, geo.L + (4, 3)) * geo.omega_mask[b][..., None, None]
               for k in range(n)] for b in ids]
    eta = np.stack([np.stack([f.reshape(V, 12)[sites[b]] for f in fields[b]]) for b in ids])
    tol = 1e-12 if inner == "f64" else 1e-11
    G, st = ctx.logdet_force(n, eta, prm=dd4d.params(tol, inner_prec=inner))
    assert st == 0
    o = Oracle(U, 0.13, geo)
    ref, _ = o.logdet_force_stochastic(fields)
    act = _active(o, geo)
    assert np.all(G[~act] == 0)
    scale = np.abs(ref).max()
    assert scale > 0
    assert np.abs(G - ref).max() <= (1e-8 if inner == "f64" else 1e-7) * scale
