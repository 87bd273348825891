"""GPU samples of the reweighting factor W_N = det{1 - R_{N+1}(W_1)} (paper Sec. 4,
Eq. rw): per source s = |eta|^2 - |M eta|^2 and R_{N+1}(W_1) eta against the
oracle, which forms M in the paper's product form c_N W_1 prod_k (W_1 - z_k)
while the library runs the Chebyshev recurrence in w.  Inner solves to 1e-12
(FP64) or 1e-11 (FP32 inner, double-float defect correction); R eta must agree
to 1e-8 relative and s to 1e-8 |eta|^2."""

import numpy as np
import pytest
import torch

from paper_2211_06902_gb300 import dd4d, synth
from oracle.dd import Oracle
from oracle.geometry import uniform_cores

from gpu_common import config1, make_case, relerr

pytestmark = pytest.mark.gpu

CASES = {
    "1D 8x4x4x2": lambda: make_case((8, 4, 4, 2), 0.13, 0.4, 6, [[(0, 1), (4, 5)], [], [], []]),
    "4^4": lambda: make_case((4,) * 4, 0.13, 0.3, 1, uniform_cores((4,) * 4, 1, 1)),
}


def _sources(geo, ctx, n, seed):
    dpi = ctx.geom_sites(dd4d.SET_DPI)
    V = int(np.prod(geo.L))
    fields = [synth.complex_gaussian(seed, synth.TAG_CHI + k, geo.L + (4, 3)) * geo.dPi[..., None, None]
              for k in range(n)]
    return fields, np.stack([f.reshape(V, 12)[dpi] for f in fields]), dpi


def _check(U, kappa, geo, fields, dpi, N, c, s, r_eta):
    o = Oracle(U, kappa, geo)
    V = int(np.prod(geo.L))
    s_ref = o.reweight_samples(N, c, fields)
    for k, f in enumerate(fields):
        e = f.reshape(V, 12)[dpi]
        r_ref = e - o.reweight_apply(N, c, f).reshape(V, 12)[dpi]
        assert relerr(r_eta[k], r_ref) < 1e-8
        assert abs(s[k] - s_ref[k]) <= 1e-8 * np.sum(np.abs(e) ** 2)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("N,c", [(4, 0.5), (6, 0.0)])
@pytest.mark.parametrize("inner", ["f64", "f32"])
def test_samples_match_oracle(name, N, c, inner):
    U, ctx, info, geo = CASES[name]()
    fields, eta, dpi = _sources(geo, ctx, 2, 5)
    r_eta = np.zeros_like(eta)
    tol = 1e-12 if inner == "f64" else 1e-11
    s, st = ctx.reweight_samples(N, c, eta, r_eta, dd4d.params(tol, inner_prec=inner))
    assert st == 0
    _check(U, 0.13, geo, fields, dpi, N, c, s, r_eta)


def test_config1_sample():
    U, ctx, info, geo = config1()
    fields, eta, dpi = _sources(geo, ctx, 1, 8)
    r_eta = np.zeros_like(eta)
    s, st = ctx.reweight_samples(2, 0.5, eta, r_eta, dd4d.params(1e-12))
    assert st == 0
    _check(U, 0.13, geo, fields, dpi, 2, 0.5, s, r_eta)


def test_device_buffers_match_host_buffers():
    U, ctx, info, geo = CASES["4^4"]()
    fields, eta, dpi = _sources(geo, ctx, 3, 9)
    prm = dd4d.params(1e-12)
    s_h, _ = ctx.reweight_samples(4, 0.5, eta, None, prm)
    de = torch.from_numpy(eta).cuda()
    dr = torch.zeros_like(de)
    s_d, st = ctx.reweight_samples(4, 0.5, de, dr, prm)
    assert st == 0
    assert np.array_equal(s_h, s_d)
    r_h = np.zeros_like(eta)
    ctx.reweight_samples(4, 0.5, eta, r_h, prm)
    assert np.array_equal(dr.cpu().numpy(), r_h)


def test_invalid_arguments():
    U, ctx, info, geo = CASES["4^4"]()
    fields, eta, dpi = _sources(geo, ctx, 1, 1)
    for N, c in [(3, 0.5), (0, 0.5), (4, 1.0), (4, -0.1)]:
        with pytest.raises(dd4d.DDError):
            ctx.reweight_samples(N, c, eta)
