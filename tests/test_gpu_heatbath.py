"""GPU heat-bath of the multi-boson fields (paper Sec. 4, the fields of Eq. WW):
chi_k = W_{u_k}^{-1} eta_k.  Parity with the oracle's dense solve on 4^4, and
on config 1 the exact identity S_MB(chi) = sum_k |eta_k|^2 evaluated by the
library's own action (block and frame solves to 1e-10, heat-bath to 1e-10)."""

import numpy as np
import pytest

from paper_2211_06902_gb300 import dd4d, synth
from oracle.dd import Oracle, field_roots
from oracle.geometry import uniform_cores

from gpu_common import config1, make_case, relerr

pytestmark = pytest.mark.gpu


def _etas(geo, ctx, n_f, seed):
    dpi = ctx.geom_sites(dd4d.SET_DPI)
    V = int(np.prod(geo.L))
    fields = [synth.complex_gaussian(seed, 40 + k, geo.L + (4, 3)) * geo.dPi[..., None, None]
              for k in range(n_f)]
    return fields, np.stack([f.reshape(V, 12)[dpi] for f in fields]), dpi


def test_heatbath_matches_oracle_4x4():
    L = (4,) * 4
    U, ctx, info, geo = make_case(L, 0.13, 0.3, 1, uniform_cores(L, 1, 1))
    u = field_roots(4, 0.5)
    fields, eta, dpi = _etas(geo, ctx, len(u), 3)
    chi = np.zeros_like(eta)
    st = ctx.multiboson_heatbath(u, eta, chi, tol=1e-11, prm=dd4d.params(1e-12))
    assert st["status"] == 0 and st["converged"] == len(u), st
    ref = Oracle(U, 0.13, geo).heatbath(u, fields)
    V = int(np.prod(L))
    for k in range(len(u)):
        assert relerr(chi[k], ref[k].reshape(V, 12)[dpi]) < 1e-9


@pytest.mark.parametrize("inner", ["f64", "f32"])
def test_heatbath_action_identity_config1(inner):
    """S_MB at the generated fields is sum |eta|^2 (|W_u chi - eta| <= 1e-10 |eta|)."""
    U, ctx, info, geo = config1()
    u = field_roots(8, 0.5)                      # 4 fields
    _, eta, _ = _etas(geo, ctx, len(u), 5)
    chi = np.zeros_like(eta)
    prm = dd4d.params(1e-11, inner_prec=inner)
    st = ctx.multiboson_heatbath(u, eta, chi, tol=1e-10, prm=prm)
    assert st["status"] == 0 and st["max_relres"] <= 1e-10, st
    S = ctx.multiboson_action(u, chi, prm)[0]
    ref = float(np.vdot(eta, eta).real)
    # |W chi|^2 = |eta + e|^2 with |e| <= ~1e-10 |eta| (recursive residual plus
    # the inexact w of the 1e-11 inner solves)
    assert abs(S - ref) <= 5e-10 * ref


def test_heatbath_rejects_a_zero_root():
    U, ctx, info, geo = config1()
    _, eta, _ = _etas(geo, ctx, 1, 1)
    with pytest.raises(dd4d.DDError):
        ctx.multiboson_heatbath(np.array([0.0 + 0.0j]), eta, np.zeros_like(eta))
