"""GPU parity of w (Eqs. Wz, offdiagW1) and the multi-boson action (Eqs.
MBaction, localMB, globalMB) vs the oracle.

Solves run to 1e-10 (the solver tolerance); w must agree with the oracle to
1e-8 relative and the action S, each S^a and S^r to 1e-9 relative.
"""

import numpy as np
import pytest

from paper_2211_06902_gb300 import dd4d, synth
from oracle.dd import Oracle, field_roots
from oracle.geometry import uniform_cores

from gpu_common import config1, make_case, relerr

pytestmark = pytest.mark.gpu

CASES = {
    "8^4": lambda: config1(),
    "4^4": lambda: make_case((4,) * 4, 0.13, 0.3, 1, uniform_cores((4,) * 4, 1, 1)),
    "6x4^3": lambda: make_case((6, 4, 4, 4), 0.13, 0.3, 1,
                               [[(0, 1), (3, 4)]] + [[(0, 0), (2, 2)]] * 3),
    "uneven 12x8x8x10": lambda: make_case(
        (12, 8, 8, 10), 0.13, 0.5, 4,
        [[(0, 3), (6, 8)], [(1, 2), (5, 6)], [(0, 4), (6, 6)], [(0, 2), (4, 7)]]),
}


def _chis(geo, ctx, n_f, seed):
    dpi = ctx.geom_sites(dd4d.SET_DPI)
    assert np.array_equal(dpi, geo.sites(geo.dPi))
    V = int(np.prod(geo.L))
    chis = []
    for k in range(n_f):
        f = synth.complex_gaussian(seed, synth.TAG_CHI + 16 * k, geo.L + (4, 3))
        chis.append(f * geo.dPi[..., None, None])
    vec = np.stack([c.reshape(V, 12)[dpi] for c in chis])
    return chis, vec, dpi


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("inner", ["f64", "f32"])
def test_apply_w(name, inner):
    U, ctx, info, geo = CASES[name]()
    o = Oracle(U, ctx_kappa(name), geo)
    chis, vec, dpi = _chis(geo, ctx, 2, 1)
    out = np.zeros_like(vec)
    st = ctx.apply_w(2, vec, out, dd4d.params(1e-10, inner_prec=inner))
    assert st == 0
    V = int(np.prod(geo.L))
    for k in range(2):
        ref = o.apply_w(chis[k]).reshape(V, 12)[dpi]
        assert relerr(out[k], ref) < 1e-8


def ctx_kappa(name):
    return 0.13


@pytest.mark.parametrize("name", list(CASES))
def test_multiboson_action(name):
    U, ctx, info, geo = CASES[name]()
    o = Oracle(U, 0.13, geo)
    u = field_roots(4, 0.5)
    chis, vec, dpi = _chis(geo, ctx, 2, 3)
    S, Sb, Sr, st = ctx.multiboson_action(u, vec, dd4d.params(1e-10))
    assert st == 0
    S0, Sb0, Sr0 = o.multiboson_action(u, chis)
    assert abs(S - S0) <= 1e-9 * S0
    assert abs(Sr - Sr0) <= 1e-9 * S0
    assert np.max(np.abs(Sb - np.array(Sb0))) <= 1e-9 * S0
    assert abs(S - (Sb.sum() + Sr)) <= 1e-12 * S


def test_action_kappa_zero():
    L = (4,) * 4
    U, ctx, info, geo = make_case(L, 0.0, 0.3, 1, uniform_cores(L, 1, 1))
    u = field_roots(6, 0.3)
    chis, vec, dpi = _chis(geo, ctx, 3, 5)
    S, Sb, Sr, st = ctx.multiboson_action(u, vec, dd4d.params(1e-10))
    expect = sum(abs(uk) ** 2 * np.sum(np.abs(c) ** 2) for uk, c in zip(u, chis))
    assert abs(S - expect) <= 1e-12 * expect


def test_action_with_graph_and_autotune_matches_plain_call():
    U, ctx, info, geo = CASES["uneven 12x8x8x10"]()
    u = field_roots(6, 0.5)
    chis, vec, dpi = _chis(geo, ctx, 3, 11)
    a = ctx.multiboson_action(u, vec, dd4d.params(1e-10, inner_prec="f32"))
    b = ctx.multiboson_action(u, vec, dd4d.params(1e-10, inner_prec="f32", graph=True,
                                                   autotune=True))
    assert a[3] == b[3] == 0
    assert abs(a[0] - b[0]) <= 1e-10 * a[0] and np.allclose(a[1], b[1], rtol=1e-9)
    S0, Sb0, Sr0 = Oracle(U, 0.13, geo).multiboson_action(u, chis)
    assert abs(b[0] - S0) <= 1e-9 * S0


def test_action_deterministic():
    U, ctx, info, geo = config1()
    u = field_roots(4, 0.5)
    chis, vec, dpi = _chis(geo, ctx, 2, 9)
    a = ctx.multiboson_action(u, vec, dd4d.params(1e-10))
    b = ctx.multiboson_action(u, vec, dd4d.params(1e-10))
    assert a[0] == b[0] and a[2] == b[2] and np.array_equal(a[1], b[1])


def test_whole_solve_graph_in_w_and_action():
    """w and the action with every batched solve (uneven framed blocks, frame
    pieces and the frame Lambda1 in one batch) run as one graph launch each:
    bit-identical to the host-driven solves, and equal to the oracle."""
    U, ctx, info, geo = CASES["uneven 12x8x8x10"]()
    u = field_roots(6, 0.5)
    chis, vec, dpi = _chis(geo, ctx, 3, 12)
    w0, w1 = np.zeros_like(vec), np.zeros_like(vec)
    assert ctx.apply_w(3, vec, w0, dd4d.params(1e-10, inner_prec="f32")) == 0
    g = dd4d.params(1e-10, inner_prec="f32", graph_solve=True)
    for _ in range(2):                          # the second call replays the graphs
        assert ctx.apply_w(3, vec, w1, g) == 0
        assert np.array_equal(w0, w1)
    a = ctx.multiboson_action(u, vec, dd4d.params(1e-10, inner_prec="f32"))
    b = ctx.multiboson_action(u, vec, g)
    assert a[3] == b[3] == 0 and a[0] == b[0] and np.array_equal(a[1], b[1])
    S0, Sb0, Sr0 = Oracle(U, 0.13, geo).multiboson_action(u, chis)
    assert abs(b[0] - S0) <= 1e-9 * S0
