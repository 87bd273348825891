"""Pins of the oracle's parallel-transport convolution network.

The gradients are checked against central finite differences of the loss (in
the real and imaginary part of sampled weights), the adjoint layer against the
inner-product identity <y, T phi> = <T^+ y, phi>, and the layer against gauge
covariance (U, phi) -> (U^g, g phi) => y -> g y.
"""

import numpy as np

from paper_2211_06902_gb300 import synth
from oracle import net
from oracle.lattice import gauge_transform_links

SIDE = (3, 4, 3, 3)


def _setup(seed=1, channels=(4, 6, 4)):
    L = (6, 6, 4, 4)
    U = synth.gauge_field(L, 0.5, seed)
    Ub = net.box_links(U, (5, 1, 3, 0), SIDE)
    Ws = net.init_weights(seed, channels)
    Ws = [w + 0.1 * synth.complex_gaussian(seed, 90 + k, w.shape) for k, w in enumerate(Ws)]
    return U, Ub, Ws


def test_adjoint_identity():
    U, Ub, Ws = _setup()
    phi = synth.complex_gaussian(2, 7, (4,) + SIDE + (3,))
    g = synth.complex_gaussian(3, 7, (6,) + SIDE + (3,))
    lhs = np.vdot(g, net.layer(Ub, Ws[0], phi))
    rhs = np.vdot(net.layer_adjoint(Ub, Ws[0], g), phi)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_weight_gradient_finite_differences():
    U, Ub, Ws = _setup()
    n = int(np.prod(SIDE)) * 12
    pairs = [(synth.complex_gaussian(4, 8 + k, (n,)), synth.complex_gaussian(5, 8 + k, (n,)))
             for k in range(2)]
    L0, grads = net.loss_and_grads(Ub, Ws, pairs, SIDE)
    h = 1e-6
    rng = np.random.default_rng(0)
    for l in range(len(Ws)):
        for _ in range(3):
            idx = tuple(rng.integers(0, s) for s in Ws[l].shape)
            for part, unit in (("re", 1.0), ("im", 1j)):
                Wp = [w.copy() for w in Ws]
                Wm = [w.copy() for w in Ws]
                Wp[l][idx] += h * unit
                Wm[l][idx] -= h * unit
                fd = (net.loss_and_grads(Ub, Wp, pairs, SIDE)[0]
                      - net.loss_and_grads(Ub, Wm, pairs, SIDE)[0]) / (2 * h)
                an = grads[l][idx].real if part == "re" else grads[l][idx].imag
                assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (l, idx, part, fd, an)


def test_gauge_covariance():
    L = (6, 6, 4, 4)
    U = synth.gauge_field(L, 0.5, 3)
    gx = synth.gauge_transform(4, L)
    origin = (5, 1, 3, 0)
    Ws = net.init_weights(2, (4, 5, 4))
    phi = synth.complex_gaussian(6, 9, (4,) + SIDE + (3,))
    idx = np.indices(SIDE)
    gl = gx[tuple((origin[m] + idx[m]) % L[m] for m in range(4))]
    y = net.layer(net.box_links(U, origin, SIDE), Ws[0], phi)
    gphi = np.einsum("...ab,c...b->c...a", gl, phi)
    yg = net.layer(net.box_links(gauge_transform_links(U, gx), origin, SIDE), Ws[0], gphi)
    assert np.max(np.abs(yg - np.einsum("...ab,c...b->c...a", gl, y))) < 1e-13


def test_identity_network_is_identity():
    U, Ub, _ = _setup()
    Ws = [np.zeros((9, 4, 4), dtype=np.complex128) for _ in range(2)]
    for W in Ws:
        W[0] = np.eye(4)
    b = synth.complex_gaussian(7, 1, (int(np.prod(SIDE)) * 12,))
    y, _ = net.forward(Ub, Ws, b, SIDE)
    assert np.allclose(y, b)
