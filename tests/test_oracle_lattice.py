"""Pins of the oracle's Wilson-Dirac operator (Sec. 1 and 3 of the paper).

Every check compares the oracle with something other than itself: the
Clifford algebra, the free-field momentum-space form of D, its closed-form
log det, gamma_5-hermiticity, gauge covariance, and brute-force comparison of
the two independent formulations (array shifts vs assembled sparse matrix).
"""

import numpy as np
import pytest

from paper_2211_06902_gb300 import synth
from oracle.lattice import (apply_D, apply_D_restricted, dirac_block, dirac_matrix,
                            gammas, gauge_transform_links)


def test_clifford_and_gamma5():
    g, g5 = gammas()
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T)
        for nu in range(4):
            anti = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(anti, 2.0 * (mu == nu) * np.eye(4), atol=1e-15)
    assert np.allclose(g5, np.diag([1, 1, -1, -1]))


def _momenta(L, n, time_bc=-1):
    """Allowed lattice momenta: antiperiodic in time shifts p0 by pi/L0."""
    shift = 0.5 if time_bc == -1 else 0.0
    return [2 * np.pi * (n[0] + shift) / L[0]] + [2 * np.pi * n[mu] / L[mu] for mu in (1, 2, 3)]


@pytest.mark.parametrize("n", [(0, 0, 0, 0), (1, 2, 0, 1), (3, 1, 1, 0)])
def test_free_field_plane_wave(n):
    """D e^{ipx} v = e^{ipx} [1 - 2k sum cos p + 2ik sum gamma_mu sin p_mu] v (U = 1)."""
    L = (6, 4, 4, 2)
    kappa = 0.13
    g, _ = gammas()
    p = _momenta(L, n)
    x = np.indices(L)
    phase = np.exp(1j * sum(p[mu] * x[mu] for mu in range(4)))
    v = synth.complex_gaussian(7, 9, (4, 3))
    psi = phase[..., None, None] * v
    out = apply_D(synth.unit_gauge(L), psi, kappa)
    M = (1 - 2 * kappa * sum(np.cos(p))) * np.eye(4) + 2j * kappa * sum(
        g[mu] * np.sin(p[mu]) for mu in range(4))
    expect = phase[..., None, None] * (M @ v)
    assert np.max(np.abs(out - expect)) < 1e-13


@pytest.mark.parametrize("L,time_bc", [((4, 4, 4, 4), -1), ((4, 2, 2, 2), 1)])
def test_free_field_logdet_closed_form(L, time_bc):
    """ln det D_free = 6 sum_p ln[(1 - 2k sum cos p)^2 + 4k^2 sum sin^2 p]."""
    kappa = 0.13
    V = int(np.prod(L))
    D = dirac_matrix(synth.unit_gauge(L), kappa, np.arange(V), time_bc).toarray()
    sign, logabs = np.linalg.slogdet(D)
    total = 0.0
    for n in np.ndindex(*L):
        p = np.array(_momenta(L, n, time_bc))
        a = 1 - 2 * kappa * np.cos(p).sum()
        total += 6 * np.log(a * a + 4 * kappa ** 2 * (np.sin(p) ** 2).sum())
    assert abs(logabs - total) < 1e-10
    assert abs(sign - 1) < 1e-12


def test_gamma5_hermiticity():
    """gamma_5 D gamma_5 = D^+ for a random gauge field (and any restriction)."""
    L = (4, 4, 4, 4)
    U = synth.gauge_field(L, 0.5, 11)
    V = int(np.prod(L))
    _, g5 = gammas()
    G5 = np.kron(g5, np.eye(3))
    for sites in (np.arange(V), np.arange(0, V, 3)):
        D = dirac_matrix(U, 0.13, sites).toarray()
        n = len(sites)
        G = np.kron(np.eye(n), G5)
        assert np.max(np.abs(G @ D @ G - D.conj().T)) < 1e-14


def test_gauge_covariance():
    """D[U^g] (g psi) = g (D[U] psi) with U^g_mu(x) = g(x) U_mu(x) g(x+mu)^+."""
    L = (4, 4, 2, 6)
    U = synth.gauge_field(L, 0.6, 3)
    gx = synth.gauge_transform(5, L)
    psi = synth.complex_gaussian(3, 2, L + (4, 3))
    gpsi = np.einsum("...ab,...sb->...sa", gx, psi)
    lhs = apply_D(gauge_transform_links(U, gx), gpsi, 0.12)
    rhs = np.einsum("...ab,...sb->...sa", gx, apply_D(U, psi, 0.12))
    assert np.max(np.abs(lhs - rhs)) < 1e-13


def test_kappa_zero_is_identity():
    L = (2, 2, 2, 4)
    U = synth.gauge_field(L, 0.4, 1)
    psi = synth.complex_gaussian(1, 2, L + (4, 3))
    assert np.array_equal(apply_D(U, psi, 0.0), psi)


@pytest.mark.parametrize("time_bc", [-1, 1])
def test_sparse_matrix_equals_shift_form(time_bc):
    """Two independent formulations of D agree (full lattice and restricted)."""
    L = (4, 4, 2, 4)
    V = int(np.prod(L))
    U = synth.gauge_field(L, 0.5, 4)
    psi = synth.complex_gaussian(4, 2, L + (4, 3))
    M = dirac_matrix(U, 0.14, np.arange(V), time_bc)
    a = (M @ psi.reshape(-1)).reshape(psi.shape)
    b = apply_D(U, psi, 0.14, time_bc)
    assert np.max(np.abs(a - b)) < 1e-13
    rng = np.random.default_rng(0)
    mask = rng.random(L) < 0.6
    sites = np.flatnonzero(mask.ravel())
    Mx = dirac_matrix(U, 0.14, sites, time_bc)
    ax = Mx @ psi.reshape(V, 12)[sites].ravel()
    bx = apply_D_restricted(U, psi, 0.14, mask, time_bc).reshape(V, 12)[sites].ravel()
    assert np.max(np.abs(ax - bx)) < 1e-13
    # D_X equals the dense global D with rows and columns masked (brute force)
    Dd = M.toarray()
    idx = (12 * sites[:, None] + np.arange(12)[None, :]).ravel()
    assert np.max(np.abs(Dd[np.ix_(idx, idx)] - Mx.toarray())) == 0.0
    other = np.setdiff1d(np.arange(V), sites)
    jdx = (12 * other[:, None] + np.arange(12)[None, :]).ravel()
    Dxy = dirac_block(U, 0.14, sites, other, time_bc).toarray()
    assert np.max(np.abs(Dd[np.ix_(idx, jdx)] - Dxy)) == 0.0
