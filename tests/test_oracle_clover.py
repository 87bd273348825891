"""Pins of the oracle's clover (Sheikholeslami-Wohlert) term, the site-local 12x12
term the paper allows in D (Sec. 1), A(x) = 1 + i kappa c_sw sum_{mu<nu}
sigma_mu_nu F_mu_nu(x):

* free field (unit links): A = 1 and D equals the Wilson operator;
* A(x) is Hermitian and commutes with gamma_5 (two 6x6 chiral blocks);
* abelian constant field in one plane: F_mu_nu = i sin(b q) in closed form,
  zero in the other planes, F_nu_mu = -F_mu_nu;
* gauge covariance A^g(x) = g(x) A(x) g(x)^+;
* gamma_5-hermiticity of the dense D with the clover term;
* Eq. (detD) closes with the clover term (the identity is algebraic in the
  block structure of D, which a site-local term does not change);
* locality: with the clover term a core link of the boundary layer reaches the
  neighbouring block's action, a link one layer inside does not.
"""

import numpy as np
import pytest

from paper_2211_06902_gb300 import synth
from oracle.dd import Oracle
from oracle.geometry import Decomposition, uniform_cores
from oracle.lattice import (apply_D, clover_term, dirac_matrix, field_strength,
                            gauge_transform_links, sigma_munu)

G5 = np.kron(np.diag([1.0, 1.0, -1.0, -1.0]), np.eye(3))


def _unit_links(L):
    U = np.zeros(tuple(L) + (4, 3, 3), dtype=np.complex128)
    U[...] = np.eye(3)
    return U


def test_free_field():
    L = (4, 2, 2, 2)
    U = _unit_links(L)
    A = clover_term(U, 0.13, 1.7)
    assert np.allclose(A, np.eye(12), atol=1e-15)
    psi = synth.complex_gaussian(1, synth.TAG_RHS, L + (4, 3))
    assert np.allclose(apply_D(U, psi, 0.13, csw=1.7), apply_D(U, psi, 0.13))


def test_hermitian_and_chirally_block_diagonal():
    L = (4, 4, 2, 2)
    U = synth.gauge_field(L, 0.6, 3)
    A = clover_term(U, 0.13, 1.5).reshape(-1, 12, 12)
    assert np.abs(A - np.conj(np.swapaxes(A, 1, 2))).max() < 1e-14
    assert np.abs(A @ G5 - G5 @ A).max() < 1e-14
    assert np.abs(A - np.eye(12)).max() > 1e-3                  # the term is not trivial


@pytest.mark.parametrize("mu,nu", [(0, 1), (1, 3), (2, 3)])
def test_abelian_constant_field(mu, nu):
    """U_nu(x) = exp(i b x_mu q) with b L_mu in 2 pi Z, all other links 1: every
    plaquette of the mu-nu plane is exp(i b q), so F_mu_nu = i sin(b q)."""
    L = (4, 4, 4, 4)
    b = 2 * np.pi / L[mu]
    q = np.array([1.0, -1.0, 0.0])
    U = _unit_links(L)
    xs = np.indices(L)[mu]
    U[..., nu, :, :] = np.einsum("...,ab->...ab", np.ones(L), np.eye(3))
    for c in range(3):
        U[..., nu, c, c] = np.exp(1j * b * xs * q[c])
    expect = 1j * np.diag(np.sin(b * q))
    F = field_strength(U, mu, nu)
    assert np.abs(F - expect).max() < 1e-14
    assert np.abs(field_strength(U, nu, mu) + F).max() < 1e-14
    for a in range(4):
        for c in range(a + 1, 4):
            if (a, c) != (min(mu, nu), max(mu, nu)):
                assert np.abs(field_strength(U, a, c)).max() < 1e-14
    kappa, csw = 0.12, 1.3
    ref = np.eye(12) + 1j * kappa * csw * np.kron(sigma_munu()[mu, nu], expect)
    assert np.abs(clover_term(U, kappa, csw) - ref).max() < 1e-14


def test_gauge_covariance():
    L = (4, 4, 2, 2)
    U = synth.gauge_field(L, 0.5, 8)
    g = synth.gauge_field(L, 1.0, 9)[..., 0, :, :]
    A = clover_term(U, 0.13, 1.2)
    Ag = clover_term(gauge_transform_links(U, g), 0.13, 1.2)
    G = np.einsum("st,...ab->...satb", np.eye(4), g).reshape(tuple(L) + (12, 12))
    assert np.abs(Ag - G @ A @ np.conj(np.swapaxes(G, -1, -2))).max() < 1e-13


def test_gamma5_hermiticity():
    L = (4, 2, 2, 2)
    U = synth.gauge_field(L, 0.5, 2)
    V = int(np.prod(L))
    D = dirac_matrix(U, 0.13, np.arange(V), csw=1.4).toarray()
    g5 = np.kron(np.eye(V), G5)
    assert np.abs(g5 @ D @ g5 - D.conj().T).max() < 1e-14
    assert np.abs(D - dirac_matrix(U, 0.13, np.arange(V)).toarray()).max() > 1e-3


def test_detD_identity_with_clover():
    L, cores = (4,) * 4, uniform_cores((4,) * 4, 1, 1)
    U = synth.gauge_field(L, 0.4, 5)
    f = Oracle(U, 0.13, Decomposition(L, cores), csw=1.0).logdet_factors()
    rhs = f["W1"][1] + f["Lambda1"][1] + sum(x[1] for x in f["Omega"]) - sum(x[1] for x in f["Phi"])
    assert abs(f["D"][1] - rhs) < 1e-9
    V = int(np.prod(L))
    wilson = np.linalg.slogdet(dirac_matrix(U, 0.13, np.arange(V)).toarray())[1]
    assert abs(f["D"][1] - wilson) > 1e-3                       # the clover term changes det D


def _parts_fd(U, g, csw, x, mu, t=3, eps=1e-4):
    from scipy.linalg import expm
    from oracle.dd import field_roots, gell_mann
    u = field_roots(2, 0.5)
    chis = [synth.complex_gaussian(2, synth.TAG_CHI, g.L + (4, 3)) * g.dPi[..., None, None]]
    out = []
    for e in (eps, -eps):
        Up = U.copy()
        Up[x + (mu,)] = expm(1j * e * gell_mann()[t] / 2) @ U[x + (mu,)]
        S, sb, sr = Oracle(Up, 0.13, g, csw=csw).multiboson_action(u, chis)
        out.append(np.array(list(sb) + [sr]))
    return (out[0] - out[1]) / (2 * eps)


def test_clover_locality_needs_one_more_layer():
    """With the clover term a link of the core's boundary layer enters the clover
    term of the adjacent frame sites, which lie in the neighbouring block's
    Omega0^b, so S^b depends on it (here the 1D case: dPi1 is empty and S^r = 0);
    a link one layer inside the core reaches no frame site's clover, so only S^a
    of its own block changes.  Without the clover term the boundary-layer link
    enters no other block either."""
    L, cores = (8, 4, 4, 2), [[(0, 2), (4, 6)], [], [], []]
    U = synth.gauge_field(L, 0.4, 6)
    g = Decomposition(L, cores)
    inner, edge = (1, 0, 0, 0), (0, 0, 0, 0)            # spatial links of block 0's core
    d_in = _parts_fd(U, g, 1.0, inner, 1)
    d_edge = _parts_fd(U, g, 1.0, edge, 1)
    d_edge_wilson = _parts_fd(U, g, 0.0, edge, 1)
    assert abs(d_in[0]) > 1e-4                           # S^0 depends on its core links
    assert np.abs(d_in[1:]).max() < 1e-8                 # S^1 and S^r do not
    assert abs(d_edge[1]) > 1e-6                         # clover: S^1 sees the boundary layer
    assert np.abs(d_edge_wilson[1:]).max() < 1e-8        # Wilson: it does not
