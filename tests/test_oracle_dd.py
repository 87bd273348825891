"""Pins of the oracle's solves, w, roots, multi-boson action and log-det factors.

* Eq. (detD): ln|det D| = ln|det W_1| + ln|det D_Lambda1|
  + sum_a [ln|det D_Omega0^a| - ln|det D_Phi1^a|], every factor a dense LU of
  an independently assembled matrix, on 4^4 and 6x4^3 (Sec. 3).
* W_1 is fixed by three printed statements (Sec. 3), each checked against
  dense blocks of D assembled here: the upper-right block of Eq. (offdiagW1);
  M = diag(D^d, D^_{dPi1}) W_1 is gamma_5-hermitian (D^d and D^_{dPi1} in their
  printed forms); the Schur complement of M onto dLambda0 is the D~ of Eq.
  (Dtilde).  Given the first, the second fixes the lower-left block and the
  third then fixes the upper-left one, so W_1 is determined.
* Eq. (WW): det P_N(W_1) = c_N^n prod_{k<=N/2} det(W_{u_k}^dag W_{u_k}), i.e.
  the conjugate roots pair up; the Dirichlet-extension completion of the
  hopping block (the same determinant, Eq. detD) breaks it (planted mistake).
* w as a vector operation equals w as an assembled dense matrix.
* kappa = 0 gives w = 0 and S = sum_k |u_k|^2 |chi_k|^2.
* Block locality of S^a and of S^r (Sec. 4, Eqs. localMB, globalMB).
* Gauge invariance of S.
* Roots: the polynomial identity z c_N prod (z - z_k) = 1 - R_{N+1}(z) with
  Chebyshev R evaluated by numpy's Chebyshev module; c = 0 gives roots of unity.
* The oracle's iterative solver agrees with a sparse direct LU.
* Reweighting factor (Eq. rw): the product form c_N W_1 prod (W_1 - z_k) equals the
  spectral form with numpy's Chebyshev R; c = 0 gives 1 - w^{N+1}; ln|W_N| from the
  spectrum equals the sum of dense LU log-dets of the factors; the Gaussian-source
  estimator's sample mean lies within 5 exact sigma of 1/det(M^dag M).
* Force on the active links (links inside a core): central finite differences of the
  total action S along exp(i eps T_t) equal the block-local analytic force (so S^r and
  the other blocks do not depend on those links), including a link across the
  antiperiodic time boundary; planted sign, projector, boundary and adjoint mistakes fail.
* d ln|det D_Omega0^a| / d eps on active links against finite differences of the dense
  slogdet; the block-local effective force against finite differences of the whole
  factorized effective action of Eq. (SFeffN).
"""

import math

import numpy as np
import pytest
from numpy.polynomial import chebyshev as C

from paper_2211_06902_gb300 import synth
from oracle.dd import Oracle, bicgstab, field_roots, gell_mann, pn_leading, roots
from oracle.geometry import Decomposition, uniform_cores
from oracle.lattice import dirac_matrix, gauge_transform_links

L44 = (4, 4, 4, 4)
L6444 = (6, 4, 4, 4)
CORES6444 = [[(0, 1), (3, 4)]] + [[(0, 0), (2, 2)]] * 3


def _slog_sum(pairs, signs=(1,)):
    return sum(p[1] for p in pairs)


@pytest.mark.parametrize("L,cores", [(L44, uniform_cores(L44, 1, 1)), (L6444, CORES6444)])
def test_det_factorization_identity(L, cores):
    U = synth.gauge_field(L, 0.3, 1)
    o = Oracle(U, 0.13, Decomposition(L, cores))
    f = o.logdet_factors()
    rhs = f["W1"][1] + f["Lambda1"][1] + sum(x[1] for x in f["Omega"]) - sum(x[1] for x in f["Phi"])
    assert abs(f["D"][1] - rhs) < 1e-10
    sign = f["W1"][0] * f["Lambda1"][0] * np.prod([x[0] for x in f["Omega"]]) \
        / np.prod([x[0] for x in f["Phi"]])
    assert abs(sign - f["D"][0]) < 1e-10
    assert abs(f["D"][0].imag) < 1e-12                  # det D real (gamma_5-hermiticity)


_W_CACHE = {}


def _w_case(L, cores, seed=1):
    """(U, geometry, oracle, dense w) of one lattice; the dense w is assembled once
    per case and shared by the tests that read it (none of them modifies it)."""
    key = (tuple(L), repr(cores), seed)
    if key not in _W_CACHE:
        U = synth.gauge_field(L, 0.3, seed)
        g = Decomposition(L, cores)
        o = Oracle(U, 0.13, g)
        _W_CACHE[key] = (U, g, o, o.w_matrix())
    return _W_CACHE[key]


def test_det_identity_fails_for_a_wrong_w():
    """A plausible mistake (dropping the frame solve) breaks Eq. (detD)."""
    U, g, o, w = _w_case(L44, uniform_cores(L44, 1, 1))
    dpi = g.sites(g.dPi)
    isC = np.repeat(g.C.ravel()[dpi], 12)
    w_bad = w.copy()
    w_bad[np.ix_(isC, ~isC)] = 0
    f = o.logdet_factors()
    rhs_bad = np.linalg.slogdet(np.eye(len(w)) - w_bad)[1] + f["Lambda1"][1] \
        + sum(x[1] for x in f["Omega"]) - sum(x[1] for x in f["Phi"])
    assert abs(f["D"][1] - rhs_bad) > 1e-3


def test_w_vector_equals_w_matrix():
    U = synth.gauge_field(L44, 0.4, 2)
    g = Decomposition(L44, uniform_cores(L44, 1, 1))
    o = Oracle(U, 0.13, g)
    chi = synth.complex_gaussian(2, synth.TAG_CHI, L44 + (4, 3)) * g.dPi[..., None, None]
    dpi = g.sites(g.dPi)
    wv = o.apply_w(chi).reshape(-1, 12)[dpi].ravel()
    wm = o.w_matrix() @ chi.reshape(-1, 12)[dpi].ravel()
    assert np.linalg.norm(wv - wm) / np.linalg.norm(wm) < 1e-11
    out = o.apply_w(chi)
    assert np.all(out[~g.dPi] == 0)


L2D = (8, 8, 2, 2)
CORES2D = [[(0, 1), (4, 5)], [(0, 1), (4, 5)], [], []]
W1_CASES = [(L44, uniform_cores(L44, 1, 1)), (L6444, CORES6444), (L2D, CORES2D)]


class _Dense:
    """Dense blocks D_{X,Y} of the full operator assembled once (no oracle helpers)."""

    def __init__(self, U, kappa, g):
        V = int(np.prod(g.L))
        self.D = dirac_matrix(U, kappa, np.arange(V)).toarray()
        self.g = g

    @staticmethod
    def idx(sites):
        return (12 * np.asarray(sites)[:, None] + np.arange(12)).ravel()

    def __call__(self, X, Y=None):
        Y = X if Y is None else Y
        return self.D[np.ix_(self.idx(X), self.idx(Y))]

    def inv(self, X):
        return np.linalg.inv(self(X))


@pytest.mark.parametrize("L,cores", W1_CASES)
def test_w1_is_fixed_by_the_printed_blocks(L, cores):
    """(i) Eq. (offdiagW1): rows dLambda0^a of W_1 on dPi1 are P D_Omega^-1 D_{Phi, X*}
    (zero off X* = dOmega0^{a*}); (ii) M = diag(D^d, D^_{dPi1}) W_1 is gamma_5-hermitian,
    with D^d_a = D_{dL0a} - D_{dL0a,L0bar} D_{L0bar}^-1 D_{L0bar,dL0a} - D_{dL0a,Phi} D_Phi^-1
    D_{Phi,dL0a} and D^_{dPi1} = D_{dPi1} - D_{dPi1,E} D_E^-1 D_{E,dPi1}; (iii) the Schur
    complement of M onto dLambda0 is Eq. (Dtilde)'s D~ = D_{dL0} - D_{dL0,L0bar} D_{L0bar}^-1
    D_{L0bar,dL0} - D_{dL0,Lambda1} D_{Lambda1}^-1 D_{Lambda1,dL0}."""
    U, g, o, w = _w_case(L, cores)
    d = _Dense(U, 0.13, g)
    dpi = g.sites(g.dPi)
    pos = np.full(int(np.prod(L)), -1)
    pos[dpi] = np.arange(len(dpi))
    r = lambda sites: d.idx(pos[np.asarray(sites)])            # rows of W_1 (dPi order)
    W1 = np.eye(12 * len(dpi)) - w
    Bs, Cs, Es = g.sites(g.B), g.sites(g.C), g.sites(g.E)
    Diag = np.zeros_like(W1)
    for a in range(g.nblocks):
        B, F = g.sites(g.B_mask[a]), g.sites(g.phi_mask[a])
        A = g.sites(g.core_mask[a] & ~g.B_mask[a])
        Dd = d(B) - d(B, F) @ d.inv(F) @ d(F, B)
        if len(A):
            Dd -= d(B, A) @ d.inv(A) @ d(A, B)
        Diag[np.ix_(r(B), r(B))] = Dd
        # (i)
        om = g.sites(g.omega_mask[a])
        G = d.inv(om)
        ib = d.idx(np.searchsorted(om, B))
        iF = d.idx(np.searchsorted(om, F))
        Xs = g.sites(g.ext_star_mask[a])
        if len(Cs):
            ref = np.zeros((12 * len(B), 12 * len(Cs)), dtype=complex)
            if len(Xs):
                ref[:, d.idx(np.searchsorted(Cs, Xs))] = G[np.ix_(ib, iF)] @ d(F, Xs)
            got = W1[np.ix_(r(B), r(Cs))]
            assert np.abs(got - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())
    if len(Cs):
        Sh = d(Cs) - (d(Cs, Es) @ d.inv(Es) @ d(Es, Cs) if len(Es) else 0)
        Diag[np.ix_(r(Cs), r(Cs))] = Sh
    M = Diag @ W1
    g5 = np.tile(np.repeat([1.0, -1.0], 6), len(dpi))
    # (ii)
    assert np.abs(g5[:, None] * M * g5[None, :] - M.conj().T).max() < 1e-12 * np.abs(M).max()
    # (iii)
    l1, a0 = g.sites(g.Lambda1), g.sites(g.A)
    Dt = d(Bs) - d(Bs, l1) @ d.inv(l1) @ d(l1, Bs)
    if len(a0):
        Dt -= d(Bs, a0) @ d.inv(a0) @ d(a0, Bs)
    rb, rc = r(Bs), r(Cs)
    schur = M[np.ix_(rb, rb)]
    if len(Cs):
        schur = schur - M[np.ix_(rb, rc)] @ np.linalg.solve(M[np.ix_(rc, rc)], M[np.ix_(rc, rb)])
    assert np.abs(schur - Dt).max() < 1e-11 * np.abs(Dt).max()


def _eq_ww_gap(W1, N, c):
    """ln det P_N(W_1) minus ln[c_N^n prod_{k<=N/2} det(W_{u_k}^dag W_{u_k})], complex
    (P_N(W_1) = c_N prod_{k=1..N} (W_1 - z_k), W_1 - z_k = u_k - w = W_{u_k})."""
    n = len(W1)
    u = roots(N, c)
    lds = [np.linalg.slogdet(W1 - (1 - uk) * np.eye(n)) for uk in u]
    lhs = sum(ld + 1j * np.angle(s) for s, ld in lds)
    rhs = sum(2 * ld for _, ld in lds[: N // 2])
    gap = lhs - rhs
    return gap.real, math.remainder(gap.imag, 2 * math.pi), abs(lhs.real)


@pytest.mark.parametrize("L,cores", W1_CASES)
def test_eq_ww_pairs_conjugate_roots(L, cores):
    """Eq. (WW) holds exactly: the roots k and N+1-k are complex conjugates and
    det(W_1 - conj z) = conj det(W_1 - z) (the characteristic polynomial of W_1 is real)."""
    U, g, o, w = _w_case(L, cores)
    W1 = np.eye(len(w)) - w
    for N, c in ([(4, 0.5), (6, 0.0)] if L == L44 else [(4, 0.5)]):
        re, im, scale = _eq_ww_gap(W1, N, c)
        assert abs(re) < 1e-10 * max(1.0, scale) and abs(im) < 1e-10, (N, c, re, im)


def test_dirichlet_completion_keeps_det_but_breaks_eq_ww():
    """Planted mistake: completing the upper-left block of W_1 as the Dirichlet
    extension (rows dLambda0^a: P D_Omega^-1 D_{Omega,ext}; rows dPi1:
    P D_Lambda1^-1 D_{Lambda1,dL0}) gives the same det W_1 (Eq. detD) but a
    characteristic polynomial that is not real, so Eq. (WW) fails."""
    U, g, o, w = _w_case(L44, uniform_cores(L44, 1, 1))
    d = _Dense(U, 0.13, g)
    dpi = g.sites(g.dPi)
    pos = np.full(int(np.prod(L44)), -1)
    pos[dpi] = np.arange(len(dpi))
    r = lambda sites: d.idx(pos[np.asarray(sites)])
    Wd = np.eye(12 * len(dpi), dtype=complex)
    for a in range(g.nblocks):
        om, ex, B = g.sites(g.omega_mask[a]), g.sites(g.ext_mask[a]), g.sites(g.B_mask[a])
        G = d.inv(om) @ d(om, ex)
        Wd[np.ix_(r(B), r(ex))] += G[d.idx(np.searchsorted(om, B))]
    l1, Bs, Cs = g.sites(g.Lambda1), g.sites(g.B), g.sites(g.C)
    G = d.inv(l1) @ d(l1, Bs)
    Wd[np.ix_(r(Cs), r(Bs))] += G[d.idx(np.searchsorted(l1, Cs))]
    W1 = np.eye(len(Wd)) - w
    assert abs(np.linalg.slogdet(Wd)[1] - np.linalg.slogdet(W1)[1]) < 1e-10
    re, im, _ = _eq_ww_gap(Wd, 4, 0.5)
    assert abs(re) > 1e-4
    re, im, _ = _eq_ww_gap(W1, 4, 0.5)
    assert abs(re) < 1e-10


def test_kappa_zero_action():
    U = synth.gauge_field(L44, 0.3, 1)
    g = Decomposition(L44, uniform_cores(L44, 1, 1))
    o = Oracle(U, 0.0, g)
    u = field_roots(4, 0.5)
    chis = [synth.complex_gaussian(1, 10 + k, L44 + (4, 3)) * g.dPi[..., None, None]
            for k in range(2)]
    S, sa, sr = o.multiboson_action(u, chis)
    expect = sum(abs(uk) ** 2 * np.sum(np.abs(c) ** 2) for uk, c in zip(u, chis))
    assert abs(S - expect) < 1e-12 * expect
    assert abs(S - (sum(sa) + sr)) < 1e-12 * S


def test_block_locality_of_the_action():
    """A link inside Lambda0^a changes only S^a; a link inside the frame changes
    S^r and only the S^b whose framed block touches it (Sec. 4)."""
    L = (6,) * 4
    g = Decomposition(L, uniform_cores(L, 2, 1))
    U = synth.gauge_field(L, 0.3, 1)
    u = field_roots(4, 0.5)[:1]
    chi = [synth.complex_gaussian(1, synth.TAG_CHI, L + (4, 3)) * g.dPi[..., None, None]]
    S0, sa0, sr0 = Oracle(U, 0.13, g).multiboson_action(u, chi)
    assert abs(S0 - (sum(sa0) + sr0)) < 1e-12 * S0
    # link U_1(x) with x and x+1^ in the core of block 5
    a = 5
    x = tuple(b[0] for b in g.blocks[a].core)
    U1 = U.copy()
    U1[x + (1,)] = synth.gauge_field((1, 1, 1, 1), 0.9, 77)[0, 0, 0, 0, 0]
    S1, sa1, sr1 = Oracle(U1, 0.13, g).multiboson_action(u, chi)
    assert sa1[a] != sa0[a]
    assert all(sa1[b] == sa0[b] for b in range(g.nblocks) if b != a)
    assert sr1 == sr0
    # link U_2(y) with y and y+2^ in the frame Lambda1
    ys = np.argwhere(g.Lambda1 & np.roll(g.Lambda1, -1, axis=2))
    y = tuple(int(v) for v in ys[0])
    U2 = U.copy()
    U2[y + (2,)] = synth.gauge_field((1, 1, 1, 1), 0.9, 78)[0, 0, 0, 0, 0]
    S2, sa2, sr2 = Oracle(U2, 0.13, g).multiboson_action(u, chi)
    assert sr2 != sr0
    yp = list(y)
    yp[2] = (yp[2] + 1) % L[2]
    # S^b holds D_{Omega_b} and, through D^h, the frame pieces Phi_c that meet Phi_b or
    # dOmega0^{b*}, or whose dOmega0^{c*} meets Phi_b (frame links only)
    def reach(b):
        m = g.omega_mask[b].copy()
        for c in range(g.nblocks):
            if c != b and ((g.phi_mask[c] & (g.phi_mask[b] | g.ext_star_mask[b])).any()
                           or (g.phi_mask[b] & g.ext_star_mask[c]).any()):
                m |= g.phi_mask[c]
        return m
    for b in range(g.nblocks):
        if not (reach(b)[y] or reach(b)[tuple(yp)]):
            assert sa2[b] == sa0[b]


def test_gauge_invariance_of_the_action():
    L = L6444
    g = Decomposition(L, CORES6444)
    U = synth.gauge_field(L, 0.3, 2)
    gx = synth.gauge_transform(9, L)
    u = field_roots(4, 0.5)
    chis = [synth.complex_gaussian(2, 20 + k, L + (4, 3)) * g.dPi[..., None, None] for k in range(2)]
    S, sa, sr = Oracle(U, 0.13, g).multiboson_action(u, chis)
    gchis = [np.einsum("...ab,...sb->...sa", gx, c) for c in chis]
    Sg, sag, srg = Oracle(gauge_transform_links(U, gx), 0.13, g).multiboson_action(u, gchis)
    assert abs(S - Sg) < 1e-11 * S
    assert np.allclose(sa, sag, rtol=1e-10)


@pytest.mark.parametrize("N,c", [(4, 0.5), (12, 0.3), (24, 0.7), (6, 0.0)])
def test_roots_polynomial_identity(N, c):
    u = roots(N, c)
    z_k = 1 - u
    rng = np.random.default_rng(N)
    for z in rng.normal(size=4) + 1j * rng.normal(size=4):
        if c == 0:
            rhs = 1 - (1 - z) ** (N + 1)                    # limit c -> 0
            lead = -(-1.0) ** (N + 1)
        else:
            coef = np.zeros(N + 2)
            coef[N + 1] = 1
            rhs = 1 - C.chebval((1 - z) / c, coef) / C.chebval(1 / c, coef)
            lead = -(2.0 ** N) * (-1.0 / c) ** (N + 1) / C.chebval(1 / c, coef)
        lhs = z * lead * np.prod(z - z_k)
        assert abs(lhs - rhs) < 1e-10 * max(1, abs(rhs))


def test_roots_special_cases():
    u = roots(6, 0.0)
    assert np.allclose(u, np.exp(2j * np.pi * np.arange(1, 7) / 7))
    u = roots(8, 0.4)
    assert np.allclose(u[::-1], np.conj(u))                 # u_{N+1-k} = conj(u_k)
    assert len(field_roots(8, 0.4)) == 4
    with pytest.raises(ValueError):
        field_roots(5, 0.4)


def test_iterative_solver_matches_direct_lu():
    L = (4, 4, 4, 4)
    U = synth.gauge_field(L, 0.5, 6)
    V = int(np.prod(L))
    sites = np.arange(0, V, 2)
    M = dirac_matrix(U, 0.13, sites)
    b = synth.complex_gaussian(6, synth.TAG_RHS, (M.shape[0],))
    from scipy.sparse.linalg import splu
    xd = splu(M.tocsc()).solve(b)
    xi, rel = bicgstab(lambda v: M @ v, b, 1e-13)
    assert rel < 1e-12
    assert np.linalg.norm(xi - xd) < 1e-11 * np.linalg.norm(xd)


def test_heatbath_fields_reproduce_their_gaussian_sources():
    """chi_k = W_{u_k}^{-1} eta_k (dense solve) makes the multi-boson action,
    evaluated independently by the vector form of w, equal sum_k |eta_k|^2
    (Sec. 4, Eqs. WW / MBaction); the fields live on dPi only; a plausible
    mistake (solving with the conjugate roots) breaks the identity."""
    U = synth.gauge_field(L44, 0.3, 1)
    g = Decomposition(L44, uniform_cores(L44, 1, 1))
    o = Oracle(U, 0.13, g)
    u = field_roots(4, 0.5)
    etas = [synth.complex_gaussian(3, 40 + k, L44 + (4, 3)) * g.dPi[..., None, None]
            for k in range(len(u))]
    chis = o.heatbath(u, etas)
    S, _, _ = o.multiboson_action(u, chis)
    ref = sum(float(np.vdot(e, e).real) for e in etas)
    assert abs(S - ref) <= 1e-10 * ref
    assert all(np.all(c[~g.dPi] == 0) for c in chis)
    bad = o.heatbath(np.conj(u), etas)
    S_bad, _, _ = o.multiboson_action(u, bad)
    assert abs(S_bad - ref) > 1e-3 * ref


L1D = (8, 4, 4, 2)
CORES1D = [[(0, 1), (4, 5)], [], [], []]      # thick time slices: only x0 decomposed


def test_one_dimensional_decomposition_formula():
    """Sec. 3, 1D case (Fig. 1dDD): with only time decomposed, dPi1 is empty,
    every frame slice lies in two Phi's, so prod det D_Phi = (det D_Lambda1)^2,
    and Eq. (detD) becomes det D = det W_1 prod_a det D_Omega^a / det D_Lambda1."""
    U = synth.gauge_field(L1D, 0.4, 6)
    g = Decomposition(L1D, CORES1D)
    assert g.nblocks == 2 and not g.C.any() and np.array_equal(g.dPi, g.B)
    cover = sum(m.astype(int) for m in g.phi_mask)
    assert np.all(cover[g.Lambda1] == 2) and np.all(cover[g.Lambda0] == 0)
    f = Oracle(U, 0.13, g).logdet_factors()
    phi = sum(x[1] for x in f["Phi"])
    assert abs(phi - 2 * f["Lambda1"][1]) < 1e-10
    one_d = f["W1"][1] + sum(x[1] for x in f["Omega"]) - f["Lambda1"][1]
    assert abs(f["D"][1] - one_d) < 1e-10


def test_undecomposed_direction_adds_no_hyperplane():
    g1 = Decomposition(L1D, CORES1D)
    t = np.indices(L1D)[0]
    assert np.array_equal(g1.dPi, np.isin(t, [0, 1, 4, 5]))
    with pytest.raises(ValueError):
        Decomposition(L1D, [[], [], [], []])
    with pytest.raises(ValueError):
        Decomposition(L1D, [[(0, 1)], [], [], []])


def test_two_dimensional_decomposition_identity():
    """Time and x1 decomposed, x2 and x3 not: the frame has corners (dPi1 is not
    empty) and the domains wrap around in x2, x3; Eq. (detD) holds as in 4D."""
    L = (8, 8, 2, 2)
    cores = [[(0, 1), (4, 5)], [(0, 1), (4, 5)], [], []]
    U = synth.gauge_field(L, 0.4, 7)
    g = Decomposition(L, cores)
    assert g.nblocks == 4 and g.C.any()
    f = Oracle(U, 0.13, g).logdet_factors()
    rhs = f["W1"][1] + f["Lambda1"][1] + sum(x[1] for x in f["Omega"]) - sum(x[1] for x in f["Phi"])
    assert abs(f["D"][1] - rhs) < 1e-10


# -- reweighting factor W_N = det{1 - R_{N+1}(W_1)} (Sec. 4, Eq. rw) ---------------
RW_L = (4, 2, 2, 2)
RW_CORES = [[(0, 0), (2, 2)], [], [], []]


def _rw_case(kappa):
    U = synth.gauge_field(RW_L, 0.3, 1)
    g = Decomposition(RW_L, RW_CORES)
    return Oracle(U, kappa, g), g


def _dpi_vec(g, f):
    return f.reshape(-1, 12)[g.sites(g.dPi)].reshape(-1)


def _r_of_eigs(lam, N, c):
    """R_{N+1} at the eigenvalues 1 - lam of W_1, by numpy's Chebyshev module."""
    if c == 0.0:
        return lam ** (N + 1)
    coef = np.zeros(N + 2)
    coef[N + 1] = 1
    return C.chebval(lam / c, coef) / C.chebval(1 / c, coef)


@pytest.mark.parametrize("N,c", [(4, 0.5), (2, 0.3), (6, 0.0)])
def test_reweight_product_form_equals_spectral_form(N, c):
    """M eta from the product c_N W_1 prod (W_1 - z_k) equals V diag(1 - R(1 - lam)) V^-1 eta
    with w = V diag(lam) V^-1 and R from numpy's Chebyshev series."""
    o, g = _rw_case(0.13)
    W = o.w_matrix()
    lam, V = np.linalg.eig(W)
    eta = synth.complex_gaussian(2, synth.TAG_CHI, RW_L + (4, 3)) * g.dPi[..., None, None]
    got = _dpi_vec(g, o.reweight_apply(N, c, eta))
    e = _dpi_vec(g, eta)
    ref = V @ ((1 - _r_of_eigs(lam, N, c)) * np.linalg.solve(V, e))
    assert np.linalg.norm(got - ref) < 1e-9 * np.linalg.norm(e)


def test_reweight_c0_is_one_minus_w_power():
    """c = 0: roots of unity, R_{N+1}(W_1) = w^{N+1}, M = 1 - w^{N+1}."""
    o, g = _rw_case(0.13)
    N = 4
    eta = synth.complex_gaussian(3, synth.TAG_CHI, RW_L + (4, 3)) * g.dPi[..., None, None]
    y = eta
    for _ in range(N + 1):
        y = o.apply_w(y)
    m = o.reweight_apply(N, 0.0, eta)
    assert np.linalg.norm(m - (eta - y)) < 1e-10 * np.linalg.norm(eta)


@pytest.mark.parametrize("N,c", [(4, 0.5), (6, 0.0)])
def test_reweight_determinant_two_ways(N, c):
    """ln|W_N| as sum_i ln|1 - R(1 - lam_i)| equals
    n ln|c_N| + ln|det W_1| + sum_k ln|det(u_k - w)| (dense LU of each factor)."""
    o, g = _rw_case(0.13)
    W = o.w_matrix()
    n = W.shape[0]
    spectral = float(np.sum(np.log(np.abs(1 - _r_of_eigs(np.linalg.eigvals(W), N, c)))))
    product = n * math.log(abs(pn_leading(N, c))) + np.linalg.slogdet(np.eye(n) - W)[1]
    product += sum(np.linalg.slogdet(uk * np.eye(n) - W)[1] for uk in roots(N, c))
    assert abs(spectral - product) < 1e-9 * max(1.0, abs(product))


def test_reweight_estimator_mean():
    """E[exp(|eta|^2 - |M eta|^2)] = 1/det(M^dag M) over complex Gaussian sources;
    the sample mean of 300 sources lies within 5 sigma, sigma from the exact
    variance det(2 M^dag M - 1)^-1 - det(M^dag M)^-2 (dense M from the spectrum)."""
    N, c, K = 2, 0.5, 300
    o, g = _rw_case(0.11)
    W = o.w_matrix()
    n = W.shape[0]
    lam, V = np.linalg.eig(W)
    M = V @ np.diag(1 - _r_of_eigs(lam, N, c)) @ np.linalg.inv(V)
    A = M.conj().T @ M
    ld_a = np.linalg.slogdet(A)[1]
    ld_2a = np.linalg.slogdet(2 * A - np.eye(n))[1]
    mean = math.exp(-ld_a)
    sigma = math.sqrt(math.exp(-ld_2a) - mean ** 2)
    etas = [synth.complex_gaussian(5, synth.TAG_CHI + k, RW_L + (4, 3)) * g.dPi[..., None, None]
            for k in range(K)]
    s = o.reweight_samples(N, c, etas)
    assert mean < 0.8                                    # the factor is far from 1 here
    assert abs(np.mean(np.exp(s)) - mean) < 5 * sigma / math.sqrt(K)


# -- force of the factorized multi-boson action on the active links (Sec. 4) -------
def _perturbed_action(U, kappa, g, u, chis, x, mu, t, eps):
    from scipy.linalg import expm
    Up = U.copy()
    Up[tuple(x) + (mu,)] = expm(1j * eps * gell_mann()[t] / 2) @ U[tuple(x) + (mu,)]
    return Oracle(Up, kappa, g).multiboson_action(u, chis)[0]


@pytest.mark.parametrize("case", ["1D", "2D"])
def test_mb_force_matches_finite_differences_of_total_action(case):
    """F = dS/d eps for U_mu(x) -> exp(i eps T_t) U_mu(x) on active links, S the
    total action sum_a S^a + S^r: the block-local force is the whole derivative,
    i.e. S^r and the other blocks' S^b do not depend on the active links."""
    if case == "1D":
        L, cores = (8, 4, 4, 2), [[(0, 1), (4, 5)], [], [], []]
        picks = [(0, 0, 1), (0, 1, 4), (0, 3, 7), (1, 0, 2), (1, 2, 0)]    # (block, link #, t)
    else:
        # two decomposed directions: frame corners, so dPi1 is not empty and the
        # frame-piece term Q chi of the block sources enters
        L, cores = (8, 8, 2, 2), [[(0, 1), (4, 5)], [(0, 1), (4, 5)], [], []]
        picks = [(0, 3, 6), (3, 10, 1), (2, 21, 7)]
    U = synth.gauge_field(L, 0.3, 4)
    g = Decomposition(L, cores)
    o = Oracle(U, 0.13, g)
    u = field_roots(4, 0.5)
    chis = [synth.complex_gaussian(6, synth.TAG_CHI + k, L + (4, 3)) * g.dPi[..., None, None]
            for k in range(len(u))]
    F = o.mb_force(u, chis)
    eps = 1e-4
    for a, n, t in picks:
        links = o.active_links(a)
        x, mu = links[n % len(links)]
        fd = (_perturbed_action(U, 0.13, g, u, chis, x, mu, t, eps)
              - _perturbed_action(U, 0.13, g, u, chis, x, mu, t, -eps)) / (2 * eps)
        assert abs(fd - F[x + (mu, t)]) < 1e-6 * max(1.0, abs(fd)), (a, x, mu, t, fd, F[x + (mu, t)])


def test_mb_force_support_and_time_boundary():
    """The force vanishes off the active links; a core that spans the time extent
    (time not decomposed) has active links across x0 = L0-1 -> 0, whose force
    carries the antiperiodic sign (checked by finite differences)."""
    L, cores = (4, 8, 2, 2), [[], [(0, 1), (4, 5)], [], []]
    U = synth.gauge_field(L, 0.3, 5)
    g = Decomposition(L, cores)
    o = Oracle(U, 0.13, g)
    u = field_roots(2, 0.5)
    chis = [synth.complex_gaussian(7, synth.TAG_CHI, L + (4, 3)) * g.dPi[..., None, None]]
    F = o.mb_force(u, chis)
    act = np.zeros(L + (4,), dtype=bool)
    for a in range(g.nblocks):
        for x, mu in o.active_links(a):
            act[x + (mu,)] = True
    assert np.all(F[~act] == 0) and np.any(F[act] != 0)
    x, mu, t = (L[0] - 1, 0, 0, 1), 0, 2
    assert act[x + (mu,)]
    eps = 1e-4
    fd = (_perturbed_action(U, 0.13, g, u, chis, x, mu, t, eps)
          - _perturbed_action(U, 0.13, g, u, chis, x, mu, t, -eps)) / (2 * eps)
    assert abs(fd - F[x + (mu, t)]) < 1e-6 * max(1.0, abs(fd))


def _fd_links(U, fn, x, mu, t, eps=1e-4):
    from scipy.linalg import expm
    vals = []
    for e in (eps, -eps):
        Up = U.copy()
        Up[tuple(x) + (mu,)] = expm(1j * e * gell_mann()[t] / 2) @ U[tuple(x) + (mu,)]
        vals.append(fn(Up))
    return (vals[0] - vals[1]) / (2 * eps)


def test_logdet_force_matches_finite_differences():
    """d ln|det D_Omega0^a| / d eps on active links against central differences of the
    dense slogdet of the assembled block matrix."""
    L, cores = (8, 4, 4, 2), [[(0, 1), (4, 5)], [], [], []]
    U = synth.gauge_field(L, 0.4, 3)
    g = Decomposition(L, cores)
    o = Oracle(U, 0.13, g)
    G = o.logdet_force()
    for a, n, t in [(0, 0, 2), (0, 5, 7), (1, 3, 0)]:
        x, mu = o.active_links(a)[n]
        sites = g.sites(g.omega_mask[a])
        fd = _fd_links(U, lambda Up: np.linalg.slogdet(dirac_matrix(Up, 0.13, sites).toarray())[1], x, mu, t)
        assert abs(fd - G[x + (mu, t)]) < 1e-6 * max(1.0, abs(fd)), (a, x, mu, t, fd, G[x + (mu, t)])
    assert np.abs(G).max() > 1e-3


def test_effective_force_matches_finite_differences_of_the_effective_action():
    """The block-local force equals the derivative of the whole factorized effective
    action of Eq. (SFeffN): sum_a [-ln|det D_Omega0^a| + ln|det D_Phi1^a|] - ln|det D_Lambda1|
    + S_MB (dense log-dets, total multi-boson action)."""
    L, cores = (8, 4, 4, 2), [[(0, 1), (4, 5)], [], [], []]
    U = synth.gauge_field(L, 0.4, 3)
    g = Decomposition(L, cores)
    o = Oracle(U, 0.13, g)
    u = field_roots(2, 0.5)
    chis = [synth.complex_gaussian(4, synth.TAG_CHI, L + (4, 3)) * g.dPi[..., None, None]]

    def seff(Up):
        ld = lambda m: np.linalg.slogdet(dirac_matrix(Up, 0.13, g.sites(m)).toarray())[1]
        val = -ld(g.Lambda1) + Oracle(Up, 0.13, g).multiboson_action(u, chis)[0]
        for a in range(g.nblocks):
            val += -ld(g.omega_mask[a]) + ld(g.phi_mask[a])
        return val
    F = o.effective_force(u, chis)
    for a, n, t in [(0, 2, 1), (1, 6, 5)]:
        x, mu = o.active_links(a)[n]
        fd = _fd_links(U, seff, x, mu, t)
        assert abs(fd - F[x + (mu, t)]) < 1e-6 * max(1.0, abs(fd)), (a, x, mu, t, fd, F[x + (mu, t)])


def test_logdet_force_noise_estimate_matches_the_exact_trace():
    """The noise estimate of d ln|det D_Omega0^a| / d eps (complex Gaussian noise,
    E[eta eta^dag] = 1) lies within 5 standard errors of the dense trace on every
    active link and generator; a planted mistake (z = D_Omega^{-1} eta instead of
    the adjoint solve) is far outside."""
    L, cores = (8, 4, 4, 2), [[(0, 1), (4, 5)], [], [], []]
    U = synth.gauge_field(L, 0.4, 3)
    g = Decomposition(L, cores)
    o = Oracle(U, 0.13, g)
    exact = o.logdet_force()
    n = 96
    etas = [[synth.complex_gaussian(11, 500 + 100 * a + k, L + (4, 3)) * g.omega_mask[a][..., None, None]
             for k in range(n)] for a in range(g.nblocks)]
    G, SD = o.logdet_force_stochastic(etas)
    act = SD > 0
    assert act.sum() > 100
    z = (G[act] - exact[act]) / (SD[act] / math.sqrt(n))
    assert np.abs(z).max() < 5.0, np.abs(z).max()
    assert np.all(G[~act] == 0)
    # planted mistake: the forward solve in place of the adjoint one
    bad = Oracle(U, 0.13, g)
    bad.omega_solver(0).solve_adjoint_field = bad.omega_solver(0).solve_field
    bad.omega_solver(1).solve_adjoint_field = bad.omega_solver(1).solve_field
    Gb, _ = bad.logdet_force_stochastic(etas)
    zb = (Gb[act] - exact[act]) / (SD[act] / math.sqrt(n))
    assert np.abs(zb).max() > 6.0
