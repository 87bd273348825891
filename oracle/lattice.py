"""Lattice, gamma matrices and the Wilson-Dirac operator (oracle, FP64, CPU).

Test infrastructure only (see the package docstring).

Conventions (the paper only asks for a local D, Sec. 3; these readings are
fixed so that raw vectors can be compared):

* Sites x = (x0, x1, x2, x3), x0 is time; fields have layout
  [L0, L1, L2, L3, 4 (spin), 3 (colour)]; global site index is lexicographic
  with x3 fastest; the 12 internal components are ordered spin-major
  (index = 3*spin + colour).
* Boundary conditions: periodic in x1..x3; in x0 the hop across the
  x0 = L0-1 <-> 0 boundary is multiplied by ``time_bc`` (-1: antiperiodic).
  The stored links themselves are not modified.
* Chiral basis: gamma_0 = [[0,-1],[-1,0]], gamma_k = [[0,-i s_k],[i s_k,0]]
  (2x2 blocks, s_k Pauli), gamma_5 = gamma_0 gamma_1 gamma_2 gamma_3
  = diag(1,1,-1,-1).
* Wilson operator in kappa normalisation (r = 1):
  (D psi)(x) = A(x) psi(x) - kappa sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
                                           + (1 + gamma_mu) U_mu(x-mu)^+ psi(x-mu) ]
  with A(x) = 1 without the clover term (c_sw = 0).  With it (the site-local
  12x12 term the paper allows in D, Sec. 1) A(x) = 1 + i kappa c_sw
  sum_{mu<nu} sigma_mu_nu F_mu_nu(x), sigma_mu_nu = (i/2)[gamma_mu, gamma_nu],
  F_mu_nu = (Q_mu_nu - Q_mu_nu^+)/8 and Q_mu_nu the sum of the four plaquettes
  of the mu-nu plane that start and end at x (the clover), all traversed mu
  first; the links enter the clover unmodified (the time boundary sign belongs
  to the fermion hops).
* Restriction to a site set X (Sec. 3 notation D_X, D_{X,Y}):
  D_X = P_X D P_X and D_{X,Y} = P_X D P_Y, i.e. hops leaving X are dropped
  (Dirichlet boundary).
"""

import numpy as np
import scipy.sparse as sp


def pauli():
    s1 = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    s2 = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
    s3 = np.array([[1, 0], [0, -1]], dtype=np.complex128)
    return s1, s2, s3


def gammas():
    """gamma_0..gamma_3 (shape [4,4,4]) and gamma_5 in the chiral basis."""
    z = np.zeros((2, 2), dtype=np.complex128)
    one = np.eye(2, dtype=np.complex128)
    g = np.zeros((4, 4, 4), dtype=np.complex128)
    g[0] = np.block([[z, -one], [-one, z]])
    for k, s in enumerate(pauli()):
        g[k + 1] = np.block([[z, -1j * s], [1j * s, z]])
    g5 = g[0] @ g[1] @ g[2] @ g[3]
    return g, g5


def site_index(L, x):
    """Lexicographic global index (x3 fastest) of coordinates x (arrays ok)."""
    return ((x[0] * L[1] + x[1]) * L[2] + x[2]) * L[3] + x[3]


def sigma_munu():
    """sigma_mu_nu = (i/2)[gamma_mu, gamma_nu], shape [4, 4, 4, 4]."""
    g, _ = gammas()
    s = np.zeros((4, 4, 4, 4), dtype=np.complex128)
    for mu in range(4):
        for nu in range(4):
            s[mu, nu] = 0.5j * (g[mu] @ g[nu] - g[nu] @ g[mu])
    return s


def _dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


def clover_leaves(U, mu, nu):
    """Q_mu_nu(x): the four plaquettes of the mu-nu plane at x, mu first."""
    def sh(f, d, step):                 # f(x + step * e_d)
        return np.roll(f, -step, axis=d)
    Um, Un = U[..., mu, :, :], U[..., nu, :, :]
    # x -> x+mu -> x+mu+nu -> x+nu -> x
    q = Um @ sh(Un, mu, 1) @ _dag(sh(Um, nu, 1)) @ _dag(Un)
    # x -> x+nu -> x+nu-mu -> x-mu -> x
    q = q + Un @ _dag(sh(sh(Um, mu, -1), nu, 1)) @ _dag(sh(Un, mu, -1)) @ sh(Um, mu, -1)
    # x -> x-mu -> x-mu-nu -> x-nu -> x
    q = q + (_dag(sh(Um, mu, -1)) @ _dag(sh(sh(Un, mu, -1), nu, -1))
             @ sh(sh(Um, mu, -1), nu, -1) @ sh(Un, nu, -1))
    # x -> x-nu -> x-nu+mu -> x+mu -> x
    q = q + _dag(sh(Un, nu, -1)) @ sh(Um, nu, -1) @ sh(sh(Un, nu, -1), mu, 1) @ _dag(Um)
    return q


def field_strength(U, mu, nu):
    """F_mu_nu(x) = (Q_mu_nu - Q_mu_nu^+) / 8 (anti-Hermitian 3x3 per site)."""
    q = clover_leaves(U, mu, nu)
    return (q - _dag(q)) / 8.0


def clover_term(U, kappa, csw):
    """A(x) = 1 + i kappa c_sw sum_{mu<nu} sigma_mu_nu (x) F_mu_nu(x), shape L + (12, 12)."""
    L = U.shape[:4]
    sig = sigma_munu()
    A = np.zeros(tuple(L) + (12, 12), dtype=np.complex128)
    A[...] = np.eye(12)
    for mu in range(4):
        for nu in range(mu + 1, 4):
            F = field_strength(U, mu, nu)
            A += 1j * kappa * csw * np.einsum("st,...ab->...satb", sig[mu, nu], F).reshape(
                tuple(L) + (12, 12))
    return A


def apply_D(U, psi, kappa, time_bc=-1, csw=0.0):
    """Wilson-Dirac operator on the full lattice, psi of shape [L0..L3,4,3]."""
    g, _ = gammas()
    L = psi.shape[:4]
    one = np.eye(4)
    if csw:
        A = clover_term(U, kappa, csw)
        out = np.einsum("...ij,...j->...i", A, psi.reshape(tuple(L) + (12,))).reshape(psi.shape)
    else:
        out = psi.copy()
    for mu in range(4):
        Umu = U[..., mu, :, :]
        fwd = np.roll(psi, -1, axis=mu)            # psi(x + mu)
        bwd = np.roll(psi, +1, axis=mu)            # psi(x - mu)
        Uback = np.roll(Umu, +1, axis=mu)          # U_mu(x - mu)
        if mu == 0:
            fwd[L[0] - 1] *= time_bc               # hop L0-1 -> 0
            bwd[0] *= time_bc                      # hop 0 -> L0-1
        uf = np.einsum("...ab,...sb->...sa", Umu, fwd)
        ub = np.einsum("...ba,...sb->...sa", np.conj(Uback), bwd)
        out -= kappa * (np.einsum("st,...tc->...sc", one - g[mu], uf)
                        + np.einsum("st,...tc->...sc", one + g[mu], ub))
    return out


def apply_D_restricted(U, psi, kappa, mask, time_bc=-1, csw=0.0):
    """D_X psi = P_X D P_X psi with X given by a boolean mask of shape L."""
    m = mask[..., None, None]
    return m * apply_D(U, m * psi, kappa, time_bc, csw)


def dirac_matrix(U, kappa, sites, time_bc=-1, csw=0.0):
    """Sparse matrix of D_X for the ordered list ``sites`` of global indices.

    Row/column (i, a) stands for site sites[i] and internal component a
    (spin-major).  Entries follow the definition of D above: A(x) on the
    diagonal (identity at c_sw = 0), -kappa (1 -/+ gamma_mu) (x) U for hops
    whose both ends lie in X.
    """
    g, _ = gammas()
    L = U.shape[:4]
    V = int(np.prod(L))
    sites = np.asarray(sites, dtype=np.int64)
    n = len(sites)
    pos = np.full(V, -1, dtype=np.int64)
    pos[sites] = np.arange(n)
    x = np.array(np.unravel_index(sites, L))
    Uf = U.reshape(V, 4, 3, 3)
    comp = np.arange(12)
    if csw:
        A = clover_term(U, kappa, csw).reshape(V, 12, 12)[sites]
        r = 12 * np.arange(n)[:, None, None] + comp[None, :, None]
        c = 12 * np.arange(n)[:, None, None] + comp[None, None, :]
        rows = [np.broadcast_to(r, A.shape).ravel()]
        cols = [np.broadcast_to(c, A.shape).ravel()]
        vals = [A.ravel()]
    else:
        rows = [np.arange(12 * n)]
        cols = [np.arange(12 * n)]
        vals = [np.ones(12 * n, dtype=np.complex128)]
    one = np.eye(4)
    for mu in range(4):
        for step in (+1, -1):
            y = x.copy()
            y[mu] = (x[mu] + step) % L[mu]
            yi = site_index(L, y)
            j = pos[yi]
            keep = j >= 0
            if not np.any(keep):
                continue
            phase = np.ones(n)
            if mu == 0:
                cross = (x[0] == L[0] - 1) if step == 1 else (x[0] == 0)
                phase[cross] = time_bc
            if step == 1:
                spin = one - g[mu]
                link = Uf[sites, mu]                       # U_mu(x)
            else:
                spin = one + g[mu]
                link = np.conj(np.swapaxes(Uf[yi, mu], 1, 2))  # U_mu(x-mu)^+
            blk = np.einsum("st,mab->msatb", spin, link[keep]).reshape(-1, 12, 12)
            blk = -kappa * phase[keep][:, None, None] * blk
            i_k = np.nonzero(keep)[0]
            r = 12 * i_k[:, None, None] + comp[None, :, None]
            c = 12 * j[keep][:, None, None] + comp[None, None, :]
            rows.append(np.broadcast_to(r, blk.shape).ravel())
            cols.append(np.broadcast_to(c, blk.shape).ravel())
            vals.append(blk.ravel())
    M = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(12 * n, 12 * n)).tocsr()
    M.sum_duplicates()
    M.eliminate_zeros()
    return M


def dirac_block(U, kappa, row_sites, col_sites, time_bc=-1, csw=0.0):
    """Sparse matrix of D_{X,Y} = P_X D P_Y for disjoint ordered site lists X, Y
    (hops only: the site-local term lies on the diagonal, outside D_{X,Y})."""
    row_sites = np.asarray(row_sites, dtype=np.int64)
    col_sites = np.asarray(col_sites, dtype=np.int64)
    both = np.concatenate([row_sites, col_sites])
    M = dirac_matrix(U, kappa, both, time_bc, csw)
    nr = 12 * len(row_sites)
    return M[:nr, nr:]


def gauge_transform_links(U, g):
    """U^g_mu(x) = g(x) U_mu(x) g(x+mu)^+ (the time boundary phase is not a link)."""
    out = np.empty_like(U)
    for mu in range(4):
        gp = np.roll(g, -1, axis=mu)
        out[..., mu, :, :] = g @ U[..., mu, :, :] @ np.conj(np.swapaxes(gp, -1, -2))
    return out
