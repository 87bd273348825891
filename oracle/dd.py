"""Block solves, the operator w, the multi-boson action and log-det factors.

Test infrastructure only (see the package docstring).  FP64 throughout.

Operator w = 1 - W_1 (Sec. 3, Eqs. Wz and offdiagW1): W_1 is the matrix the
paper prints, diag(D^d, D^_{dPi1})^{-1} times the block matrix of the second
Schur decomposition (D^d + D^h, D^_{dL0,dPi1}; D^_{dPi1,dL0}, D^_{dPi1}),
with the hopping block D^h in its printed symmetrised form.  Two forms:
``w1_dense_blocks`` assembles every block densely (small lattices) and
``apply_w`` applies the same blocks to a vector with block, frame-piece and
frame solves.  The readings taken where the print is incomplete are listed at
the W_1 section below.

Multi-boson action (Sec. 4, Eqs. MBaction, localMB, globalMB) with roots
u_k = 1 - z_k:
    S   = sum_k |W_{u_k} chi_k|^2 = sum_a S^a + S^r,
    S^a = sum_k |P_{dLambda0^a} (u_k - w) chi_k|^2,
    S^r = sum_k |P_{dPi1} (u_k - w) chi_k|^2.
"""

import math

import numpy as np
import scipy.sparse.linalg as spla

from .lattice import apply_D, dirac_block, dirac_matrix, gammas


class DomainSolver:
    """Solves D_X x = b for one site set X.

    Vectors are solved with the BiCGstab routine below to a relative residual
    of 1e-13 (checked on return); the sparse LU (exact up to rounding) is built
    only on request, for the dense matrices of small lattices.
    """

    TOL = 1e-13

    def __init__(self, U, kappa, mask, time_bc=-1, csw=0.0):
        self.L = U.shape[:4]
        self.sites = np.flatnonzero(mask.ravel())
        self.M = dirac_matrix(U, kappa, self.sites, time_bc, csw)
        self._lu = None

    @property
    def lu(self):
        if self._lu is None:
            self._lu = spla.splu(self.M.tocsc(), permc_spec="MMD_AT_PLUS_A")
        return self._lu

    def solve_vec(self, b):
        """b: vector of length 12*|X| (site-major, 12 components per site)."""
        x, relres = bicgstab(lambda v: self.M @ v, b, self.TOL)
        if not relres <= 10 * self.TOL:
            raise RuntimeError("oracle solve did not converge: %g" % relres)
        return x

    def solve_field(self, b):
        """b: field [L0..L3,4,3] supported on X; returns D_X^{-1} b as a field."""
        V = int(np.prod(self.L))
        x = self.solve_vec(b.reshape(V, 12)[self.sites].ravel())
        out = np.zeros((V, 12), dtype=np.complex128)
        out[self.sites] = x.reshape(-1, 12)
        return out.reshape(b.shape)

    def solve_adjoint_field(self, b):
        """(D_X^dag)^{-1} b for a field supported on X (BiCGstab on the conjugate
        transpose of the assembled matrix)."""
        V = int(np.prod(self.L))
        MH = self.M.conj().T.tocsr()
        x, relres = bicgstab(lambda v: MH @ v, b.reshape(V, 12)[self.sites].ravel(), self.TOL)
        if not relres <= 10 * self.TOL:
            raise RuntimeError("oracle adjoint solve did not converge: %g" % relres)
        out = np.zeros((V, 12), dtype=np.complex128)
        out[self.sites] = x.reshape(-1, 12)
        return out.reshape(b.shape)


def bicgstab(matvec, b, tol=1e-13, maxiter=100000):
    """Textbook BiCGstab (van der Vorst 1992) for large sets X; returns (x, relres)."""
    x = np.zeros_like(b)
    r = b.copy()
    rhat = b.copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0:
        return x, 0.0
    rho = alpha = omega = 1.0 + 0j
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    for _ in range(maxiter):
        rho_new = np.vdot(rhat, r)
        beta = (rho_new / rho) * (alpha / omega)
        rho = rho_new
        p = r + beta * (p - omega * v)
        v = matvec(p)
        alpha = rho / np.vdot(rhat, v)
        s = r - alpha * v
        t = matvec(s)
        omega = np.vdot(t, s) / np.vdot(t, t)
        x = x + alpha * p + omega * s
        r = s - omega * t
        if np.linalg.norm(r) <= tol * bnorm:
            break
    true = np.linalg.norm(b - matvec(x)) / bnorm
    return x, true


class Oracle:
    """D, the decomposition and the solvers for one gauge field."""

    def __init__(self, U, kappa, geom, time_bc=-1, csw=0.0):
        self.U = U
        self.kappa = kappa
        self.g = geom
        self.time_bc = time_bc
        self.csw = csw
        self._solvers = {}

    def D(self, psi):
        return apply_D(self.U, psi, self.kappa, self.time_bc, self.csw)

    def solver(self, key, mask):
        if key not in self._solvers:
            self._solvers[key] = DomainSolver(self.U, self.kappa, mask, self.time_bc, self.csw)
        return self._solvers[key]

    def omega_solver(self, a):
        return self.solver(("omega", a), self.g.omega_mask[a])

    def phi_solver(self, a):
        return self.solver(("phi", a), self.g.phi_mask[a])

    def frame_solver(self):
        return self.solver(("Lambda1",), self.g.Lambda1)

    # -- W_1 (Sec. 3, Eqs. Wz and offdiagW1) ------------------------------
    #
    # W_1 = diag(D^d, D^_{dPi1})^{-1} M on dPi = dLambda0 u dPi1 with the blocks
    # the paper prints (Sec. 3), X* = dOmega0^{a*} the exterior boundary of
    # Omega0^a inside dPi1 and E = Lambda1bar = Lambda1 minus dPi1:
    #
    #   D^d_a       = D_{dL0a} - D_{dL0a,L0bar_a} D_{L0bar_a}^-1 D_{L0bar_a,dL0a}
    #                          - D_{dL0a,Phi_a} D_{Phi_a}^-1 D_{Phi_a,dL0a}
    #   D^h_{a,b}   = -1/2 D_{dL0a,Phi_a} [ D_{Phi_a}^-1 - D_{Phi_a}^-1 D_{Phi_a,X*a} D_{Phi_b}^-1
    #                   + D_{Phi_b}^-1 - D_{Phi_a}^-1 D_{X*b,Phi_b} D_{Phi_b}^-1 ] D_{Phi_b,dL0b}   (a != b)
    #   [D^d]^-1 D^_{dL0,dPi1} = sum_a P_{dL0a} D_{Omega_a}^-1 D_{Phi_a,X*a}      (Eq. offdiagW1)
    #   D^_{dPi1}   = D_{dPi1} - D_{dPi1,E} D_E^-1 D_{E,dPi1}
    #   D^_{dPi1,dL0} = - sum_b D_{X*b,Phi_b} D_{Phi_b}^-1 D_{Phi_b,dL0b}
    #
    # Readings: a product of two operators on different site sets acts on the
    # sites they share (each D_X^-1 is D_X^-1 P_X, extended by zero off X);
    # D^_{dPi1} eliminates Lambda1bar (the print has D_{Lambda1}^-1 there, which
    # is not a Schur complement); D^_{dPi1,dL0}, which the paper names but does
    # not print, is the elimination of Phi_b seen from dPi1, the gamma_5-adjoint
    # of the printed -D_{dL0a,Phi_a} D_{Phi_a}^-1 D_{Phi_a,X*a} behind Eq.
    # offdiagW1.  Then W_1 = 1 + offdiagonal, w = 1 - W_1, W_u = u - w.

    def _dmat(self, rows, cols=None):
        """Dense D_{X,Y} for ordered site lists (cols None: D_X)."""
        if cols is None:
            return dirac_matrix(self.U, self.kappa, rows, self.time_bc, self.csw).toarray()
        return dirac_block(self.U, self.kappa, rows, cols, self.time_bc, self.csw).toarray()

    @staticmethod
    def _take(sub, full):
        """Component indices (12 per site) of the sites of ``sub`` that lie in
        ``full`` (both in increasing global order), and the matching positions
        in ``sub``."""
        sub = np.asarray(sub, dtype=np.int64)
        full = np.asarray(full, dtype=np.int64)
        j = np.searchsorted(full, sub)
        hit = (j < len(full)) & (full[np.minimum(j, len(full) - 1)] == sub) if len(full) else \
            np.zeros(len(sub), dtype=bool)
        i_sub = np.flatnonzero(hit)
        i_full = j[i_sub]
        c = np.arange(12)
        return (12 * i_full[:, None] + c).ravel(), (12 * i_sub[:, None] + c).ravel()

    def w1_dense_blocks(self):
        """Dense W_1 on dPi (sites in increasing global order) assembled from the
        printed blocks listed above, with D^d_a and D^_{dPi1} (small lattices)."""
        g = self.g
        dpi = g.sites(g.dPi)
        n = 12 * len(dpi)
        W1 = np.eye(n, dtype=np.complex128)
        nb = g.nblocks
        S = [g.sites(m) for m in g.B_mask]
        F = [g.sites(m) for m in g.phi_mask]
        X = [g.sites(m) for m in g.ext_star_mask]
        Finv = [np.linalg.inv(self._dmat(F[a])) for a in range(nb)]
        Dd = []
        for a in range(nb):
            bulk = g.sites(g.core_mask[a] & ~g.B_mask[a])
            d = self._dmat(S[a]) - self._dmat(S[a], F[a]) @ Finv[a] @ self._dmat(F[a], S[a])
            if len(bulk):
                d -= self._dmat(S[a], bulk) @ np.linalg.solve(self._dmat(bulk), self._dmat(bulk, S[a]))
            Dd.append(d)
        rows = [self._take(S[a], dpi)[0] for a in range(nb)]

        def fa_from(vec_sites, vec, fa):
            """Entries of ``vec`` (rows on vec_sites) at the sites of fa, in fa's order."""
            out = np.zeros((12 * len(fa), vec.shape[1]), dtype=np.complex128)
            i_vec, i_fa = self._take(fa, vec_sites)
            out[i_fa] = vec[i_vec]
            return out

        D_SF = [self._dmat(S[a], F[a]) for a in range(nb)]            # D_{dL0a, Phi_a}
        D_FX = [self._dmat(F[a], X[a]) if len(X[a]) else None for a in range(nb)]
        for b in range(nb):
            Xb = self._dmat(F[b], S[b])                     # D_{Phi_b, dL0b}
            Yb = Finv[b] @ Xb                               # D_{Phi_b}^-1 D_{Phi_b, dL0b}
            Zb = self._dmat(X[b], F[b]) @ Yb if len(X[b]) else None   # D_{X*b, Phi_b} (...)
            for a in range(nb):
                if a == b:
                    continue
                # the three terms of the bracket that start with D_{Phi_a}^-1, then the one that does not
                under = fa_from(F[b], Xb, F[a])
                if D_FX[a] is not None:
                    under -= D_FX[a] @ fa_from(F[b], Yb, X[a])
                if Zb is not None:
                    under -= fa_from(X[b], Zb, F[a])
                bracket = Finv[a] @ under + fa_from(F[b], Yb, F[a])
                h = -0.5 * D_SF[a] @ bracket
                W1[np.ix_(rows[a], rows[b])] += np.linalg.solve(Dd[a], h)
        # upper-right block (Eq. offdiagW1), printed as P D_Omega^-1 D_{Phi, X*}
        cs = g.sites(g.C)
        if len(cs):
            rows_c = self._take(cs, dpi)[0]
            for a in range(nb):
                if not len(X[a]):
                    continue
                om = g.sites(g.omega_mask[a])
                G = np.linalg.inv(self._dmat(om))
                i_om_f, _ = self._take(F[a], om)
                i_om_b, _ = self._take(S[a], om)
                blk = G[np.ix_(i_om_b, i_om_f)] @ self._dmat(F[a], X[a])
                W1[np.ix_(rows[a], self._take(X[a], dpi)[0])] += blk
            # lower-left block D^_{dPi1}^-1 D^_{dPi1, dL0}
            es = g.sites(g.E)
            Shat = self._dmat(cs)
            if len(es):
                Shat = Shat - self._dmat(cs, es) @ np.linalg.solve(self._dmat(es), self._dmat(es, cs))
            DC0 = np.zeros((12 * len(cs), 12 * len(dpi)), dtype=np.complex128)
            for b in range(nb):
                if not len(X[b]):
                    continue
                Zb = self._dmat(X[b], F[b]) @ Finv[b] @ self._dmat(F[b], S[b])
                i_c, _ = self._take(X[b], cs)
                DC0[np.ix_(i_c, rows[b])] -= Zb
            W1[rows_c] += np.linalg.solve(Shat, DC0)
        else:
            Shat = np.zeros((0, 0), dtype=np.complex128)
        return W1, Dd, Shat

    def w_matrix(self):
        """Dense matrix of w = 1 - W_1 on dPi (sites in increasing global order)."""
        W1, _, _ = self.w1_dense_blocks()
        return np.eye(len(W1)) - W1

    def _masked(self, mask, f):
        return mask[..., None, None] * f

    def _D(self, rows, cols, f):
        """D_{X,Y} f = P_X D P_Y f for boolean masks X, Y."""
        return self._masked(rows, self.D(self._masked(cols, f)))

    def block_sources(self, chi):
        """Per block a the source s_a of the Omega0^a solve in the first row of
        W_1 (Eqs. Wz, offdiagW1), and the source v of the dPi1 row:

            (W_1 chi)_{dL0a} = chi_{dL0a} + P_{dL0a} D_{Omega_a}^-1 s_a,
            s_a = sum_{b != a} D^h_{a,b} chi_{dL0b} + D_{Phi_a, X*a} chi_{dPi1},
            (W_1 chi)_{dPi1} = chi_{dPi1} + P_{dPi1} D_{Lambda1}^-1 v,
            v = D^_{dPi1, dL0} chi_{dL0}.

        [D^d_a]^-1 acting on a field on dL0a is P_{dL0a} D_{Omega_a}^-1 (the
        inverse of a Schur complement is the matching block of the inverse);
        likewise D^_{dPi1}^-1 = P_{dPi1} D_{Lambda1}^-1 on dPi1.  D^h chi is the
        printed bracket; D_{Phi_a}^-1 is applied once per block a to the sum over
        b of the bracket's terms that carry it."""
        g = self.g
        nb = g.nblocks
        F, X, Bm = g.phi_mask, g.ext_star_mask, g.B_mask
        t = [self._D(F[b], Bm[b], chi) for b in range(nb)]          # D_{Phi_b, dL0b} chi
        Y = [self.phi_solver(b).solve_field(t[b]) for b in range(nb)]
        Z = [self._D(X[b], F[b], Y[b]) for b in range(nb)]           # D_{X*b, Phi_b} Y_b
        sources = []
        for a in range(nb):
            inner = np.zeros_like(chi)        # terms of the bracket under D_{Phi_a}^-1
            outer = np.zeros_like(chi)        # the term D_{Phi_b}^-1 (...) without it
            for b in range(nb):
                if b == a:
                    continue
                inner += self._masked(F[a], t[b])                    # D_{Phi_a}^-1 P_{Phi_a} ...
                inner -= self._D(F[a], X[a], Y[b])                   # - D_{Phi_a}^-1 D_{Phi_a,X*a} D_{Phi_b}^-1
                inner -= self._masked(F[a], Z[b])                    # - D_{Phi_a}^-1 D_{X*b,Phi_b} D_{Phi_b}^-1
                outer += self._masked(F[a], Y[b])                    # + D_{Phi_b}^-1 on Phi_a
            bracket = self.phi_solver(a).solve_field(inner) + outer
            h = -0.5 * self._D(Bm[a], F[a], bracket)
            sources.append(h + self._D(F[a], X[a], chi))
        v = -sum(Z)                                                  # D^_{dPi1, dL0} chi
        return sources, self._masked(g.C, v)

    def apply_w(self, chi):
        """w chi = chi - W_1 chi for a field chi supported on dPi (the vector
        form of the blocks above); result supported on dPi."""
        g = self.g
        sources, v = self.block_sources(chi)
        out = np.zeros_like(chi)
        for a in range(g.nblocks):
            psi = self.omega_solver(a).solve_field(self._masked(g.omega_mask[a], sources[a]))
            bm = g.B_mask[a]
            out[bm] = -psi[bm]
        if g.C.any():
            y = self.frame_solver().solve_field(self._masked(g.Lambda1, v))
            out[g.C] = -y[g.C]
        return out

    def apply_W1(self, chi):
        return chi * self.g.dPi[..., None, None] - self.apply_w(chi)

    def multiboson_action(self, u, chis):
        """(S, [S^a], S^r) for roots u[k] and fields chis[k] supported on dPi."""
        g = self.g
        sa = [[] for _ in range(g.nblocks)]
        sr = []
        for uk, chi in zip(u, chis):
            r = uk * chi - self.apply_w(chi)
            for a in range(g.nblocks):
                sa[a].append(float(np.sum(np.abs(r[g.B_mask[a]]) ** 2)))
            sr.append(float(np.sum(np.abs(r[g.C]) ** 2)))
        s_blocks = [math.fsum(v) for v in sa]
        s_r = math.fsum(sr)
        return math.fsum(s_blocks + [s_r]), s_blocks, s_r

    def heatbath(self, u, etas):
        """Multi-boson fields by heat-bath (Sec. 4, after Eq. WW): the weight
        exp(-|W_u chi|^2) is sampled exactly by chi = W_u^{-1} eta with eta a
        complex Gaussian of density exp(-|eta|^2).  Definition written out: a
        dense solve of (u - w) chi = eta on dPi for each root u_k and source
        eta_k (fields on the full lattice, supported on dPi)."""
        g = self.g
        dpi = g.sites(g.dPi)
        W = self.w_matrix()
        n = W.shape[0]
        out = []
        for uk, eta in zip(u, etas):
            e = eta.reshape(-1, 12)[dpi].reshape(-1)
            chi = np.linalg.solve(uk * np.eye(n) - W, e)
            f = np.zeros_like(eta).reshape(-1, 12)
            f[dpi] = chi.reshape(-1, 12)
            out.append(f.reshape(eta.shape))
        return out

    # -- force of the factorized multi-boson action on the active links -----
    def active_links(self, a):
        """Links (x, mu) of block a with both end points in its core Lambda0^a
        (the links a multi-level update of block a changes; Sec. 4: S^r and the
        S^b, b != a, do not depend on them)."""
        g = self.g
        cm = g.core_mask[a]
        out = []
        for mu in range(4):
            nxt = np.roll(cm, -1, axis=mu)                     # x + mu in the core
            for x in np.argwhere(cm & nxt):
                out.append((tuple(int(v) for v in x), mu))
        return out

    def mb_force(self, u, chis):
        """F[x, mu, t] = d S_MB / d eps at U_mu(x) -> exp(i eps T_t) U_mu(x),
        T_t = lambda_t / 2, for the active links of every block (zero elsewhere).

        Only S^a of the link's block depends on it, through D_{Omega0^a}
        (Eq. localMB; the source s_a of ``block_sources`` holds frame links and
        the links from the core boundaries into the frames only): with
        y_k = D_Omega^{-1} s_a(chi_k) and r_k = P_{dLambda0^a}(u_k chi_k + y_k),
        S^a = sum_k |r_k|^2 and dy = -D_Omega^{-1} dD y, so
        dS = -2 Re sum_k <z_k, dD y_k> with z_k = (D_Omega^dag)^{-1} r_k.  dD has the two entries of the link in
        the definition of D: row x, column x+mu: -kappa (1 - gamma_mu) (i T U);
        row x+mu, column x: -kappa (1 + gamma_mu) (-i U^dag T) (times the time
        boundary sign where the link crosses x0 = L0-1 -> 0)."""
        if self.csw:
            raise NotImplementedError("the force of the clover term is not part of this oracle")
        g = self.g
        L = g.L
        gam, _ = gammas()
        one = np.eye(4)
        T = gell_mann() / 2
        F = np.zeros(tuple(L) + (4, 8))
        srcs = [self.block_sources(chi)[0] for chi in chis]
        for a in range(g.nblocks):
            links = self.active_links(a)
            if not links:
                continue
            om = self.omega_solver(a)
            pairs = []
            for uk, chi, s in zip(u, chis, srcs):
                y = om.solve_field(g.omega_mask[a][..., None, None] * s[a])
                r = g.B_mask[a][..., None, None] * (uk * chi + y)
                pairs.append((y, om.solve_adjoint_field(r)))
            for x, mu in links:
                xp = list(x)
                xp[mu] = (xp[mu] + 1) % L[mu]
                xp = tuple(xp)
                bc = self.time_bc if (mu == 0 and x[0] == L[0] - 1) else 1.0
                Uxm = self.U[x + (mu,)]
                for t in range(8):
                    dfwd = -self.kappa * bc * np.kron(one - gam[mu], 1j * T[t] @ Uxm)
                    dbwd = -self.kappa * bc * np.kron(one + gam[mu], -1j * Uxm.conj().T @ T[t])
                    val = 0.0
                    for y, z in pairs:
                        val += np.vdot(z[x].ravel(), dfwd @ y[xp].ravel())
                        val += np.vdot(z[xp].ravel(), dbwd @ y[x].ravel())
                    F[x + (mu, t)] = -2.0 * val.real
        return F

    def logdet_force(self, max_dim=6000):
        """G[x, mu, t] = d ln|det D_{Omega0^a}| / d eps at U_mu(x) -> exp(i eps T_t) U_mu(x)
        for the active links of every block a (zero elsewhere): Re Tr[D_Omega^{-1} dD_Omega],
        with the two entries of dD_Omega as in mb_force and D_Omega^{-1} the dense inverse
        (small blocks only: 12 |Omega0^a| <= max_dim)."""
        if self.csw:
            raise NotImplementedError("the force of the clover term is not part of this oracle")
        g = self.g
        L = g.L
        V = int(np.prod(L))
        gam, _ = gammas()
        one = np.eye(4)
        T = gell_mann() / 2
        G = np.zeros(tuple(L) + (4, 8))
        for a in range(g.nblocks):
            links = self.active_links(a)
            if not links:
                continue
            om = self.omega_solver(a)
            if 12 * len(om.sites) > max_dim:
                raise ValueError("block too large for the dense inverse")
            Minv = np.linalg.inv(om.M.toarray())
            pos = np.full(V, -1, dtype=np.int64)
            pos[om.sites] = np.arange(len(om.sites))

            def blk(r, c):                      # (D_Omega^{-1})_{r, c}, 12 x 12
                i, j = pos[np.ravel_multi_index(r, L)], pos[np.ravel_multi_index(c, L)]
                return Minv[12 * i:12 * i + 12, 12 * j:12 * j + 12]
            for x, mu in links:
                xp = list(x)
                xp[mu] = (xp[mu] + 1) % L[mu]
                xp = tuple(xp)
                bc = self.time_bc if (mu == 0 and x[0] == L[0] - 1) else 1.0
                Uxm = self.U[x + (mu,)]
                g_xpx, g_xxp = blk(xp, x), blk(x, xp)
                for t in range(8):
                    dfwd = -self.kappa * bc * np.kron(one - gam[mu], 1j * T[t] @ Uxm)
                    dbwd = -self.kappa * bc * np.kron(one + gam[mu], -1j * Uxm.conj().T @ T[t])
                    G[x + (mu, t)] = np.trace(g_xpx @ dfwd + g_xxp @ dbwd).real
        return G

    def logdet_force_stochastic(self, etas):
        """Noise estimate of G = d ln|det D_{Omega0^a}| / d eps on the active links
        (Sec. 4, Eq. SFeffN): ln|det D| = Re ln det D and d ln det D = Tr[D^{-1} dD];
        with noise vectors eta_k on Omega0^a of E[eta eta^dag] = 1 (the complex
        Gaussians of the input recipe), Tr[D^{-1} dD] = E[<(D^dag)^{-1} eta, dD eta>],
        so G = (1/n) sum_k Re <z_k, dD eta_k>, z_k = (D_Omega^dag)^{-1} eta_k.
        etas[a][k]: field on the full lattice supported on Omega0^a (noise k of
        block a).  Returns G (zero off the active links) and the per-link sample
        standard deviation of the n terms."""
        if self.csw:
            raise NotImplementedError("the force of the clover term is not part of this oracle")
        g = self.g
        L = g.L
        gam, _ = gammas()
        one = np.eye(4)
        T = gell_mann() / 2
        G = np.zeros(tuple(L) + (4, 8))
        SD = np.zeros(tuple(L) + (4, 8))
        for a in range(g.nblocks):
            links = self.active_links(a)
            if not links:
                continue
            om = self.omega_solver(a)
            pairs = [(eta, om.solve_adjoint_field(eta)) for eta in etas[a]]
            n = len(pairs)
            for x, mu in links:
                xp = list(x)
                xp[mu] = (xp[mu] + 1) % L[mu]
                xp = tuple(xp)
                bc = self.time_bc if (mu == 0 and x[0] == L[0] - 1) else 1.0
                Uxm = self.U[x + (mu,)]
                for t in range(8):
                    dfwd = -self.kappa * bc * np.kron(one - gam[mu], 1j * T[t] @ Uxm)
                    dbwd = -self.kappa * bc * np.kron(one + gam[mu], -1j * Uxm.conj().T @ T[t])
                    terms = []
                    for eta, z in pairs:
                        v = np.vdot(z[x].ravel(), dfwd @ eta[xp].ravel())
                        v += np.vdot(z[xp].ravel(), dbwd @ eta[x].ravel())
                        terms.append(v.real)
                    G[x + (mu, t)] = np.mean(terms)
                    SD[x + (mu, t)] = np.std(terms, ddof=1) if n > 1 else 0.0
        return G, SD

    def effective_force(self, u, chis):
        """Force of the block-local part of the factorized effective action (Sec. 4,
        Eq. SFeffN) on the active links: d/d eps of sum_a [-ln|det D_{Omega0^a}| + sum_k
        S^a_MB]; the other terms (ln det D_{Phi1^a}, ln det D_{Lambda1}, S^r) do not
        depend on the active links."""
        return self.mb_force(u, chis) - self.logdet_force()

    def reweight_apply(self, N, c, eta):
        """M eta with M = 1 - R_{N+1}(W_1) = W_1 P_N(W_1) (Sec. 4, Eq. rw), in the
        paper's product form P_N(z) = c_N prod_{k=1..N} (z - z_k): each factor
        W_1 - z_k = u_k - w, then W_1 = 1 - w, then the constant c_N."""
        y = eta.copy()
        for uk in roots(N, c):
            y = uk * y - self.apply_w(y)
        y = y - self.apply_w(y)
        return pn_leading(N, c) * y

    def reweight_samples(self, N, c, etas):
        """Per source eta (complex Gaussian, density exp(-|eta|^2), on dPi):
        s = |eta|^2 - |M eta|^2.  E[exp(s)] = 1/det(M^dag M) = |W_N|^-2, the
        stochastic estimate of the reweighting factor of Eq. (rw) (reading:
        the paper names the factor but no estimator)."""
        out = []
        for eta in etas:
            m = self.reweight_apply(N, c, eta)
            out.append(float(np.sum(np.abs(eta) ** 2) - np.sum(np.abs(m) ** 2)))
        return np.array(out)

    def logdet_factors(self):
        """slogdet of D, W_1, D_{Lambda1}, D_{Omega0^a}, D_{Phi1^a} (dense LU)."""
        g = self.g
        V = int(np.prod(g.L))
        D = dirac_matrix(self.U, self.kappa, np.arange(V), self.time_bc, self.csw).toarray()
        out = {"D": np.linalg.slogdet(D)}
        del D
        w = self.w_matrix()
        out["W1"] = np.linalg.slogdet(np.eye(w.shape[0]) - w)
        del w
        out["Lambda1"] = np.linalg.slogdet(self.frame_solver().M.toarray())
        out["Omega"] = [np.linalg.slogdet(self.omega_solver(a).M.toarray())
                        for a in range(g.nblocks)]
        out["Phi"] = [np.linalg.slogdet(self.phi_solver(a).M.toarray())
                      for a in range(g.nblocks)]
        return out


def roots(N, c):
    """u_k = 1 - z_k, k = 1..N, of P_N(z) = (1 - R_{N+1}(z))/z (Sec. 4).

    u_k = cos(2 pi k/(N+1)) + i sqrt(1 - c^2) sin(2 pi k/(N+1)).
    """
    k = np.arange(1, N + 1)
    phi = 2.0 * np.pi * k / (N + 1)
    return np.cos(phi) + 1j * math.sqrt(1.0 - c * c) * np.sin(phi)


def field_roots(N, c):
    """The N/2 roots that carry a multi-boson field: k = 1..N/2 (Eq. WW)."""
    if N % 2:
        raise ValueError("N must be even")
    return roots(N, c)[: N // 2]


def gell_mann():
    """The eight Gell-Mann matrices lambda_1..lambda_8, shape [8, 3, 3]."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1], lam[1][1, 0] = -1j, 1j
    lam[2][0, 0], lam[2][1, 1] = 1, -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2], lam[4][2, 0] = -1j, 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2], lam[6][2, 1] = -1j, 1j
    lam[7] = np.diag([1, 1, -2]) / math.sqrt(3)
    return lam


def chebyshev_T(n, x):
    """T_n(x) = cosh(n arccosh x) for x >= 1."""
    return math.cosh(n * math.acosh(x))


def pn_leading(N, c):
    """c_N of P_N(z) = c_N prod_k (z - z_k) (Sec. 4) for the roots above.

    With R_{N+1}(z) = T_{N+1}((1 - z)/c) / T_{N+1}(1/c) (reading of c), the
    leading coefficient of 1 - R_{N+1}(z) = z P_N(z) is
    -2^N (-1/c)^{N+1} / T_{N+1}(1/c) = 2^N / (c^{N+1} T_{N+1}(1/c)) for N even;
    at c = 0, R_{N+1}(z) = (1 - z)^{N+1} and c_N = 1.
    """
    if N % 2:
        raise ValueError("N must be even")
    if c == 0.0:
        return 1.0
    return 2.0 ** N / (c ** (N + 1) * chebyshev_T(N + 1, 1.0 / c))
