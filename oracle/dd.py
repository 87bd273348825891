"""Block solves, the operator w, the multi-boson action and log-det factors.

Test infrastructure only (see the package docstring).  FP64 throughout.

Operator w (Sec. 3, Eqs. Wz and offdiagW1; reading of the garbled hopping
block): for chi on dPi = dLambda0 u dPi1,

    (w chi)_{dLambda0^a} = - P_{dLambda0^a} D_{Omega0^a}^{-1} D_{Omega0^a, ext(Omega0^a)} chi
    (w chi)_{dPi1}       = - P_{dPi1} D_{Lambda1}^{-1} D_{Lambda1, dLambda0} chi_{dLambda0}

and W_1 = 1 - w on dPi, W_u = u - w.  The first line is the Dirichlet
(Poisson-kernel) extension of chi into the framed block; it contains the
paper's upper-right block P D_Omega^-1 D_{Phi, dOmega*} chi_{dPi1} and
completes the upper-left block; the second line is the paper's lower-left
block D^_{dPi1}^{-1} D^_{dPi1, dLambda0}.  The reading is pinned by the
determinant identity Eq. (detD) and by the Green's-function identity (tests).

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

    # -- w and W_1 (Eqs. Wz, offdiagW1) ---------------------------------
    def apply_w(self, chi):
        """w chi for a field chi supported on dPi; result supported on dPi."""
        g = self.g
        out = np.zeros_like(chi)
        for a in range(g.nblocks):
            ext = chi * g.ext_mask[a][..., None, None]
            src = g.omega_mask[a][..., None, None] * self.D(ext)     # D_{Omega, ext} chi
            psi = self.omega_solver(a).solve_field(src)
            bm = g.B_mask[a]
            out[bm] = -psi[bm]
        ext = chi * g.B[..., None, None]
        src = g.Lambda1[..., None, None] * self.D(ext)                # D_{Lambda1, dLambda0} chi
        y = self.frame_solver().solve_field(src)
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

    # -- dense forms for the determinant identity (small lattices) ----------
    def w_matrix(self):
        """Dense matrix of w on dPi (sites in increasing global order)."""
        g = self.g
        V = int(np.prod(g.L))
        dpi = g.sites(g.dPi)
        pos = np.full(V, -1, dtype=np.int64)
        pos[dpi] = np.arange(len(dpi))
        n = 12 * len(dpi)
        W = np.zeros((n, n), dtype=np.complex128)

        def comp_index(sites):
            return (12 * pos[sites][:, None] + np.arange(12)[None, :]).ravel()

        for a in range(g.nblocks):
            om = g.sites(g.omega_mask[a])
            ex = g.sites(g.ext_mask[a])
            rhs = dirac_block(self.U, self.kappa, om, ex, self.time_bc, self.csw).toarray()
            G = self.omega_solver(a).lu.solve(rhs)
            opos = np.full(V, -1, dtype=np.int64)
            opos[om] = np.arange(len(om))
            bs = g.sites(g.B_mask[a])
            rows_in_om = (12 * opos[bs][:, None] + np.arange(12)[None, :]).ravel()
            W[np.ix_(comp_index(bs), comp_index(ex))] = -G[rows_in_om]
        l1 = g.sites(g.Lambda1)
        bsites = g.sites(g.B)
        rhs = dirac_block(self.U, self.kappa, l1, bsites, self.time_bc, self.csw).toarray()
        G = self.frame_solver().lu.solve(rhs)
        lpos = np.full(V, -1, dtype=np.int64)
        lpos[l1] = np.arange(len(l1))
        cs = g.sites(g.C)
        rows_in_l1 = (12 * lpos[cs][:, None] + np.arange(12)[None, :]).ravel()
        W[np.ix_(comp_index(cs), comp_index(bsites))] = -G[rows_in_l1]
        return W

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
        (Eq. localMB): with y_k = D_Omega^{-1} D_{Omega,ext} chi_k and
        r_k = P_{dLambda0^a}(u_k chi_k + y_k), S^a = sum_k |r_k|^2 and
        dy = -D_Omega^{-1} dD y, so dS = -2 Re sum_k <z_k, dD y_k> with
        z_k = (D_Omega^dag)^{-1} r_k.  dD has the two entries of the link in
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
        for a in range(g.nblocks):
            links = self.active_links(a)
            if not links:
                continue
            om = self.omega_solver(a)
            ext = g.ext_mask[a][..., None, None]
            pairs = []
            for uk, chi in zip(u, chis):
                y = om.solve_field(g.omega_mask[a][..., None, None] * self.D(chi * ext))
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
