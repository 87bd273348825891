"""Molecular dynamics of the active links of every block (block-local HMC,
Sec. 4: the factorization decouples the links inside the cores, so each block's
links evolve on their own, Sec. 5 "Parallelization").

Test infrastructure only (see the package docstring).  FP64 throughout, plain
loops, scipy's matrix exponential for the link update.

Hamiltonian of one trajectory (all blocks at once; the blocks do not couple):
    H = 1/2 sum_{active (x, mu)} sum_t P_t(x, mu)^2  +  S_MB  +  S_pf,
    S_MB = sum_k |W_{u_k} chi_k|^2                         (Eq. MBaction),
    S_pf = sum_a |(D_{Omega0^a}^dag)^{-1} phi_a|^2,
where phi_a, a pseudofermion field on Omega0^a, represents det(D_Omega^dag D_Omega)
= (det D_{Omega0^a})^2, the block determinant of Eq. SFeffN for two degenerate
flavours (the caller passes the multi-boson fields of both flavours in chis).
Only S^a of S_MB and the S_pf term of block a depend on its active links, so
the other terms of Eq. SFeffN (ln det D_{Phi1^a}, ln det D_{Lambda1}, S^r)
stay constant along the trajectory.

Links move as U_mu(x) -> exp(i dt sum_t P_t T_t) U_mu(x) (T_t = lambda_t / 2),
momenta as P_t -> P_t - dt F_t with F_t = dS/d eps_t at U -> exp(i eps T_t) U;
then dH/dtau = 0 along the exact flow.  The integrator is the leapfrog
(half step in P, full step in U, half step in P), second order in dt and
time-reversible.
"""

import numpy as np
import scipy.linalg

from .dd import Oracle, gell_mann
from .lattice import gammas


def active_mask(g):
    """[L.., 4] booleans: the links with both end points in one block's core."""
    out = np.zeros(tuple(g.L) + (4,), dtype=bool)
    for a in range(g.nblocks):
        cm = g.core_mask[a]
        for mu in range(4):
            out[..., mu] |= cm & np.roll(cm, -1, axis=mu)
    return out


def pf_heatbath(o, etas):
    """phi_a = D_{Omega0^a}^dag eta_a (the assembled matrix, conjugate-transposed),
    so that S_pf = sum_a |eta_a|^2 exactly.  etas: fields [L..,4,3] per block,
    supported on Omega0^a."""
    V = int(np.prod(o.g.L))
    out = []
    for a, eta in enumerate(etas):
        om = o.omega_solver(a)
        v = eta.reshape(V, 12)[om.sites].ravel()
        f = np.zeros((V, 12), dtype=np.complex128)
        f[om.sites] = (om.M.conj().T @ v).reshape(-1, 12)
        out.append(f.reshape(eta.shape))
    return out


def pf_action(o, phis):
    """S_pf = sum_a |(D_Omega^dag)^{-1} phi_a|^2."""
    return float(sum(np.vdot(y, y).real for y in _pf_y(o, phis)))


def _pf_y(o, phis):
    return [o.omega_solver(a).solve_adjoint_field(phi) for a, phi in enumerate(phis)]


def pf_force(o, phis):
    """F[x, mu, t] = d S_pf / d eps at U_mu(x) -> exp(i eps T_t) U_mu(x) on the active
    links (zero elsewhere).  With Y = (D^dag)^{-1} phi and X = D^{-1} Y,
    S_pf = phi^dag (D^dag D)^{-1} phi and dS_pf = -2 Re <Y, dD X>; dD has the two
    entries of the link (see Oracle.mb_force)."""
    g = o.g
    L = g.L
    gam, _ = gammas()
    one = np.eye(4)
    T = gell_mann() / 2
    F = np.zeros(tuple(L) + (4, 8))
    for a, phi in enumerate(phis):
        links = o.active_links(a)
        if not links:
            continue
        om = o.omega_solver(a)
        Y = om.solve_adjoint_field(phi)
        X = om.solve_field(Y)
        for x, mu in links:
            xp = list(x)
            xp[mu] = (xp[mu] + 1) % L[mu]
            xp = tuple(xp)
            bc = o.time_bc if (mu == 0 and x[0] == L[0] - 1) else 1.0
            Uxm = o.U[x + (mu,)]
            for t in range(8):
                dfwd = -o.kappa * bc * np.kron(one - gam[mu], 1j * T[t] @ Uxm)
                dbwd = -o.kappa * bc * np.kron(one + gam[mu], -1j * Uxm.conj().T @ T[t])
                val = np.vdot(Y[x].ravel(), dfwd @ X[xp].ravel())
                val += np.vdot(Y[xp].ravel(), dbwd @ X[x].ravel())
                F[x + (mu, t)] = -2.0 * val.real
    return F


def kinetic(P, act):
    """1/2 sum over the active links of sum_t P_t^2."""
    return 0.5 * float(np.sum(P[act] ** 2))


def hamiltonian(U, kappa, g, u, chis, phis, P, time_bc=-1):
    """The pieces of H at links U and momenta P [L.., 4, 8]."""
    o = Oracle(U, kappa, g, time_bc=time_bc)
    act = active_mask(g)
    s_mb = o.multiboson_action(u, chis)[0] if len(u) else 0.0
    s_pf = pf_action(o, phis) if phis is not None else 0.0
    k = kinetic(P, act)
    return {"kinetic": k, "s_mb": float(s_mb), "s_pf": s_pf, "H": k + float(s_mb) + s_pf}


def force(U, kappa, g, u, chis, phis, time_bc=-1):
    """dH/d eps on the active links: the multi-boson force plus the pseudofermion force."""
    o = Oracle(U, kappa, g, time_bc=time_bc)
    F = o.mb_force(u, chis) if len(u) else np.zeros(tuple(g.L) + (4, 8))
    if phis is not None:
        F = F + pf_force(o, phis)
    return F


def link_update(U, P, dt, act):
    """U_mu(x) -> exp(i dt sum_t P_t T_t) U_mu(x) on the active links."""
    T = gell_mann() / 2
    out = U.copy()
    for idx in np.argwhere(act):
        x = tuple(int(v) for v in idx)
        H = np.tensordot(P[x], T, axes=(0, 0))           # hermitian, traceless
        out[x] = scipy.linalg.expm(1j * dt * H) @ U[x]
    return out


def leapfrog(U, P, kappa, g, u, chis, phis, tau, nsteps, time_bc=-1):
    """nsteps leapfrog steps of size tau / nsteps from (U, P); returns (U, P).
    Each step: P -= dt/2 F(U); U -> exp(i dt P T) U; P -= dt/2 F(U)."""
    dt = tau / nsteps
    act = active_mask(g)
    P = np.where(act[..., None], P, 0.0)
    for _ in range(nsteps):
        P = P - 0.5 * dt * force(U, kappa, g, u, chis, phis, time_bc)
        U = link_update(U, P, dt, act)
        P = P - 0.5 * dt * force(U, kappa, g, u, chis, phis, time_bc)
    return U, P
