"""Pins of the oracle's block-local molecular dynamics (oracle/md.py) by what the
mathematics fixes, independent of the CUDA path:

* the pseudofermion heat-bath phi = D^dag eta gives S_pf = |eta|^2 exactly;
* the pseudofermion force equals central finite differences of S_pf;
* the link update keeps SU(3) (unitary, det 1) and leaves inactive links alone;
* the leapfrog is time-reversible (forward, flip P, forward, flip P = start);
* its energy violation falls as dt^2 (second order) and H is conserved within it;
* a planted mistake (force of the wrong sign) breaks the dt^2 scaling.
"""

import numpy as np
import pytest
import scipy.linalg

from paper_2211_06902_gb300 import synth
from oracle import md
from oracle.dd import Oracle, field_roots, gell_mann
from oracle.geometry import Decomposition

L = (4, 2, 2, 2)
CORES = [[(0, 0), (2, 2)], [], [], []]
KAPPA = 0.13


@pytest.fixture(scope="module")
def case():
    U = synth.gauge_field(L, 0.4, 3)
    g = Decomposition(L, CORES)
    o = Oracle(U, KAPPA, g)
    u = field_roots(4, 0.5)
    chis = [synth.complex_gaussian(4, synth.TAG_CHI + k, L + (4, 3)) * g.dPi[..., None, None]
            for k in range(len(u))]
    etas = [synth.complex_gaussian(5, synth.TAG_RHS + a, L + (4, 3)) * g.omega_mask[a][..., None, None]
            for a in range(g.nblocks)]
    phis = md.pf_heatbath(o, etas)
    P = synth.momenta(L, 6) * md.active_mask(g)[..., None]
    return U, g, o, u, chis, etas, phis, P


def test_active_links_are_the_core_links(case):
    U, g, o, *_ = case
    act = md.active_mask(g)
    listed = {(x, mu) for a in range(g.nblocks) for x, mu in o.active_links(a)}
    assert {(tuple(int(v) for v in i[:4]), int(i[4])) for i in np.argwhere(act)} == listed
    # one-site time cores: only the spatial links of the core slices
    assert not act[..., 0].any() and act[0, ..., 1:].all() and act[2, ..., 1:].all()


def test_pf_heatbath_gives_the_gaussian_norm(case):
    U, g, o, u, chis, etas, phis, P = case
    s = md.pf_action(o, phis)
    ref = sum(np.vdot(e, e).real for e in etas)
    assert abs(s - ref) < 1e-11 * ref


def test_pf_force_matches_finite_differences(case):
    U, g, o, u, chis, etas, phis, P = case
    F = md.pf_force(o, phis)
    T = gell_mann() / 2
    h = 1e-4
    for (x, mu, t) in [((0, 0, 0, 0), 1, 0), ((2, 1, 0, 1), 3, 5), ((0, 1, 1, 0), 2, 7)]:
        vals = []
        for sgn in (1, -1):
            Up = U.copy()
            Up[x + (mu,)] = scipy.linalg.expm(1j * sgn * h * T[t]) @ U[x + (mu,)]
            vals.append(md.pf_action(Oracle(Up, KAPPA, g), phis))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(F[x + (mu, t)] - fd) < 1e-6 * max(1.0, abs(fd))
    assert np.all(F[~md.active_mask(g)] == 0)


def test_link_update_stays_in_su3_and_only_moves_active_links(case):
    U, g, o, u, chis, etas, phis, P = case
    act = md.active_mask(g)
    U2 = md.link_update(U, P, 0.3, act)
    m = U2[act]
    assert np.abs(np.einsum("nji,njk->nik", m.conj(), m) - np.eye(3)).max() < 1e-13
    assert np.abs(np.linalg.det(m) - 1).max() < 1e-13
    assert np.array_equal(U2[~act], U[~act])
    assert np.abs(m - U[act]).max() > 1e-2


def test_leapfrog_is_reversible(case):
    U, g, o, u, chis, etas, phis, P = case
    U1, P1 = md.leapfrog(U, P, KAPPA, g, u, chis, phis, 0.2, 2)
    U2, P2 = md.leapfrog(U1, -P1, KAPPA, g, u, chis, phis, 0.2, 2)
    assert np.abs(U2 - U).max() < 1e-11
    assert np.abs(-P2 - P).max() < 1e-10


def _dH(case, n, force=None, monkeypatch=None):
    U, g, o, u, chis, etas, phis, P = case
    H0 = md.hamiltonian(U, KAPPA, g, u, chis, phis, P)["H"]
    U1, P1 = md.leapfrog(U, P, KAPPA, g, u, chis, phis, 0.4, n)
    return md.hamiltonian(U1, KAPPA, g, u, chis, phis, P1)["H"] - H0, H0


def test_energy_violation_is_second_order(case):
    d2, H0 = _dH(case, 2)
    d4, _ = _dH(case, 4)
    assert abs(d4) < 1e-2 * H0
    assert 3.0 < d2 / d4 < 5.5, (d2, d4)


def test_planted_wrong_sign_force_breaks_the_scaling(case, monkeypatch):
    real = md.force
    monkeypatch.setattr(md, "force", lambda *a, **k: -real(*a, **k))
    d2, H0 = _dH(case, 2)
    d4, _ = _dH(case, 4)
    assert not (3.0 < d2 / d4 < 5.5 and abs(d4) < 1e-2 * H0), (d2, d4)
