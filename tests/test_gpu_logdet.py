"""GPU dense check of the block factorization of det D (paper Sec. 3, Eq. detD).

Every factor (D, D_Lambda1, each D_Omega0^a and D_Phi1^a, W_1 = 1 - w) is
assembled on the GPU from the library's own operators and factorised by the
library's FP64 LU; each ln|det| is compared with the oracle's dense slogdet
(numpy LAPACK) and the identity must close to 1e-9 (W_1's columns come from
block / frame solves to 1e-13; a column error eps moves ln|det W_1| by at
most ~ n |W_1^-1| eps).
"""

import numpy as np
import pytest

from paper_2211_06902_gb300 import dd4d
from oracle.dd import Oracle
from oracle.geometry import uniform_cores

from gpu_common import make_case

pytestmark = pytest.mark.gpu

CASES = {
    "4^4": ((4,) * 4, uniform_cores((4,) * 4, 1, 1)),
    "6x4^3": ((6, 4, 4, 4), [[(0, 1), (3, 4)]] + [[(0, 0), (2, 2)]] * 3),
}


@pytest.mark.parametrize("name", list(CASES))
def test_logdet_identity_matches_oracle(name):
    L, cores = CASES[name]
    U, ctx, info, geo = make_case(L, 0.13, 0.3, 1, cores)
    rep = ctx.logdet_check(dd4d.params(1e-13, maxiter=5000))
    assert abs(rep["residual"]) < 1e-9, rep
    f = Oracle(U, 0.13, geo).logdet_factors()
    assert abs(rep["logabs_D"] - f["D"][1]) < 1e-9
    assert abs(rep["logabs_Lambda1"] - f["Lambda1"][1]) < 1e-9
    assert np.max(np.abs(rep["logabs_omega"] - np.array([x[1] for x in f["Omega"]]))) < 1e-9
    assert np.max(np.abs(rep["logabs_phi"] - np.array([x[1] for x in f["Phi"]]))) < 1e-9
    assert abs(rep["logabs_W1"] - f["W1"][1]) < 1e-8
    # det D is real (gamma_5-hermiticity): phase 0 or pi, and both sides agree
    assert min(abs(rep["phase_D"]), abs(abs(rep["phase_D"]) - np.pi)) < 1e-9
    d = np.remainder(rep["phase_D"] - rep["phase_rhs"] + np.pi, 2 * np.pi) - np.pi
    assert abs(d) < 1e-8


def test_logdet_rejects_large_lattice():
    L = (8, 8, 8, 8)
    U, ctx, info, geo = make_case(L, 0.13, 0.3, 1, uniform_cores(L, 3, 1))
    with pytest.raises(dd4d.DDError):
        ctx.logdet_check()
