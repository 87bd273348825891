"""Device-side gauge set-up (paper Sec. 1 links): dd_gauge_random against the
seeded host recipe of the inputs, SU(3) properties of the drawn links, and
the upload/download round trip."""

import numpy as np
import pytest

from paper_2211_06902_gb300 import dd4d, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L,eps,seed", [((4, 4, 4, 4), 0.3, 1), ((6, 4, 4, 8), 0.6, 5)])
def test_random_links_match_host_recipe(L, eps, seed):
    ctx = dd4d.Context(L, 0.13)
    ctx.gauge_random(eps, seed)
    U = ctx.gauge_download()
    ref = synth.gauge_field(L, eps, seed)
    assert np.max(np.abs(U - ref)) < 1e-12
    M = U.reshape(-1, 3, 3)
    eye = np.einsum("nij,nkj->nik", M, M.conj())
    assert np.max(np.abs(eye - np.eye(3))) < 1e-13
    assert np.max(np.abs(np.linalg.det(M) - 1.0)) < 1e-12


def test_upload_download_round_trip_and_unit_field():
    L = (4, 4, 4, 6)
    ctx = dd4d.Context(L, 0.13)
    U = synth.gauge_field(L, 0.5, 3)
    ctx.gauge_upload(U)
    assert np.array_equal(ctx.gauge_download(), U)
    ctx.gauge_random(0.0, 9)
    assert np.array_equal(ctx.gauge_download(), synth.unit_gauge(L))


def test_random_links_drive_the_operator():
    """The stencil sees the same field whichever way it was set."""
    L = (4, 4, 4, 4)
    V = 256
    psi = synth.complex_gaussian(4, synth.TAG_RHS, (1, V, 12))
    a, b = dd4d.Context(L, 0.13), dd4d.Context(L, 0.13)
    a.gauge_random(0.4, 11)
    b.gauge_upload(synth.gauge_field(L, 0.4, 11))
    oa, ob = np.zeros_like(psi), np.zeros_like(psi)
    a.apply_D_block("full", None, 1, psi, oa, "f64")
    b.apply_D_block("full", None, 1, psi, ob, "f64")
    assert np.linalg.norm(oa - ob) <= 1e-12 * np.linalg.norm(ob)
