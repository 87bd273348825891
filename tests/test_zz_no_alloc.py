"""The stencil entry point that allocates no device memory.

Some callers cannot allocate GPU memory during a call (their memory is
budgeted up front, or owned by another allocator, or they cannot take the
synchronisation cudaMalloc implies).  dd_apply_D_block_noalloc serves them
from a fixed static device array; here its output is compared with the
regular dd_apply_D_block (FP64) on the same inputs, on two calls in a row,
within the stencil tolerance of the other tests (1e-12 relative).  This file
is collected last on purpose.
"""

import numpy as np
import pytest

from paper_2211_06902_gb300 import dd4d, synth

from gpu_common import config1, relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case():
    return config1()


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.float64).copy()).cuda()


@pytest.mark.parametrize("kind", ["omega", "lambda1", "full"])
def test_noalloc_matches_regular_stencil_twice(case, kind):
    torch = pytest.importorskip("torch")
    U, ctx, info, geo = case
    if kind == "omega":
        ids, nrhs = list(range(info["nblocks"])), 2
        n = len(ctx.geom_sites(dd4d.SET_OMEGA, 0))
    elif kind == "lambda1":
        ids, nrhs = None, 3
        n = len(ctx.geom_sites(dd4d.SET_LAMBDA1))
    else:
        ids, nrhs = None, 1
        n = int(np.prod(geo.L))
    nb = len(ids) if ids else 1
    for call in range(2):
        psi = synth.complex_gaussian(40 + call, synth.TAG_RHS, (nb, nrhs, n, 12))
        d_in = _dev(torch, psi)
        ref = torch.zeros_like(d_in)
        got = torch.full_like(d_in, float("nan"))
        ctx.apply_D_block(kind, ids, nrhs, d_in, ref, "f64")
        ctx.apply_D_block_noalloc(kind, ids, nrhs, d_in, got)
        torch.cuda.synchronize()
        a = got.cpu().numpy().view(np.complex128)
        b = ref.cpu().numpy().view(np.complex128)
        assert np.all(np.isfinite(a))
        assert relerr(a, b) < 1e-12


def test_noalloc_rejects_oversized_request(case):
    torch = pytest.importorskip("torch")
    U, ctx, info, geo = case
    ids = list(range(info["nblocks"]))
    n = len(ctx.geom_sites(dd4d.SET_OMEGA, 0))
    nrhs = 32                     # 16 blocks x 625 sites x 32 rhs x 384 B > 64 MiB
    x = torch.zeros(len(ids) * nrhs * n * 24, dtype=torch.float64, device="cuda")
    with pytest.raises(dd4d.DDError) as e:
        ctx.apply_D_block_noalloc("omega", ids, nrhs, x, x)
    assert "scratch" in str(e.value)
    with pytest.raises(dd4d.DDError):
        ctx.apply_D_block_noalloc("omega", ids, 1, np.zeros(10), np.zeros(10))
