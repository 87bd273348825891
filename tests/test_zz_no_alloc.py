"""The stencil entry point that allocates no device memory.

Some callers cannot allocate GPU memory during a call (their memory is
budgeted up front, or owned by another allocator, or they cannot take the
synchronisation cudaMalloc implies).  dd_apply_D_block_noalloc serves them
from a fixed static device array; here its output is compared with the
regular dd_apply_D_block (FP64) and with the oracle's restricted operator on
the same inputs, on two calls in a row, within the stencil tolerance of the
other tests (1e-12 relative), on every domain kind and on a side stream.
This file is collected last on purpose.
"""

import numpy as np
import pytest

from paper_2211_06902_gb300 import dd4d, synth
from oracle.lattice import apply_D_restricted

from gpu_common import config1, from_field, relerr, to_field

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case():
    return config1()


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.float64).copy()).cuda()


@pytest.mark.parametrize("kind,side_stream", [("omega", False), ("phi", False), ("lambda1", False),
                                              ("full", False), ("omega", True)])
def test_noalloc_matches_regular_stencil_twice(case, kind, side_stream):
    torch = pytest.importorskip("torch")
    U, ctx, info, geo = case
    L = geo.L
    if kind in ("omega", "phi"):
        ids, nrhs = list(range(info["nblocks"])), 2
        which = dd4d.SET_OMEGA if kind == "omega" else dd4d.SET_PHI
        sites = [ctx.geom_sites(which, b) for b in ids]
        masks = [(geo.omega_mask if kind == "omega" else geo.phi_mask)[b] for b in ids]
    elif kind == "lambda1":
        ids, nrhs = None, 3
        sites, masks = [ctx.geom_sites(dd4d.SET_LAMBDA1)], [geo.Lambda1]
    else:
        ids, nrhs = None, 1
        sites, masks = [np.arange(int(np.prod(L)))], [np.ones(L, dtype=bool)]
    nb, n = len(sites), len(sites[0])
    stream = torch.cuda.Stream() if side_stream else None
    for call in range(2):
        psi = synth.complex_gaussian(40 + call, synth.TAG_RHS, (nb, nrhs, n, 12))
        d_in = _dev(torch, psi)
        ref = torch.zeros_like(d_in)
        got = torch.full_like(d_in, float("nan"))
        ctx.apply_D_block(kind, ids, nrhs, d_in, ref, "f64")
        torch.cuda.synchronize()
        if stream is not None:
            with torch.cuda.stream(stream):
                ctx.apply_D_block_noalloc(kind, ids, nrhs, d_in, got, stream=stream)
            stream.synchronize()
        else:
            ctx.apply_D_block_noalloc(kind, ids, nrhs, d_in, got)
        torch.cuda.synchronize()
        a = got.cpu().numpy().view(np.complex128)
        b = ref.cpu().numpy().view(np.complex128)
        assert np.all(np.isfinite(a))
        assert relerr(a, b) < 1e-12
        # the oracle's D_X on the first and the last domain of the call
        for k in (0, nb - 1):
            for r in (0, nrhs - 1):
                f = to_field(L, sites[k], psi[k, r])
                want = from_field(L, sites[k], apply_D_restricted(U, f, 0.13, masks[k]))
                assert relerr(a[k, r], want) < 1e-12


def test_noalloc_later_calls_take_no_device_memory(case):
    """Once the first call has set the array up, a call leaves the device's free
    memory unchanged."""
    torch = pytest.importorskip("torch")
    U, ctx, info, geo = case
    ids = list(range(info["nblocks"]))
    n = len(ctx.geom_sites(dd4d.SET_OMEGA, 0))
    d_in = _dev(torch, synth.complex_gaussian(50, synth.TAG_RHS, (len(ids), 1, n, 12)))
    out = torch.empty_like(d_in)
    ctx.apply_D_block_noalloc("omega", ids, 1, d_in, out)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        ctx.apply_D_block_noalloc("omega", ids, 1, d_in, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_phi_needs_built_domains():
    """On a fresh context the frame pieces Phi1^a do not exist yet, and building
    them would allocate: the call refuses."""
    torch = pytest.importorskip("torch")
    U, ctx, info, geo = config1()
    n = len(geo.sites(geo.phi_mask[0]))
    x = torch.zeros(n * 24, dtype=torch.float64, device="cuda")
    with pytest.raises(dd4d.DDError) as e:
        ctx.apply_D_block_noalloc("phi", [0], 1, x, x)
    assert e.value.status == dd4d.DD_EINVAL and "Phi1" in str(e.value)
    ctx.close()


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
