"""GPU parity of the restricted Wilson stencil D_X (paper Sec. 3) vs the oracle.

FP64 must agree with the oracle to 1e-12 relative (l2 norm of the difference
over the l2 norm of the oracle output); FP32 storage/arithmetic to 2e-6 and
BF16 storage to 2e-2 (8-bit mantissa: relative rounding 2^-9 per stored
number, accumulated over 9 terms per site).
"""

import numpy as np
import pytest

from paper_2211_06902_gb300 import dd4d, synth
from oracle.geometry import Decomposition, uniform_cores
from oracle.lattice import apply_D, apply_D_restricted

from gpu_common import config1, from_field, make_case, relerr, to_field

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 2e-6, "bf16": 2e-2}


@pytest.fixture(scope="module")
def case1():
    return config1()


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
def test_full_lattice(case1, prec):
    U, ctx, info, geo = case1
    L = geo.L
    V = int(np.prod(L))
    psi = synth.complex_gaussian(1, synth.TAG_RHS, (2, V, 12))
    out = np.zeros_like(psi)
    ctx.apply_D_block("full", None, 2, psi, out, prec)
    for r in range(2):
        ref = apply_D(U, psi[r].reshape(L + (4, 3)), 0.13).reshape(V, 12)
        assert relerr(out[r], ref) < TOL[prec]


@pytest.mark.parametrize("kind,set_id", [("omega", dd4d.SET_OMEGA), ("phi", dd4d.SET_PHI)])
@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
def test_blocks(case1, kind, set_id, prec):
    U, ctx, info, geo = case1
    L = geo.L
    ids = list(range(info["nblocks"]))
    sites = [ctx.geom_sites(set_id, b) for b in ids]
    nrhs = 3
    n = len(sites[0])
    assert all(len(s) == n for s in sites)
    psi = synth.complex_gaussian(2, synth.TAG_RHS, (len(ids), nrhs, n, 12))
    out = np.zeros_like(psi)
    ctx.apply_D_block(kind, ids, nrhs, psi, out, prec)
    masks = geo.omega_mask if kind == "omega" else geo.phi_mask
    for b in ids:
        assert np.array_equal(np.sort(sites[b]), geo.sites(masks[b]))
        for r in range(nrhs):
            f = to_field(L, sites[b], psi[b, r])
            ref = from_field(L, sites[b], apply_D_restricted(U, f, 0.13, masks[b]))
            assert relerr(out[b, r], ref) < TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_frame(case1, prec):
    U, ctx, info, geo = case1
    L = geo.L
    sites = ctx.geom_sites(dd4d.SET_LAMBDA1)
    assert np.array_equal(sites, geo.sites(geo.Lambda1))
    psi = synth.complex_gaussian(3, synth.TAG_RHS, (1, 2, len(sites), 12))
    out = np.zeros_like(psi)
    ctx.apply_D_block("lambda1", None, 2, psi, out, prec)
    for r in range(2):
        f = to_field(L, sites, psi[0, r])
        ref = from_field(L, sites, apply_D_restricted(U, f, 0.13, geo.Lambda1))
        assert relerr(out[0, r], ref) < TOL[prec]


def test_uneven_blocks_and_small_cores():
    """Uneven core sizes (6/8-type mix, per-direction lists) and 1-site cores."""
    L = (12, 8, 8, 10)
    cores = [[(0, 3), (6, 8)], [(1, 2), (5, 6)], [(0, 4), (6, 6)], [(0, 2), (4, 7)]]
    U, ctx, info, geo = make_case(L, 0.12, 0.5, 7, cores)
    ids = [0, 3, 5, 9, 15]
    sites = [ctx.geom_sites(dd4d.SET_OMEGA, b) for b in ids]
    tot = sum(len(s) for s in sites)
    psi = synth.complex_gaussian(4, synth.TAG_RHS, (2 * tot, 12))
    out = np.zeros_like(psi)
    ctx.apply_D_block("omega", ids, 2, psi, out, "f64")
    off = 0
    for k, b in enumerate(ids):
        n = len(sites[k])
        for r in range(2):
            v = psi[off:off + n]
            f = to_field(L, sites[k], v)
            ref = from_field(L, sites[k], apply_D_restricted(U, f, 0.12, geo.omega_mask[b]))
            assert relerr(out[off:off + n], ref) < 1e-12
            off += n


def test_device_pointers_and_streams(case1):
    torch = pytest.importorskip("torch")
    U, ctx, info, geo = case1
    V = int(np.prod(geo.L))
    psi = synth.complex_gaussian(5, synth.TAG_RHS, (1, V, 12))
    dev = torch.from_numpy(psi.view(np.float64).copy()).cuda()
    out = torch.zeros_like(dev)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx.apply_D_block("full", None, 1, dev, out, "f64")
    s.synchronize()
    got = out.cpu().numpy().view(np.complex128)
    ref = apply_D(U, psi[0].reshape(geo.L + (4, 3)), 0.13).reshape(1, V, 12)
    assert relerr(got, ref) < 1e-12


def test_invalid_arguments(case1):
    U, ctx, info, geo = case1
    x = np.zeros((1, 10, 12), dtype=np.complex128)
    with pytest.raises(dd4d.DDError):
        ctx.apply_D_block("omega", [99], 1, x, x, "f64")
    with pytest.raises(dd4d.DDError):
        ctx.apply_D_block("full", None, 0, x, x, "f64")


@pytest.mark.parametrize("prec,nrhs", [("f64", 3), ("f32", 13), ("bf16", 13)])
def test_every_hop_variant(prec, nrhs):
    """Every compiled launch form of the hop (thread per site, several rhs per
    thread, direction split, shared-memory link bundles by bulk copy) against
    the oracle: uneven blocks whose parities end in ragged chunks and quarters,
    the frame Lambda1 (not a box), and 13 rhs, which the bundle form splits
    into two groups of 7 and 6 warps."""
    L = (12, 8, 8, 10)
    cores = [[(0, 3), (6, 8)], [(1, 2), (5, 6)], [(0, 4), (6, 6)], [(0, 2), (4, 7)]]
    U, ctx, info, geo = make_case(L, 0.12, 0.5, 7, cores)
    cases = [("omega", [0, 3, 5, 9, 15], [geo.omega_mask[b] for b in [0, 3, 5, 9, 15]],
              [ctx.geom_sites(dd4d.SET_OMEGA, b) for b in [0, 3, 5, 9, 15]]),
             ("lambda1", None, [geo.Lambda1], [ctx.geom_sites(dd4d.SET_LAMBDA1)])]
    nvar = dd4d.lib().dd_hop_variants(dd4d.PREC[prec])
    assert nvar >= 5
    for kind, ids, masks, sites in cases:
        tot = sum(len(s) for s in sites)
        psi = synth.complex_gaussian(8, synth.TAG_RHS, (nrhs * tot, 12))
        refs = []
        off = 0
        for k in range(len(sites)):
            n = len(sites[k])
            for r in range(nrhs):
                f = to_field(L, sites[k], psi[off:off + n])
                refs.append(from_field(L, sites[k], apply_D_restricted(U, f, 0.12, masks[k])))
                off += n
        ref = np.concatenate(refs)
        for v in range(nvar):
            ctx.set_hop_variant(prec, v)
            out = np.zeros_like(psi)
            ctx.apply_D_block(kind, ids, nrhs, psi, out, prec)
            assert relerr(out, ref) < TOL[prec], (kind, v)
        ctx.set_hop_variant(prec, -1)
