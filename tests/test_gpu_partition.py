"""The sharded multi-boson action with the library's stages (dd_apply_w_part).

Two ranks are emulated in one process, one after the other: rank r computes its
blocks' share of Q chi, the shares are summed on the host, each rank solves its
blocks on chi' = chi - Q chi and rank 0 the frame, and the per-rank parts are
summed.  The stages solve the same systems as the one-call path but in other
batches (the BiCGstab shadow vector depends on a system's place in its batch),
so they agree with dd_apply_w and dd_multiboson_action to the solves' tolerance
(1e-12, times the conditioning: 1e-10 asked) and with the oracle to 1e-9 (8^4
and an uneven 12x8x8x10 decomposition).
"""

import numpy as np
import pytest
import torch

from paper_2211_06902_gb300 import dd4d, partition, synth
from oracle.dd import Oracle, field_roots

from gpu_common import config1, make_case

pytestmark = pytest.mark.gpu

CASES = {
    "8^4": config1,
    "uneven 12x8x8x10": lambda: make_case((12, 8, 8, 10), 0.12, 0.5, 7,
                                          [[(0, 3), (6, 8)], [(1, 2), (5, 6)], [(0, 4), (6, 6)],
                                           [(0, 2), (4, 7)]]),
}


@pytest.mark.parametrize("name", list(CASES))
def test_two_emulated_ranks_match_one_call(name):
    U, ctx, info, geo = CASES[name]()
    kappa = 0.13 if name == "8^4" else 0.12
    nb = info["nblocks"]
    u = field_roots(4, 0.5)
    dpi = ctx.geom_sites(dd4d.SET_DPI)
    V = int(np.prod(geo.L))
    chis = [synth.complex_gaussian(5, synth.TAG_CHI + k, geo.L + (4, 3)) * geo.dPi[..., None, None]
            for k in range(len(u))]
    chi = torch.from_numpy(np.stack([c.reshape(V, 12)[dpi] for c in chis])).cuda()
    prm = dd4d.params(1e-12)
    ops = partition.LibraryOps(ctx, prm)
    bod = partition.block_of_dpi(ctx, nb, device="cuda")
    cmask = (bod < 0).to(chi.dtype)
    ut = torch.from_numpy(np.asarray(u)).cuda()
    world = 2
    q = sum(partition.frame_q_share(ops, r, world, nb, chi) for r in range(world))
    ws = [partition.local_w(ops, r, world, nb, chi, q, cmask) for r in range(world)]
    parts = sum(partition.local_parts(r, world, ut, chi, ws[r], bod, nb) for r in range(world))
    S, Sa, Sr = float(parts.sum()), parts[:nb].cpu().numpy(), float(parts[nb])
    # the stages add up to w itself
    w_one = torch.zeros_like(chi)
    ctx.apply_w(len(u), torch.view_as_real(chi), torch.view_as_real(w_one), prm)
    torch.cuda.synchronize()
    w_sum = ws[0] + ws[1]
    assert float((w_sum - w_one).abs().max()) <= 1e-10 * float(w_one.abs().max())
    S1, Sb1, Sr1, st = ctx.multiboson_action(u, torch.view_as_real(chi), prm)
    assert abs(S - S1) <= 1e-10 * S1
    assert np.allclose(Sa, Sb1, rtol=1e-10, atol=1e-10 * S1)
    assert abs(Sr - Sr1) <= 1e-10 * S1
    S0, Sa0, Sr0 = Oracle(U, kappa, geo).multiboson_action(u, chis)
    assert abs(S - S0) <= 1e-9 * S0
    assert np.allclose(Sa, Sa0, rtol=1e-9, atol=1e-9 * S0)
