"""The multi-boson action of one lattice sharded over ranks (paper Sec. 5: the
blocks can live on separate GPUs and communicate only for the global terms).

Rank r owns a contiguous range of the framed blocks (``owned_blocks``).  One
evaluation of S = sum_k |(u_k - w) chi_k|^2 (Eqs. MBaction, localMB, globalMB),
with w applied in the stages of ``dd_apply_w_part``:

1. every rank computes the share of Q chi of its own blocks' frame pieces
   Phi1^b on dPi1; a sum across the ranks gives Q chi;
2. chi' = chi - Q chi (on dPi1; identical on every rank);
3. every rank solves its own framed blocks: (w chi)_{dLambda0^a} from chi';
   the frame rank also solves the frame Lambda1 and forms
   (w chi)_{dPi1} = Q chi - P D_{Lambda1}^{-1} D_{Lambda1, dLambda0} chi;
4. S^a on the rank that owns block a, S^r on the frame rank; a sum across the
   ranks of the vector (S^0 .. S^{n-1}, S^r) gives every rank S, S^a and S^r.

Two collectives per evaluation: a sum of n_f x |dPi1| x 12 complex numbers and
a sum of nblocks + 1 doubles.  The frame solve is not split: it runs on one rank
while the others solve their blocks.

The compute of a rank is an object with three methods, arrays of shape
[n_f, n_dpi, 12] complex128 (torch tensors) in the dPi order of the context:
    frame_q(ids, chi)  -> the ids' share of Q chi on dPi1, zero elsewhere
    block_w(ids, chip) -> (w chi)_{dLambda0^a} for a in ids, zero elsewhere
    frame_w(chi)       -> -P_{dPi1} D_{Lambda1}^{-1} D_{Lambda1, dLambda0} chi, zero elsewhere
``LibraryOps`` binds them to ``dd_apply_w_part`` of a context.
"""

import torch

FRAME_RANK = 0


def owned_blocks(nblocks, rank, world):
    """Contiguous block range of a rank: sizes differ by at most one."""
    lo = (nblocks * rank) // world
    hi = (nblocks * (rank + 1)) // world
    return list(range(lo, hi))


class Comm:
    """Sums across ranks with torch.distributed (nothing to do for one rank)."""

    def __init__(self, world):
        self.world = world

    def sum_(self, t):
        if self.world > 1:
            import torch.distributed as dist
            v = torch.view_as_real(t) if t.is_complex() else t
            dist.all_reduce(v)
        return t


def frame_q_share(ops, rank, world, nblocks, chi):
    own = owned_blocks(nblocks, rank, world)
    return ops.frame_q(own, chi) if own else torch.zeros_like(chi)


def local_w(ops, rank, world, nblocks, chi, q, c_mask):
    """The entries of w chi this rank computes (zero elsewhere), from the summed Q chi."""
    own = owned_blocks(nblocks, rank, world)
    chip = chi - q                                  # q vanishes off dPi1
    w = ops.block_w(own, chip) if own else torch.zeros_like(chi)
    if rank == FRAME_RANK:
        w = w + ops.frame_w(chi) + q * c_mask[None, :, None]
    return w


def local_parts(rank, world, u, chi, w, block_of_dpi, nblocks):
    """(S^0 .. S^{n-1}, S^r) with the entries of the blocks this rank owns and, on
    the frame rank, S^r; zero elsewhere."""
    own = owned_blocks(nblocks, rank, world)
    r = u[:, None, None] * chi - w
    site2 = (r.abs() ** 2).sum(dim=(0, 2))           # |r|^2 per dPi site, summed over fields
    parts = torch.zeros(nblocks + 1, dtype=torch.float64, device=chi.device)
    if own:
        idx = block_of_dpi.clone()
        keep = (idx >= own[0]) & (idx <= own[-1])
        parts.index_add_(0, idx[keep], site2[keep])
    if rank == FRAME_RANK:
        parts[nblocks] = site2[block_of_dpi < 0].sum()
    return parts


def multiboson_action(ops, comm, rank, world, u, chi, block_of_dpi):
    """S, [S^a], S^r of the fields chi [n_f, n_dpi, 12] for the roots u [n_f]
    (complex128 tensors), identical on every rank.  block_of_dpi: the block of
    each dLambda0 site in dPi order, -1 on dPi1 (a long tensor)."""
    nblocks = int(block_of_dpi.max().item()) + 1
    c_mask = (block_of_dpi < 0).to(chi.dtype)
    q = comm.sum_(frame_q_share(ops, rank, world, nblocks, chi))
    w = local_w(ops, rank, world, nblocks, chi, q, c_mask)
    parts = comm.sum_(local_parts(rank, world, u, chi, w, block_of_dpi, nblocks))
    return float(parts.sum().item()), parts[:nblocks].tolist(), float(parts[nblocks].item())


class LibraryOps:
    """The three stages on a libdd4d context (device tensors)."""

    def __init__(self, ctx, prm=None):
        self.ctx = ctx
        self.prm = prm

    def _run(self, part, ids, chi):
        out = torch.zeros_like(chi)
        self.ctx.apply_w_part(part, chi.shape[0], ids, torch.view_as_real(chi), torch.view_as_real(out),
                              self.prm)
        return out

    def frame_q(self, ids, chi):
        return self._run("frame_q", ids, chi)

    def block_w(self, ids, chip):
        return self._run("blocks", ids, chip)

    def frame_w(self, chi):
        return self._run("frame", None, chi)


def block_of_dpi(ctx, nblocks, device=None):
    """The block of every dLambda0 site in dPi order, -1 on dPi1 (from the context)."""
    import numpy as np
    from . import dd4d
    dpi = ctx.geom_sites(dd4d.SET_DPI)
    out = np.full(len(dpi), -1, dtype=np.int64)
    for b in range(nblocks):
        out[np.searchsorted(dpi, ctx.geom_sites(dd4d.SET_B, b))] = b
    t = torch.from_numpy(out)
    return t.to(device) if device is not None else t
