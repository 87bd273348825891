"""The multi-boson action of one lattice sharded over two ranks (gloo, CPU).

Each rank owns half of the 16 framed blocks of a 6^4 lattice: it computes
its blocks' share of Q chi on dPi1 (a sum across the ranks completes it), solves
its own framed blocks on chi' = chi - Q chi, and rank 0 also solves the frame;
a sum of the per-block and frame parts gives S, S^a and S^r on every rank.  The
per-rank compute is done here with the oracle's block, frame-piece and frame
solves; the result must equal the single-rank oracle action (printed W_1 of
Sec. 3) to 1e-9 relative, on both ranks.  The library runs the same driver
with its own stages (tests/test_gpu_partition.py).
"""

import os
import socket

import numpy as np
import pytest
import torch

from paper_2211_06902_gb300 import partition, synth
from oracle.dd import Oracle, field_roots
from oracle.geometry import Decomposition, uniform_cores

L = (6, 6, 6, 6)


class OracleOps:
    """The three stages of w from the oracle's solvers (test-side adapter)."""

    def __init__(self, o):
        self.o = o
        self.g = o.g
        self.dpi = self.g.sites(self.g.dPi)
        self.V = int(np.prod(self.g.L))

    def _fields(self, t):
        a = t.numpy()
        out = []
        for k in range(a.shape[0]):
            f = np.zeros((self.V, 12), dtype=np.complex128)
            f[self.dpi] = a[k]
            out.append(f.reshape(tuple(self.g.L) + (4, 3)))
        return out

    def _tensor(self, fields):
        return torch.from_numpy(np.stack([f.reshape(self.V, 12)[self.dpi] for f in fields]))

    def frame_q(self, ids, chi):
        o, g = self.o, self.g
        out = []
        for f in self._fields(chi):
            acc = np.zeros_like(f)
            for b in ids:
                y = o.phi_solver(b).solve_field(o._D(g.phi_mask[b], g.B_mask[b], f))
                acc += y * g.C[..., None, None]
            out.append(acc)
        return self._tensor(out)

    def block_w(self, ids, chip):
        o, g = self.o, self.g
        out = []
        for f in self._fields(chip):
            w = np.zeros_like(f)
            for a in ids:
                psi = o.omega_solver(a).solve_field(o._D(g.omega_mask[a], g.ext_mask[a], f))
                w[g.B_mask[a]] = -psi[g.B_mask[a]]
            out.append(w)
        return self._tensor(out)

    def frame_w(self, chi):
        o, g = self.o, self.g
        out = []
        for f in self._fields(chi):
            y = o.frame_solver().solve_field(o._D(g.Lambda1, g.B, f))
            w = np.zeros_like(f)
            w[g.C] = -y[g.C]
            out.append(w)
        return self._tensor(out)


def _case():
    U = synth.gauge_field(L, 0.3, 1)
    g = Decomposition(L, uniform_cores(L, 2, 1))
    u = field_roots(4, 0.5)
    chis = [synth.complex_gaussian(1, synth.TAG_CHI + k, L + (4, 3)) * g.dPi[..., None, None]
            for k in range(len(u))]
    return U, g, u, chis


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        U, g, u, chis = _case()
        ops = OracleOps(Oracle(U, 0.13, g))
        chi = ops._tensor(chis)
        bod = torch.full((len(ops.dpi),), -1, dtype=torch.long)
        for b in range(g.nblocks):
            bod[torch.from_numpy(np.searchsorted(ops.dpi, g.sites(g.B_mask[b])))] = b
        S, Sa, Sr = partition.multiboson_action(ops, partition.Comm(world), rank, world,
                                                torch.from_numpy(np.asarray(u)), chi, bod)
        q.put((rank, S, Sa, Sr))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_owned_blocks_cover_every_block_once():
    for nb, world in [(16, 2), (16, 3), (5, 4), (1296, 8)]:
        got = [b for r in range(world) for b in partition.owned_blocks(nb, r, world)]
        assert got == list(range(nb))
        sizes = [len(partition.owned_blocks(nb, r, world)) for r in range(world)]
        assert max(sizes) - min(sizes) <= 1


def test_two_ranks_match_the_single_rank_oracle():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=600) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    U, g, u, chis = _case()
    S0, Sa0, Sr0 = Oracle(U, 0.13, g).multiboson_action(u, chis)
    for rank, S, Sa, Sr in res:
        assert abs(S - S0) <= 1e-9 * S0, (rank, S, S0)
        assert abs(Sr - Sr0) <= 1e-9 * S0
        assert np.allclose(Sa, Sa0, rtol=1e-9, atol=1e-9 * S0)
    assert res[0][1:] == res[1][1:]                  # both ranks hold the same numbers
