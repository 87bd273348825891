"""Four-dimensional domain decomposition of the lattice (oracle, CPU).

Test infrastructure only (see the package docstring).

Sec. 2 of the paper defines the sets in words and figures and defers the exact
definitions to an appendix of an earlier paper that is not available; the
reading used here is:

* Per direction mu a sorted list of core intervals [lo_i, hi_i] (inclusive,
  disjoint, separated by at least one frame site, periodic); at least two per
  direction.  A block Lambda0^a is the product of one core interval per
  direction; blocks are numbered lexicographically in the interval indices
  (direction 3 fastest).
* Lambda0 = union of the blocks (the active region), Lambda1 = the rest
  (the inactive, connected frame).
* dLambda0^a = sites of Lambda0^a having a neighbour outside it; the bulk
  Lambda0bar^a is the rest of the block.
* dPi = union of the hyperplanes x_mu in {lo_i, hi_i} that carry the block
  boundaries; dPi1 = dPi minus dLambda0 (it lies in Lambda1).  Lambda1bar =
  Lambda1 minus dPi1.
* Omega0^a = {x : hi_prev < x_mu < lo_next for all mu} (periodic), i.e. the
  block plus the frame up to the neighbouring hyperplanes (Fig. 2);
  Phi1^a = Omega0^a minus Lambda0^a.
* The exterior boundary of Omega0^a is the set of sites outside it with a
  neighbour inside; its part in dPi1 is the starred set of Fig. 2.
"""

import numpy as np


class Block:
    def __init__(self, idx, core, omega_start, omega_len):
        self.idx = idx                      # interval index per direction
        self.core = core                    # [(lo, hi)] * 4
        self.omega_start = omega_start      # first site of Omega per direction
        self.omega_len = omega_len          # side of Omega per direction


def _interval_mask(L, start, length):
    m = np.zeros(L, dtype=bool)
    m[(start + np.arange(length)) % L] = True
    return m


def _product(masks):
    return (masks[0][:, None, None, None] & masks[1][None, :, None, None]
            & masks[2][None, None, :, None] & masks[3][None, None, None, :])


def _neighbours_of(mask):
    """Sites that have at least one nearest neighbour in ``mask`` (periodic)."""
    out = np.zeros_like(mask)
    for mu in range(4):
        out |= np.roll(mask, 1, axis=mu) | np.roll(mask, -1, axis=mu)
    return out


class Decomposition:
    def __init__(self, L, cores):
        L = tuple(int(v) for v in L)
        self.L = L
        self.cores = [list(map(tuple, c)) for c in cores]
        # an empty core list: the direction is not decomposed (a single core
        # spanning its whole periodic extent, no frame and no hyperplane); the
        # one-dimensional decomposition in thick time slices of Sec. 3 is the
        # case with only direction 0 decomposed
        self.decomposed = [len(c) > 0 for c in self.cores]
        if not any(self.decomposed):
            raise ValueError("at least one direction must be decomposed")
        for mu in range(4):
            c = self.cores[mu]
            if not self.decomposed[mu]:
                self.cores[mu] = [(0, L[mu] - 1)]
                continue
            if len(c) < 2:
                raise ValueError("need at least two cores per decomposed direction")
            for i, (lo, hi) in enumerate(c):
                if not (0 <= lo <= hi < L[mu]):
                    raise ValueError("core outside the lattice")
                if i > 0 and lo <= c[i - 1][1] + 1:
                    raise ValueError("cores must be separated by a frame")
            if (c[0][0] + L[mu]) - c[-1][1] < 2:
                raise ValueError("cores must be separated by a frame")
        coords = np.indices(L)

        # hyperplane coordinates per direction
        planes = [sorted({v for iv in self.cores[mu] for v in iv}) if self.decomposed[mu] else []
                  for mu in range(4)]
        on_plane = np.zeros(L, dtype=bool)
        for mu in range(4):
            on_plane |= np.isin(coords[mu], planes[mu])
        self.dPi = on_plane

        self.blocks = []
        self.core_mask, self.B_mask, self.omega_mask = [], [], []
        self.phi_mask, self.ext_mask, self.ext_star_mask = [], [], []
        nc = [len(c) for c in self.cores]
        for i0 in range(nc[0]):
            for i1 in range(nc[1]):
                for i2 in range(nc[2]):
                    for i3 in range(nc[3]):
                        idx = (i0, i1, i2, i3)
                        core = [self.cores[mu][idx[mu]] for mu in range(4)]
                        start, length = [], []
                        for mu in range(4):
                            if not self.decomposed[mu]:
                                start.append(0)
                                length.append(L[mu])
                                continue
                            prev_hi = self.cores[mu][(idx[mu] - 1) % nc[mu]][1]
                            next_lo = self.cores[mu][(idx[mu] + 1) % nc[mu]][0]
                            s = (prev_hi + 1) % L[mu]
                            n = (next_lo - 1 - prev_hi) % L[mu]
                            if n == 0:
                                n = L[mu]
                            start.append(s)
                            length.append(n)
                        self.blocks.append(Block(idx, core, start, length))
        for b in self.blocks:
            cm = _product([_interval_mask(L[mu], b.core[mu][0], b.core[mu][1] - b.core[mu][0] + 1)
                           for mu in range(4)])
            om = _product([_interval_mask(L[mu], b.omega_start[mu], b.omega_len[mu])
                           for mu in range(4)])
            edge = np.zeros(L, dtype=bool)
            for mu in range(4):
                if self.decomposed[mu]:
                    edge |= (coords[mu] == b.core[mu][0]) | (coords[mu] == b.core[mu][1])
            self.core_mask.append(cm)
            self.B_mask.append(cm & edge)
            self.omega_mask.append(om)
            self.phi_mask.append(om & ~cm)
            ext = _neighbours_of(om) & ~om
            self.ext_mask.append(ext)
        self.Lambda0 = np.zeros(L, dtype=bool)
        self.B = np.zeros(L, dtype=bool)
        for cm, bm in zip(self.core_mask, self.B_mask):
            self.Lambda0 |= cm
            self.B |= bm
        self.Lambda1 = ~self.Lambda0
        self.A = self.Lambda0 & ~self.B
        self.C = self.dPi & self.Lambda1
        self.E = self.Lambda1 & ~self.C
        self.ext_star_mask = [e & self.C for e in self.ext_mask]

    @property
    def nblocks(self):
        return len(self.blocks)

    def sites(self, mask):
        """Global lexicographic indices of a mask's sites, in increasing order."""
        return np.flatnonzero(mask.ravel())

    def counts(self):
        return dict(
            nblocks=self.nblocks,
            omega=[int(m.sum()) for m in self.omega_mask],
            Lambda1=int(self.Lambda1.sum()), dPi=int(self.dPi.sum()),
            B=int(self.B.sum()), C=int(self.C.sum()), E=int(self.E.sum()),
            A=int(self.A.sum()))


def uniform_cores(L, core, frame, offset=0):
    """Cores of ``core`` sites followed by ``frame`` frame sites, per direction.

    ``core``, ``frame`` and ``offset`` may be scalars or per-direction lists.
    """
    def per(v):
        return list(v) if np.ndim(v) else [v] * 4
    core, frame, offset = per(core), per(frame), per(offset)
    out = []
    for mu in range(4):
        period = core[mu] + frame[mu]
        if L[mu] % period:
            raise ValueError("period does not divide the lattice")
        out.append([(offset[mu] + i * period, offset[mu] + i * period + core[mu] - 1)
                    for i in range(L[mu] // period)])
    return out
