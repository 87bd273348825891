"""Pins of the oracle's domain decomposition (Sec. 2 of the paper).

Set sizes are checked against closed-form counts computed here from the core
lists alone; the structural statements of Sec. 2 and 3 (disjointness,
dPi = dLambda0 u dPi1, Phi1 inside Lambda1, the bulk of the blocks not
touching Lambda1, the exterior boundary of each framed block lying on dPi, and
the double cover of the frame by the Omega intervals of Sec. 3's
one-dimensional case) are checked by brute force on the site sets.
"""

import numpy as np
import pytest

from oracle.geometry import Decomposition, uniform_cores

CASES = [
    ((8, 8, 8, 8), uniform_cores((8, 8, 8, 8), 3, 1)),
    ((4, 4, 4, 4), uniform_cores((4, 4, 4, 4), 1, 1)),
    ((6, 4, 4, 4), [[(0, 1), (3, 4)]] + [[(0, 0), (2, 2)]] * 3),
    ((16, 16, 16, 16), uniform_cores((16,) * 4, 7, 1)),
    ((32, 16, 16, 16), [[(0, 5), (7, 14), (16, 21), (23, 30)]]
     + [[(0, 5), (7, 14)]] * 3),
    ((12, 8, 8, 10), [[(0, 3), (6, 8)], [(1, 2), (5, 6)], [(0, 4), (6, 6)], [(0, 2), (4, 7)]]),
]


def _closed_form(L, cores):
    V = int(np.prod(L))
    sizes = [[hi - lo + 1 for lo, hi in c] for c in cores]
    nblk = int(np.prod([len(c) for c in cores]))
    lam0 = int(np.prod([sum(s) for s in sizes]))
    bulk = int(np.prod([sum(max(v - 2, 0) for v in s) for s in sizes]))
    planes = [len({v for iv in c for v in iv}) for c in cores]
    dpi = V - int(np.prod([L[mu] - planes[mu] for mu in range(4)]))
    B = lam0 - bulk
    omega = []
    for idx in np.ndindex(*[len(c) for c in cores]):
        side = []
        for mu in range(4):
            c = cores[mu]
            lo, hi = c[idx[mu]]
            gap_before = (lo - c[(idx[mu] - 1) % len(c)][1] - 1) % L[mu]
            gap_after = (c[(idx[mu] + 1) % len(c)][0] - hi - 1) % L[mu]
            side.append(gap_before + (hi - lo + 1) + gap_after)
        omega.append(int(np.prod(side)))
    return dict(nblocks=nblk, Lambda1=V - lam0, dPi=dpi, B=B, C=dpi - B,
                E=V - lam0 - (dpi - B), A=bulk, omega=omega)


@pytest.mark.parametrize("L,cores", CASES)
def test_set_sizes_closed_form(L, cores):
    g = Decomposition(L, cores)
    assert g.counts() == _closed_form(L, cores)


def test_config_8_4_sizes():
    """8^4 with 3^4 cores and a one-site frame: 16 blocks, Omega = 5^4."""
    g = Decomposition((8,) * 4, uniform_cores((8,) * 4, 3, 1))
    c = g.counts()
    assert (c["nblocks"], c["Lambda1"], c["dPi"], c["B"], c["C"], c["E"], c["A"]) == \
        (16, 2800, 3840, 1280, 2560, 240, 16)
    assert set(c["omega"]) == {625}


def _adjacent(m1, m2):
    hit = False
    for mu in range(4):
        hit |= np.any(m1 & (np.roll(m2, 1, axis=mu) | np.roll(m2, -1, axis=mu)))
    return bool(hit)


@pytest.mark.parametrize("L,cores", CASES[:3] + CASES[5:])
def test_structure(L, cores):
    g = Decomposition(L, cores)
    V = int(np.prod(L))
    total = np.zeros(L, dtype=int)
    for cm in g.core_mask:
        total += cm
    assert total.max() == 1                                  # disjoint blocks
    assert np.array_equal(g.B | g.C, g.dPi)                  # dPi = dLambda0 u dPi1
    assert not np.any(g.B & g.C)
    assert np.array_equal(g.B, g.dPi & g.Lambda0)
    assert not np.any(g.C & g.Lambda0)
    assert not _adjacent(g.A, g.Lambda1)                     # bulk never touches Lambda1
    for a in range(g.nblocks):
        assert not np.any(g.phi_mask[a] & g.Lambda0)         # Phi1^a inside Lambda1
        assert np.all(g.dPi[g.ext_mask[a]])                  # exterior boundary on dPi
        assert not np.any(g.ext_mask[a] & g.omega_mask[a])
        # the neighbours of dLambda0^a outside the block all lie in Phi1^a
        out = np.zeros(L, dtype=bool)
        for mu in range(4):
            out |= np.roll(g.B_mask[a], 1, axis=mu) | np.roll(g.B_mask[a], -1, axis=mu)
        out &= ~g.core_mask[a]
        assert np.all(g.phi_mask[a][out])
        # the bulk of a block has all its neighbours inside the block
        inner = g.core_mask[a] & ~g.B_mask[a]
        assert not _adjacent(inner, ~g.core_mask[a])
    assert int(g.Lambda1.sum()) + sum(int(m.sum()) for m in g.core_mask) == V


@pytest.mark.parametrize("L,cores", CASES)
def test_frame_covered_twice_per_direction(L, cores):
    """Per direction the Omega intervals cover core sites once and frame sites twice.

    This is the one-dimensional statement of Sec. 3 (each thick slice of
    Lambda1 is covered twice by the frames), which the 4D sets inherit
    direction by direction.
    """
    g = Decomposition(L, cores)
    for mu in range(4):
        cover = np.zeros(L[mu], dtype=int)
        seen = set()
        for b in g.blocks:
            if b.idx[mu] in seen:
                continue
            seen.add(b.idx[mu])
            cover[(b.omega_start[mu] + np.arange(b.omega_len[mu])) % L[mu]] += 1
        in_core = np.zeros(L[mu], dtype=bool)
        for lo, hi in cores[mu]:
            in_core[lo:hi + 1] = True
        assert np.all(cover[in_core] == 1)
        assert np.all(cover[~in_core] == 2)


def test_invalid_geometries():
    with pytest.raises(ValueError):
        Decomposition((8,) * 4, [[(0, 6)]] + [[(0, 2), (4, 6)]] * 3)
    with pytest.raises(ValueError):
        Decomposition((8,) * 4, [[(0, 2), (3, 6)]] + [[(0, 2), (4, 6)]] * 3)


def _cores(period_sizes):
    """Core intervals from (core size, frame) pairs laid end to end from x = 0."""
    out, x = [], 0
    for size, frame in period_sizes:
        out.append((x, x + size - 1))
        x += size + frame
    return out


BENCH_GEOMETRIES = {
    # L, cores, (blocks, Lambda1, dPi, B, C, E, A), set of Omega sizes
    "32^4": ((32,) * 4, [_cores([(7, 1)] * 4)] * 4,
             (256, 433920, 716800, 454656, 262144, 171776, 160000), {6561}),
    "64x32^3": ((64, 32, 32, 32), [_cores([(6, 1), (8, 1)] * 4)] + [_cores([(6, 1), (8, 1)] * 2)] * 3,
                (512, 867840, 1433600, 909312, 524288, 343552, 320000), None),
    "48^4": ((48,) * 4, [_cores([(7, 1)] * 6)] * 4,
             (1296, 2196720, 3628800, 2301696, 1327104, 869616, 810000), {6561}),
}


@pytest.mark.parametrize("name", list(BENCH_GEOMETRIES))
def test_large_configuration_sizes(name):
    """Closed-form set sizes of the benchmark geometries (counted per direction,
    no lattice masks) against the stored counts; the closed form itself is pinned
    by brute force over the site sets of the smaller lattices above."""
    L, cores, ref, omegas = BENCH_GEOMETRIES[name]
    c = _closed_form(L, cores)
    assert (c["nblocks"], c["Lambda1"], c["dPi"], c["B"], c["C"], c["E"], c["A"]) == ref
    if omegas is not None:
        assert set(c["omega"]) == omegas
    else:
        assert len(set(c["omega"])) == 5 and min(c["omega"]) == 4096 and max(c["omega"]) == 10000
