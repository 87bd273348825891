"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module only draws random numbers and shapes them into inputs: gauge links
and Gaussian fields.  It contains none of the domain-decomposition arithmetic,
so both the CUDA path and the FP64 oracle can take their inputs from here
without sharing any of the method's code.

Random numbers
--------------
A counter-based SplitMix64 stream: the n-th 64-bit draw of stream ``key`` is
``mix64(key + (n + 1) * 0x9E3779B97F4A7C15)`` with the SplitMix64 finaliser
``mix64``.  A stream key is derived from a (seed, tag) pair as
``mix64(mix64(seed) ^ (tag * 0xD1B54A32D192ED03))``.  Uniforms take the top 53
bits, ``u = ((z >> 11) + 1) * 2**-53`` in (0, 1], and normal deviates come in
Box-Muller pairs from consecutive uniforms: draw 2j -> sqrt(-2 ln u_2j)
cos(2 pi u_2j+1), draw 2j+1 -> the same radius times sin(...).

Gauge field (the links U_mu(x) of Sec. 1 of the paper)
------------------------------------------------------
U_mu(x) = exp(i eps H), H = sum_a h_a lambda_a / 2 with the eight Gell-Mann
matrices lambda_a and h_a ~ N(0, 1).  The h_a are consumed in link order: site
x lexicographic with x3 fastest, then mu = 0..3, then a = 1..8.  The exponential
is taken through the eigen-decomposition of the Hermitian H.  Array layout:
``[L0, L1, L2, L3, 4 (mu), 3, 3]`` complex128, x0 is time.

Quark-type fields (spinors, multi-boson fields, right-hand sides)
----------------------------------------------------------------
Complex Gaussians with Re, Im ~ N(0, 1/2), i.e. E|z|^2 = 1 per component.
"""

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_TAGMUL = 0xD1B54A32D192ED03

# stream tags used across the project
TAG_GAUGE = 1
TAG_RHS = 2
TAG_CHI = 3
TAG_PERTURB = 4
TAG_NET = 5
TAG_MOMENTA = 6


def _mix64(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed, tag):
    """64-bit key of the (seed, tag) stream."""
    s = _mix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF))
    t = np.uint64((tag * _TAGMUL) & 0xFFFFFFFFFFFFFFFF)
    return _mix64(s ^ t)


def raw64(key, start, count):
    """Draws start .. start+count-1 of the stream ``key`` (uint64 array)."""
    n = np.arange(start, start + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(np.uint64(key) + (n + np.uint64(1)) * _GOLDEN)


def uniforms(key, start, count):
    z = raw64(key, start, count)
    return ((z >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)


def normals(seed, tag, count):
    """``count`` N(0,1) deviates of stream (seed, tag), Box-Muller pairs."""
    key = stream_key(seed, tag)
    npair = (count + 1) // 2
    u = uniforms(key, 0, 2 * npair).reshape(npair, 2)
    r = np.sqrt(-2.0 * np.log(u[:, 0]))
    ang = 2.0 * np.pi * u[:, 1]
    out = np.empty((npair, 2))
    out[:, 0] = r * np.cos(ang)
    out[:, 1] = r * np.sin(ang)
    return out.reshape(-1)[:count]


def gell_mann():
    """The eight Gell-Mann matrices lambda_1..lambda_8, shape [8, 3, 3]."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1], lam[1][1, 0] = -1j, 1j
    lam[2][0, 0], lam[2][1, 1] = 1, -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2], lam[4][2, 0] = -1j, 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2], lam[6][2, 1] = -1j, 1j
    lam[7] = np.diag([1, 1, -2]) / np.sqrt(3.0)
    return lam


def gauge_field(L, eps, seed):
    """Random SU(3) links U = exp(i eps H), layout [L0,L1,L2,L3,4,3,3] complex128."""
    L = tuple(int(v) for v in L)
    V = int(np.prod(L))
    h = normals(seed, TAG_GAUGE, V * 4 * 8).reshape(V * 4, 8)
    H = np.einsum("na,aij->nij", h, gell_mann() / 2.0)
    H = 0.5 * (H + np.conj(np.swapaxes(H, 1, 2)))
    e, v = np.linalg.eigh(H)
    U = np.einsum("nij,nj,nkj->nik", v, np.exp(1j * eps * e), np.conj(v))
    return np.ascontiguousarray(U.reshape(L + (4, 3, 3)))


def unit_gauge(L):
    """U_mu(x) = 1 everywhere (free field)."""
    L = tuple(int(v) for v in L)
    U = np.zeros(L + (4, 3, 3), dtype=np.complex128)
    U[..., :, :] = np.eye(3)
    return U


def complex_gaussian(seed, tag, shape):
    """Complex Gaussian array with Re, Im ~ N(0, 1/2)."""
    shape = tuple(int(s) for s in shape)
    n = int(np.prod(shape))
    g = normals(seed, tag, 2 * n).reshape(n, 2) * np.sqrt(0.5)
    return (g[:, 0] + 1j * g[:, 1]).reshape(shape)


def momenta(L, seed):
    """Gaussian momenta P_t(x, mu) ~ N(0, 1), layout [L0,L1,L2,L3,4,8] float64
    (the link momenta of a molecular-dynamics trajectory)."""
    L = tuple(int(v) for v in L)
    V = int(np.prod(L))
    return normals(seed, TAG_MOMENTA, V * 32).reshape(L + (4, 8))


def gauge_transform(seed, L):
    """Random SU(3) matrices g(x), layout [L0,L1,L2,L3,3,3] (for covariance tests)."""
    L = tuple(int(v) for v in L)
    V = int(np.prod(L))
    h = normals(seed, TAG_PERTURB, V * 8).reshape(V, 8)
    H = np.einsum("na,aij->nij", h, gell_mann() / 2.0)
    H = 0.5 * (H + np.conj(np.swapaxes(H, 1, 2)))
    e, v = np.linalg.eigh(H)
    g = np.einsum("nij,nj,nkj->nik", v, np.exp(1j * e), np.conj(v))
    return np.ascontiguousarray(g.reshape(L + (3, 3)))


def net_init_weights(seed, channels=(4, 16, 16, 16, 4)):
    """Seeded initial weights of the parallel-transport network, one complex
    array [9 directions, C_out, C_in] per layer: unit centre taps on the
    diagonal plus Gaussian noise of scale 0.02 / sqrt(C_in)."""
    Ws = []
    for l in range(len(channels) - 1):
        cin, cout = channels[l], channels[l + 1]
        w = complex_gaussian(seed, TAG_NET + 64 * l, (9, cout, cin)) * (0.02 / np.sqrt(cin))
        for c in range(min(cin, cout)):
            w[0, c, c] += 1.0
        Ws.append(w)
    return Ws
