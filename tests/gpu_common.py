"""Helpers shared by the GPU parity tests (inputs, layouts, oracle adapters)."""

import numpy as np

from paper_2211_06902_gb300 import dd4d, synth
from oracle.geometry import Decomposition, uniform_cores

CONFIG1 = dict(L=(8, 8, 8, 8), kappa=0.13, eps=0.3, seed=1, core=3, frame=1)


def make_case(L, kappa, eps, seed, cores):
    U = synth.gauge_field(L, eps, seed)
    ctx = dd4d.Context(L, kappa)
    ctx.gauge_upload(U)
    info = ctx.set_geometry(cores)
    geo = Decomposition(L, cores)
    return U, ctx, info, geo


def config1():
    c = CONFIG1
    cores = uniform_cores(c["L"], c["core"], c["frame"])
    return make_case(c["L"], c["kappa"], c["eps"], c["seed"], cores)


def to_field(L, sites, vec):
    """Scatter a [nsites, 12] vector to a full-lattice field [L..,4,3]."""
    V = int(np.prod(L))
    f = np.zeros((V, 12), dtype=np.complex128)
    f[sites] = vec.reshape(-1, 12)
    return f.reshape(tuple(L) + (4, 3))


def from_field(L, sites, field):
    V = int(np.prod(L))
    return field.reshape(V, 12)[sites]


def relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
