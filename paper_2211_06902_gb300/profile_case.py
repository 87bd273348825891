"""One batched block solve (or network application) on a chosen lattice, the
small cases that the ncu summaries under profiles/ were taken on.

    python -m paper_2211_06902_gb300.profile_case --L 24 --core 7 --nrhs 12 --inner f32 --variant 13
    python -m paper_2211_06902_gb300.profile_case --L 24 --nrhs 12 --net

Builds the lattice (links exp(i eps H)), the framed blocks of `core`^4 cores
with a one-site frame, Gaussian right-hand sides on every block, and runs
`--repeat` solves to 1e-10 with the requested inner precision (or, with
--net, `--repeat` applications of the 4-layer network with tensor-core
layers); --csw adds the clover term to the solves.  Prints the solver
statistics; exits non-zero if a system misses the tolerance.
"""

import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2211_06902_gb300 import dd4d, synth  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, default=24)
    ap.add_argument("--core", type=int, default=7)
    ap.add_argument("--frame", type=int, default=1)
    ap.add_argument("--nrhs", type=int, default=12)
    ap.add_argument("--kappa", type=float, default=0.135)
    ap.add_argument("--eps", type=float, default=0.5)
    ap.add_argument("--inner", default="f32", choices=["f64", "f32", "bf16"])
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--variant", type=int, default=-1,
                    help="stencil launch variant of the inner precision (-1: default)")
    ap.add_argument("--net", action="store_true", help="apply the network instead of solving")
    ap.add_argument("--csw", type=float, default=0.0, help="clover coefficient (0: no clover term)")
    a = ap.parse_args()
    import torch
    torch.cuda.init()
    L = (a.L,) * 4
    per = a.core + a.frame
    cores = [[(i * per, i * per + a.core - 1) for i in range(a.L // per)] for _ in range(4)]
    ctx = dd4d.Context(L, a.kappa)
    ctx.gauge_upload(synth.gauge_field(L, a.eps, 2))
    info = ctx.set_geometry(cores)
    ids = list(range(info["nblocks"]))
    b = synth.complex_gaussian(2, synth.TAG_RHS, (len(ids), a.nrhs, info["max_omega"], 12))
    bd = torch.from_numpy(b.view(np.float64)).cuda()
    xd = torch.zeros_like(bd)
    if a.net:
        net = dd4d.Net(ctx, synth.net_init_weights(11))
        y = torch.zeros_like(bd)
        for _ in range(a.repeat):
            net.apply(ids, a.nrhs, bd, y)
        torch.cuda.synchronize()
        print("network applied", a.repeat, "times, |y| =", float(y.norm()))
        net.close()
        ctx.close()
        return 0
    if a.csw:
        ctx.set_clover(a.csw)
    if a.variant >= 0:
        ctx.set_hop_variant(a.inner, a.variant)
    prm = dd4d.params(1e-10, inner_prec=a.inner)
    for _ in range(a.repeat):
        st = ctx.solve_blocks("omega", ids, a.nrhs, bd, xd, prm)
        print(st)
        if st["status"] != 0:
            return 1
    ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
