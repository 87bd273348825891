"""Trains the learned block preconditioner on solver-generated pairs and measures
what it gains on a held-out lattice.

Training set (defaults): 5 lattices of 32^4 (kappa 0.135, links exp(i eps H) with
eps 0.40, 0.45, 0.50, 0.55, 0.60, seeds 100..104), 256 framed blocks of 9^4 each
(7^4 cores, frame 1), 16 complex Gaussian sources per block: 20,480 pairs
(b, D_Omega^{-1} b), the targets from the library's FP64 solver.  The network
(4 layers, 4-16-16-16-4 channels of colour vectors, BF16 weights, tensor-core
layers) takes `steps` full-batch Adam steps on each lattice's pairs in turn.

Held-out test: the bench lattice (eps 0.5, seed 2), 256 blocks x 12 sources;
mixed-precision solves to 1e-10 with FGMRES(10) inner solves without and with
the network as right preconditioner, and BiCGstab with and without the network
as initial guess: iterations and device time of each.

Usage: python -m paper_2211_06902_gb300.train_net [--out net.bin] [--lattices 5]
       [--sources 16] [--steps 60] [--lr 3e-3]
Prints one JSON line; needs a GPU.
"""

import argparse
import json
import time

import numpy as np


def _cores(L, core=7, frame=1):
    return [[(i * (core + frame), i * (core + frame) + core - 1) for i in range(L[mu] // (core + frame))]
            for mu in range(4)]


def main():
    import torch

    from . import dd4d, synth
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    ap.add_argument("--lattices", type=int, default=5)
    ap.add_argument("--sources", type=int, default=16)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--size", type=int, default=32)
    args = ap.parse_args()
    L = (args.size,) * 4
    kappa = 0.135
    eps_list = [0.40, 0.45, 0.50, 0.55, 0.60][:args.lattices]
    ctx0 = dd4d.Context(L, kappa)
    ctx0.gauge_random(0.5, 2)
    info = ctx0.set_geometry(_cores(L))
    ids = list(range(info["nblocks"]))
    n = info["max_omega"]
    net = dd4d.Net(ctx0, synth.net_init_weights(11))
    train = []
    t0 = time.perf_counter()
    for k, eps in enumerate(eps_list):
        c = dd4d.Context(L, kappa)
        c.gauge_random(eps, 100 + k)
        c.set_geometry(_cores(L))
        gen = torch.Generator(device="cuda")
        gen.manual_seed(100 + k)
        bt = torch.randn((len(ids), args.sources, n, 24), generator=gen, device="cuda",
                         dtype=torch.float64) * (0.5 ** 0.5)
        st = net.train(ids, args.sources, bt, steps=args.steps, lr=args.lr, ctx=c)
        train.append({"eps": eps, "pairs": st["pairs"], "loss_first": st["loss_first"],
                      "loss_last": st["loss_last"], "seconds": st["seconds"]})
        del bt
        c.close()
        torch.cuda.empty_cache()
    train_s = time.perf_counter() - t0
    if args.out:
        net.save(args.out)
    # held-out lattice: the bench batch
    b_h = synth.complex_gaussian(2, synth.TAG_RHS, (len(ids), 12, n, 12))
    b = torch.from_numpy(b_h.view(np.float64)).cuda()
    x = torch.zeros_like(b)
    net.attach(ctx0)
    tol = 1e-10

    def timed(prm):
        ctx0.solve_blocks("omega", ids, 12, b, x, prm)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        st = ctx0.solve_blocks("omega", ids, 12, b, x, prm)
        e1.record()
        torch.cuda.synchronize()
        return {"ms": e0.elapsed_time(e1), "max_iters": st["max_iters"], "max_relres": st["max_relres"],
                "outer_cycles": st["outer_cycles"], "status": st["status"]}
    ab = {
        "bicgstab": timed(dd4d.params(tol, inner_prec="f32", autotune=True)),
        "bicgstab_net_guess": timed(dd4d.params(tol, inner_prec="f32", autotune=True, net_guess=True)),
        "fgmres10": timed(dd4d.params(tol, inner_prec="f32", autotune=True, fgmres=True, restart=10)),
        "fgmres10_net": timed(dd4d.params(tol, inner_prec="f32", autotune=True, fgmres=True, restart=10,
                                          net_precond=True)),
    }
    net.detach(ctx0)
    pairs = sum(t["pairs"] for t in train)
    print(json.dumps({"training": train, "pairs": pairs, "train_seconds": train_s,
                      "pairs_per_s_per_step": pairs * args.steps / train_s,
                      "held_out": ab, "lattice": list(L), "steps_per_lattice": args.steps}))
    net.close()
    ctx0.close()


if __name__ == "__main__":
    main()
