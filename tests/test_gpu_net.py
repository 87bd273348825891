"""GPU parallel-transport network: forward and gradients vs the FP64 oracle,
training on solver-generated pairs, and its use as the block-solve initial guess.

The oracle evaluates the same (BF16-rounded) weights in FP64.  On the FP32
CUDA cores the GPU keeps FP32 activations, so forward outputs agree to ~1e-6 and
gradients to ~1e-5 relative (tolerances 2e-5 and 2e-4, norm-wise).  On the
tensor cores (tcgen05, the default) the parallel-transported activations enter
each layer's contraction rounded to BF16 (unit roundoff 2^-9 = 2e-3) with FP32
accumulation: four layers give at most ~4 x 2e-3 relative, tolerance 2e-2.
"""

import numpy as np
import pytest

from paper_2211_06902_gb300 import dd4d, synth
from oracle import net as onet

from gpu_common import config1, relerr, to_field

pytestmark = pytest.mark.gpu


def bf16(w):
    """Round-to-nearest-even to BF16 (what the kernels use)."""
    def r(x):
        u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
        u = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
        return u.view(np.float32).astype(np.float64)
    return r(w.real) + 1j * r(w.imag)


@pytest.fixture(scope="module")
def case():
    U, ctx, info, geo = config1()
    Ws = onet.init_weights(3)
    Ws = [w + 0.05 * synth.complex_gaussian(3, 200 + k, w.shape) for k, w in enumerate(Ws)]
    return U, ctx, info, geo, Ws


def _block(ctx, U, b):
    g = ctx.geom_block(b)
    return onet.box_links(U, g["origin"], g["side"]), tuple(g["side"])


def test_forward_matches_oracle(case):
    torch = pytest.importorskip("torch")
    U, ctx, info, geo, Ws = case
    net = dd4d.Net(ctx, Ws)
    net.tensor_cores(False)
    ids, nrhs = [0, 9], 2
    n = len(ctx.geom_sites(dd4d.SET_OMEGA, 0))
    b = synth.complex_gaussian(4, synth.TAG_RHS, (len(ids), nrhs, n, 12))
    db = torch.from_numpy(b.view(np.float64).copy()).cuda()
    dy = torch.zeros_like(db)
    net.apply(ids, nrhs, db, dy)
    y = dy.cpu().numpy().view(np.complex128)
    Wr = [bf16(w) for w in Ws]
    for k, blk in enumerate(ids):
        Ub, side = _block(ctx, U, blk)
        for r in range(nrhs):
            ref, _ = onet.forward(Ub, Wr, b[k, r].ravel(), side)
            assert relerr(y[k, r].ravel(), ref) < 2e-5


@pytest.mark.parametrize("ids", [[0, 9], [5]])
def test_tensor_core_forward_matches_oracle(case, ids):
    """The tcgen05 layers (BF16 operands, FP32 accumulation in tensor memory) against
    the FP64 oracle and against the FP32 CUDA-core layers, on every site of two
    framed blocks (5^4 sites: work items with a ragged last quarter)."""
    torch = pytest.importorskip("torch")
    U, ctx, info, geo, Ws = case
    net = dd4d.Net(ctx, Ws)
    nrhs = 3
    n = len(ctx.geom_sites(dd4d.SET_OMEGA, 0))
    b = synth.complex_gaussian(7, synth.TAG_RHS, (len(ids), nrhs, n, 12))
    db = torch.from_numpy(b.view(np.float64).copy()).cuda()
    dy = torch.full_like(db, float("nan"))
    net.apply(ids, nrhs, db, dy)
    net.tensor_cores(False)
    dz = torch.zeros_like(db)
    net.apply(ids, nrhs, db, dz)
    y = dy.cpu().numpy().view(np.complex128)
    z = dz.cpu().numpy().view(np.complex128)
    assert np.all(np.isfinite(y))
    Wr = [bf16(w) for w in Ws]
    for k, blk in enumerate(ids):
        Ub, side = _block(ctx, U, blk)
        for r in range(nrhs):
            ref, _ = onet.forward(Ub, Wr, b[k, r].ravel(), side)
            e = relerr(y[k, r].ravel(), ref)
            assert 1e-7 < e < 2e-2, e            # BF16 operands: close, but not the FP32 result
            assert relerr(z[k, r].ravel(), ref) < 2e-5
    assert relerr(y, z) < 2e-2


def test_gradients_match_oracle(case):
    torch = pytest.importorskip("torch")
    U, ctx, info, geo, Ws = case
    net = dd4d.Net(ctx, Ws)
    net.tensor_cores(False)
    ids, nrhs = [2, 13], 2
    n = len(ctx.geom_sites(dd4d.SET_OMEGA, 0))
    b = synth.complex_gaussian(5, synth.TAG_RHS, (len(ids), nrhs, n, 12))
    x = synth.complex_gaussian(6, synth.TAG_RHS, (len(ids), nrhs, n, 12))
    L, G = net.loss_grad(ids, nrhs, torch.from_numpy(b.view(np.float64).copy()).cuda(),
                         torch.from_numpy(x.view(np.float64).copy()).cuda())
    Wr = [bf16(w) for w in Ws]
    L0, G0 = 0.0, [np.zeros_like(w) for w in Ws]
    for k, blk in enumerate(ids):
        Ub, side = _block(ctx, U, blk)
        l, g = onet.loss_and_grads(Ub, Wr, [(b[k, r].ravel(), x[k, r].ravel()) for r in range(nrhs)],
                                   side)
        L0 += l / len(ids)
        for q in range(len(G0)):
            G0[q] += g[q] / len(ids)
    assert abs(L - L0) < 2e-5 * L0
    for g, g0 in zip(G, G0):
        assert relerr(g, g0) < 2e-4


def test_training_and_initial_guess():
    """Training lowers the loss; the trained network as initial guess keeps every
    system at 1e-10 (oracle-checked residuals) and its effect is reported."""
    torch = pytest.importorskip("torch")
    from oracle.lattice import apply_D_restricted
    U, ctx, info, geo = config1()
    net = dd4d.Net(ctx, onet.init_weights(7))
    ids = list(range(info["nblocks"]))
    n = len(ctx.geom_sites(dd4d.SET_OMEGA, 0))
    bt = synth.complex_gaussian(7, synth.TAG_RHS, (len(ids), 4, n, 12))
    st = net.train(ids, 4, torch.from_numpy(bt.view(np.float64).copy()).cuda(), steps=60, lr=3e-3)
    assert st["loss_last"] < 0.7 * st["loss_first"], st
    net.attach()
    b = synth.complex_gaussian(8, synth.TAG_RHS, (len(ids), 2, n, 12))
    x0 = np.zeros_like(b)
    x1 = np.zeros_like(b)
    s0 = ctx.solve_blocks("omega", ids, 2, b, x0, dd4d.params(1e-10, inner_prec="f32"))
    s1 = ctx.solve_blocks("omega", ids, 2, b, x1, dd4d.params(1e-10, inner_prec="f32",
                                                               net_guess=True))
    assert s0["status"] == s1["status"] == 0
    assert s1["max_iters"] <= s0["max_iters"] + 2
    L = geo.L
    for blk in (0, 7, 15):
        sites = ctx.geom_sites(dd4d.SET_OMEGA, blk)
        for r in range(2):
            f = to_field(L, sites, b[blk, r])
            res = f - apply_D_restricted(U, to_field(L, sites, x1[blk, r]), 0.13, geo.omega_mask[blk])
            assert np.linalg.norm(res) <= 1e-10 * np.linalg.norm(f) * 1.0000001
    net.detach()


def test_network_as_fgmres_preconditioner():
    """The trained network as the variable right preconditioner of FGMRES (FP32
    inner solves): every system still reaches 1e-10 against the oracle's D_Omega,
    and the iteration counts with and without the network are recorded (the
    benchmark reports their times)."""
    torch = pytest.importorskip("torch")
    from oracle.lattice import apply_D_restricted
    U, ctx, info, geo = config1()
    net = dd4d.Net(ctx, onet.init_weights(7))
    ids = list(range(info["nblocks"]))
    n = len(ctx.geom_sites(dd4d.SET_OMEGA, 0))
    bt = synth.complex_gaussian(17, synth.TAG_RHS, (len(ids), 4, n, 12))
    net.train(ids, 4, torch.from_numpy(bt.view(np.float64).copy()).cuda(), steps=80, lr=3e-3)
    net.attach()
    b = synth.complex_gaussian(18, synth.TAG_RHS, (len(ids), 2, n, 12))
    x0, x1 = np.zeros_like(b), np.zeros_like(b)
    s0 = ctx.solve_blocks("omega", ids, 2, b, x0, dd4d.params(1e-10, inner_prec="f32", fgmres=True, restart=10))
    s1 = ctx.solve_blocks("omega", ids, 2, b, x1, dd4d.params(1e-10, inner_prec="f32", fgmres=True, restart=10,
                                                               net_precond=True))
    assert s0["status"] == s1["status"] == 0
    assert s1["max_relres"] <= 1e-10
    print("FGMRES iterations without / with the network:", s0["max_iters"], s1["max_iters"])
    L = geo.L
    for blk in (0, 7, 15):
        sites = ctx.geom_sites(dd4d.SET_OMEGA, blk)
        for r in range(2):
            f = to_field(L, sites, b[blk, r])
            res = f - apply_D_restricted(U, to_field(L, sites, x1[blk, r]), 0.13, geo.omega_mask[blk])
            assert np.linalg.norm(res) <= 1e-10 * np.linalg.norm(f) * 1.0000001
    net.detach()


def test_save_and_load_resume_exactly(tmp_path):
    """A saved network loads with the same weights and Adam state: it applies
    identically and a further training step gives identical weights."""
    torch = pytest.importorskip("torch")
    U, ctx, info, geo = config1()
    ids = list(range(4))
    n = len(ctx.geom_sites(dd4d.SET_OMEGA, 0))
    bt = torch.from_numpy(synth.complex_gaussian(9, synth.TAG_RHS, (len(ids), 2, n, 12))
                          .view(np.float64).copy()).cuda()
    net = dd4d.Net(ctx, onet.init_weights(5))
    net.train(ids, 2, bt, steps=3, lr=3e-3)
    path = tmp_path / "net.bin"
    net.save(path)
    other = dd4d.Net.load(ctx, path)
    assert other.channels == net.channels
    for a, b in zip(net.weights(), other.weights()):
        assert np.array_equal(a, b)
    b = torch.from_numpy(synth.complex_gaussian(10, synth.TAG_RHS, (len(ids), 2, n, 12))
                         .view(np.float64).copy()).cuda()
    ya, yb = torch.zeros_like(b), torch.zeros_like(b)
    net.apply(ids, 2, b, ya)
    other.apply(ids, 2, b, yb)
    torch.cuda.synchronize()
    assert torch.equal(ya, yb) and float(ya.abs().max()) > 0
    net.train(ids, 2, bt, steps=2, lr=3e-3)
    other.train(ids, 2, bt, steps=2, lr=3e-3)
    for a, b in zip(net.weights(), other.weights()):
        assert np.array_equal(a, b)
    bad = tmp_path / "bad.bin"
    bad.write_bytes(b"not a network")
    with pytest.raises(dd4d.DDError) as e:
        dd4d.Net.load(ctx, bad)
    assert e.value.status == dd4d.DD_EINVAL
