"""Gauge-covariant parallel-transport convolution network (oracle, FP64, CPU).

Test infrastructure only (see the package docstring).

The learned block preconditioner is a stack of linear parallel-transport
convolutions acting on one framed block Omega (Dirichlet boundary).  A field
phi has C channels, each a colour 3-vector per site.  With the transports
    (T_0 phi)(x)   = phi(x),
    (T_+mu phi)(x) = U_mu(x) phi(x + mu)          (0 if x + mu is outside Omega),
    (T_-mu phi)(x) = U_mu(x - mu)^+ phi(x - mu)   (0 if x - mu is outside Omega),
where the links carry the same time-boundary sign as D, one layer is
    y_c(x) = sum_{d in {0, +-mu}} sum_c' W[d, c, c'] (T_d phi_c')(x)
with complex weights W (9 directions, C_out x C_in).  Because W never touches
colour, the layer is gauge covariant: (U, phi) -> (U^g, g phi) maps y -> g y.
The network maps a right-hand side b (4 spin channels) through channels
4 -> 16 -> 16 -> 16 -> 4 to an approximation of D_Omega^{-1} b and is trained
on pairs (b, D_Omega^{-1} b) with the loss
    L = (1/S) sum_s |N(b_s) - x_s|^2 / |x_s|^2.
Gradients use the convention g = dL/dRe + i dL/dIm; for a layer y = W T phi:
    g_phi_c' = sum_d sum_c conj(W[d, c, c']) T_d^+ g_y_c,   T_+mu^+ = T_-mu,
    g_W[d, c, c'] = sum_x sum_a g_y_c(x)_a conj((T_d phi_c')(x)_a).
"""

import numpy as np

DIRS = [None, (0, 1), (1, 1), (2, 1), (3, 1), (0, -1), (1, -1), (2, -1), (3, -1)]
CHANNELS = (4, 16, 16, 16, 4)


def box_links(U, origin, side, time_bc=-1):
    """Links of a box (local coords) with the time-boundary sign folded in:
    returns fwd[mu] = U_mu(x) at each box site, shape [side..., 4, 3, 3]."""
    L = U.shape[:4]
    idx = np.indices(side)
    g = [(origin[m] + idx[m]) % L[m] for m in range(4)]
    Ub = U[g[0], g[1], g[2], g[3]].copy()
    t_last = (g[0] == L[0] - 1)
    Ub[..., 0, :, :][t_last] *= time_bc
    return Ub


def transport(Ub, phi, d):
    """T_d phi for phi of shape [side..., 3] (box, Dirichlet)."""
    if d is None:
        return phi.copy()
    mu, step = d
    out = np.zeros_like(phi)
    n = phi.shape[mu]
    sl_all = [slice(None)] * 4
    if step == 1:
        dst = list(sl_all); dst[mu] = slice(0, n - 1)
        src = list(sl_all); src[mu] = slice(1, n)
        out[tuple(dst)] = np.einsum("...ab,...b->...a", Ub[tuple(dst)][..., mu, :, :], phi[tuple(src)])
    else:
        dst = list(sl_all); dst[mu] = slice(1, n)
        src = list(sl_all); src[mu] = slice(0, n - 1)
        out[tuple(dst)] = np.einsum("...ba,...b->...a", np.conj(Ub[tuple(src)][..., mu, :, :]),
                                    phi[tuple(src)])
    return out


def layer(Ub, W, phi):
    """phi: [C_in, side..., 3] -> [C_out, side..., 3]."""
    cout = W.shape[1]
    y = np.zeros((cout,) + phi.shape[1:], dtype=np.complex128)
    for k, d in enumerate(DIRS):
        T = np.stack([transport(Ub, phi[c], d) for c in range(phi.shape[0])])
        y += np.einsum("oi,i...->o...", W[k], T)
    return y


def layer_adjoint(Ub, W, g):
    """g_phi from g_y: sum_d conj(W_d)^T T_d^+ g."""
    cin = W.shape[2]
    out = np.zeros((cin,) + g.shape[1:], dtype=np.complex128)
    for k, d in enumerate(DIRS):
        dadj = None if d is None else (d[0], -d[1])
        T = np.stack([transport(Ub, g[c], dadj) for c in range(g.shape[0])])
        out += np.einsum("oi,o...->i...", np.conj(W[k]), T)
    return out


def layer_weight_grad(Ub, phi, g):
    """g_W[d, c, c'] = sum_x g_c(x) . conj(T_d phi_c'(x))."""
    G = np.zeros((9, g.shape[0], phi.shape[0]), dtype=np.complex128)
    for k, d in enumerate(DIRS):
        T = np.stack([transport(Ub, phi[c], d) for c in range(phi.shape[0])])
        G[k] = g.reshape(g.shape[0], -1) @ np.conj(T.reshape(T.shape[0], -1)).T
    return G


def spin_channels(b, side):
    """[nsites*12] (site-major, 12 = 3*spin + colour) -> [4, side..., 3]."""
    return np.moveaxis(b.reshape(tuple(side) + (4, 3)), 4, 0)


def from_channels(phi):
    return np.moveaxis(phi, 0, 4).reshape(-1)


def forward(Ub, Ws, b, side):
    """Network output and the per-layer inputs (for backprop)."""
    acts = [spin_channels(b, side)]
    for W in Ws:
        acts.append(layer(Ub, W, acts[-1]))
    return from_channels(acts[-1]), acts


def loss_and_grads(Ub, Ws, pairs, side):
    """L and dL/dW (convention dL/dRe + i dL/dIm) over (b, x) pairs."""
    S = len(pairs)
    L = 0.0
    grads = [np.zeros_like(W) for W in Ws]
    for b, x in pairs:
        y, acts = forward(Ub, Ws, b, side)
        nx = np.vdot(x, x).real
        L += np.vdot(y - x, y - x).real / nx / S
        g = spin_channels(2.0 * (y - x) / nx / S, side)
        for l in range(len(Ws) - 1, -1, -1):
            grads[l] += layer_weight_grad(Ub, acts[l], g)
            g = layer_adjoint(Ub, Ws[l], g)
    return L, grads


def init_weights(seed, channels=CHANNELS):
    """Seeded initial weights (an input, drawn by the shared input generators)."""
    from paper_2211_06902_gb300 import synth
    return synth.net_init_weights(seed, channels)
