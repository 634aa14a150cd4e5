"""Learned refinement proposal: block summaries and the per-block MLP.  Test
infrastructure only.

Not part of the paper: the library adds a small network that proposes
refinement ahead of the vorticity criterion (Section 4.4), with the plain
criterion kept as the fallback.  This module is the plain restatement used to
check the CUDA kernels.

Block summaries (27 per block, after the level synchronisation), with
G_ab = du_a/dx_b from block-local first-order differences in physical units
(forward, backward at the last cell, dx_L = length_x / (nx 2^L)):
  0..8    mean of G_ab (a-major), compressed as sign(x) log(1 + |x|)
  9..17   max |G_ab|, compressed
  18      (mean rho - 1) * 100
  19      (max rho - min rho) * 100
  20..22  mean u_x, u_y, u_z, times 20
  23      max |u|, times 20
  24, 25  mean and max |w| (w = curl u), compressed
  26      level / L_max

MLP: p = sigmoid(w3 . relu(W2 relu(W1 x + b1) + b2) + b3); parameters packed
W1[64][27], b1[64], W2[64][64], b2[64], w3[64], b3.  Loss per sample:
pw y softplus(-z) + (1 - y) softplus(z).
"""
import numpy as np

from .lattice import moments

IN, H = 27, 64
NP = H * IN + H + H * H + H + H + 1


def squash(x):
    return np.sign(x) * np.log1p(np.abs(x))


def block_features(lbm, b):
    """27 summaries of block b of a ForestLBM (3D)."""
    rho, u = moments(lbm.vs, lbm.f[b])                  # [64], [64, 3]
    L = int(lbm.mesh.level[b])
    dx = lbm.cfg["length_x"] / (lbm.cfg["nx"] * 2.0 ** L)
    ug = u.reshape(4, 4, 4, 3)                         # [k][j][i][a]

    def diff(axis):                                     # axis 0 = x (array axis 2)
        ax = 2 - axis
        fwd = np.diff(ug, axis=ax)
        last = np.take(fwd, [2], axis=ax)
        return np.concatenate([fwd, last], axis=ax) / dx

    d = [diff(0), diff(1), diff(2)]                     # d[b][..., a] = du_a/dx_b
    G = np.stack([np.stack([d[bb][..., a] for bb in range(3)], -1) for a in range(3)], -2)
    G = G.reshape(64, 3, 3)                             # [cell][a][b]
    w = np.stack([G[:, 2, 1] - G[:, 1, 2], G[:, 0, 2] - G[:, 2, 0], G[:, 1, 0] - G[:, 0, 1]], -1)
    wn = np.sqrt((w * w).sum(-1))
    out = np.zeros(IN)
    Gf = G.reshape(64, 9)
    out[0:9] = squash(Gf.mean(0))
    out[9:18] = squash(np.abs(Gf).max(0))
    out[18] = (rho.mean() - 1.0) * 100.0
    out[19] = (rho.max() - rho.min()) * 100.0
    out[20:23] = u.mean(0) * 20.0
    out[23] = np.sqrt((u * u).sum(-1)).max() * 20.0
    out[24] = squash(wn.mean())
    out[25] = squash(wn.max())
    out[26] = L / lbm.mesh.lmax
    return out


def unpack(params):
    p = np.asarray(params, np.float64)
    o = 0
    W1 = p[o:o + H * IN].reshape(H, IN); o += H * IN
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    w3 = p[o:o + H]; o += H
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def forward(params, x):
    """Logits z and probabilities p for samples x [n, 27]."""
    W1, b1, W2, b2, w3, b3 = unpack(params)
    h1 = np.maximum(x @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    z = h2 @ w3 + b3
    return z, 1.0 / (1.0 + np.exp(-z))


def softplus(t):
    return np.where(t > 0, t + np.log1p(np.exp(-np.abs(t))), np.log1p(np.exp(t)))


def loss_and_grad(params, x, y, pos_weight=1.0):
    """Summed loss and summed gradient (flat, the packing above) by the chain
    rule written out layer by layer."""
    W1, b1, W2, b2, w3, b3 = unpack(params)
    a1 = x @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    z = h2 @ w3 + b3
    p = 1.0 / (1.0 + np.exp(-z))
    loss = np.sum(pos_weight * y * softplus(-z) + (1.0 - y) * softplus(z))
    dz = pos_weight * y * (p - 1.0) + (1.0 - y) * p      # d loss / d z
    gw3 = h2.T @ dz
    gb3 = dz.sum()
    dh2 = np.outer(dz, w3) * (a2 > 0)
    gW2 = dh2.T @ h1
    gb2 = dh2.sum(0)
    dh1 = (dh2 @ W2) * (a1 > 0)
    gW1 = dh1.T @ x
    gb1 = dh1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gw3, [gb3]])
    return loss, g
