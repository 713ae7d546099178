"""Learned correction network on the AIM grid. Test infrastructure (oracle), FP64.

Not in the paper: the learned preconditioner is an extension of its preconditioned solve
(Sec. II-C). The network is a 4-layer 3-D convolutional net on the AIM grid, 3x3x3 kernels,
zero padding, no biases (so net(a x) = a net(x) for a > 0), ReLU between layers, channels
8 -> 16 -> 16 -> 16 -> 8. Its input is the projected residual P r split into Re/Im of the four
grid components (x, y, z RWG components and the charge), scaled by the RMS of the grid; the
output, scaled back, is interpolated with W = P^T to a correction in unknown space:
  M(r) = M_bd r + W net(P r).
Training minimises the grid-projected relative error |P (W net(P r) - t)|^2 / |P t|^2 with
t = A^{-1} r - M_bd r over pairs r = A x (reading: the block-diagonal part leaves mesh-scale
error modes no grid field can represent; the network acts as a grid-level correction).

Layouts: activations [C, nz, ny, nx]; weights [C_out, C_in, 3, 3, 3] indexed (dz, dy, dx).
"""
from __future__ import annotations

import numpy as np

CHANNELS = (8, 16, 16, 16, 8)


def conv3d(x, w):
    """y[o, p] = sum_i sum_d w[o, i, d] x[i, p + d - 1] (zero padding), d = (dz, dy, dx)."""
    ci, Z, Y, X = x.shape
    xp = np.zeros((ci, Z + 2, Y + 2, X + 2), dtype=x.dtype)
    xp[:, 1:-1, 1:-1, 1:-1] = x
    out = np.zeros((w.shape[0], Z, Y, X), dtype=np.result_type(x, w))
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                out += np.einsum("oi,izyx->ozyx", w[:, :, dz, dy, dx],
                                 xp[:, dz:dz + Z, dy:dy + Y, dx:dx + X])
    return out


def conv3d_grad_input(g, w):
    """dL/dx for y = conv3d(x, w) given g = dL/dy."""
    co, Z, Y, X = g.shape
    gp = np.zeros((co, Z + 2, Y + 2, X + 2), dtype=g.dtype)
    gp[:, 1:-1, 1:-1, 1:-1] = g
    out = np.zeros((w.shape[1], Z, Y, X), dtype=np.result_type(g, w))
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                # x[i, p] feeds y[o, p - d + 1]
                out += np.einsum("oi,ozyx->izyx", w[:, :, dz, dy, dx],
                                 gp[:, 2 - dz:2 - dz + Z, 2 - dy:2 - dy + Y, 2 - dx:2 - dx + X])
    return out


def conv3d_grad_weight(x, g):
    """dL/dw for y = conv3d(x, w) given g = dL/dy."""
    ci, Z, Y, X = x.shape
    xp = np.zeros((ci, Z + 2, Y + 2, X + 2), dtype=x.dtype)
    xp[:, 1:-1, 1:-1, 1:-1] = x
    gw = np.zeros((g.shape[0], ci, 3, 3, 3), dtype=np.result_type(x, g))
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                gw[:, :, dz, dy, dx] = np.einsum("ozyx,izyx->oi", g,
                                                 xp[:, dz:dz + Z, dy:dy + Y, dx:dx + X])
    return gw


def forward(x, ws, store=None):
    """Returns the list of activations [x, h1, h2, h3, out]. `store`, if given, is applied to
    each hidden activation after the ReLU (the storage format of the activations, e.g. BF16
    rounding), so that the ReLU masks and the next layer see what the kernels keep."""
    acts = [x]
    h = x
    for l, w in enumerate(ws):
        h = conv3d(h, w)
        if l < len(ws) - 1:
            h = np.maximum(h, 0.0)
            if store is not None:
                h = store(h)
        acts.append(h)
    return acts


def backward(acts, ws, gout):
    """Gradients (weights list, input) of L given gout = dL/d(out)."""
    gws = [None] * len(ws)
    g = gout
    for l in range(len(ws) - 1, -1, -1):
        gws[l] = conv3d_grad_weight(acts[l], g)
        g = conv3d_grad_input(g, ws[l])
        if l > 0:
            g = g * (acts[l] > 0)
    return gws, g


def init_weights(seed):
    """He-normal initialisation (std sqrt(2 / (27 C_in)))."""
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((co, ci, 3, 3, 3)) * np.sqrt(2.0 / (27 * ci))
            for ci, co in zip(CHANNELS[:-1], CHANNELS[1:])]


def flatten(ws):
    return np.concatenate([w.ravel() for w in ws])


def unflatten(v):
    out, o = [], 0
    for ci, co in zip(CHANNELS[:-1], CHANNELS[1:]):
        n = co * ci * 27
        out.append(np.asarray(v[o:o + n]).reshape(co, ci, 3, 3, 3))
        o += n
    return out
