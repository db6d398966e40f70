"""FP64 reference of the small 3D U-Net used as a learned Krylov initial guess.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain numpy, written from
the definitions of the layers; it shares no code with the CUDA kernels.

Architecture (all convolutions 'same' with zero padding, stride 1):
    e1 = relu(conv3(x;  Cin -> C1))
    p1 = avgpool2(e1)                      2x2x2 mean, even grid sizes
    e2 = relu(conv3(p1; C1 -> C2))
    u2 = upsample2(e2)                     nearest neighbour
    d1 = relu(conv3([e1, u2]; C1+C2 -> C1))
    y  = conv1(d1; C1 -> Cout)
Loss: mean squared error over all output elements.
Parameter layout (flat vector): for each layer in order (conv a, conv b,
conv c, conv d): weights [Co][Ci][k^3] then biases [Co].
"""
from __future__ import annotations

import numpy as np


def layer_shapes(cin, c1, c2, cout):
    return [(c1, cin, 27), (c2, c1, 27), (c1, c1 + c2, 27), (cout, c1, 1)]


def n_params(cin, c1, c2, cout):
    return sum(co * ci * k + co for co, ci, k in layer_shapes(cin, c1, c2, cout))


def unpack(theta, cin, c1, c2, cout):
    out, o = [], 0
    for co, ci, k in layer_shapes(cin, c1, c2, cout):
        w = theta[o:o + co * ci * k].reshape(co, ci, k)
        o += co * ci * k
        b = theta[o:o + co]
        o += co
        out.append((w, b))
    return out


def _taps(k):
    if k == 1:
        return [(0, 0, 0)]
    return [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def conv(x, w, b):
    """out[co, z, y, x] = b[co] + sum_ci sum_taps w[co, ci, t] x[ci, z+dz, y+dy, x+dx]."""
    ci, D, H, W = x.shape
    co = w.shape[0]
    taps = _taps(w.shape[2])
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1)))
    out = np.empty((co, D, H, W))
    out[:] = b[:, None, None, None]
    for t, (dz, dy, dx) in enumerate(taps):
        sh = xp[:, 1 + dz:1 + dz + D, 1 + dy:1 + dy + H, 1 + dx:1 + dx + W]
        out += np.einsum("oc,czyx->ozyx", w[:, :, t], sh)
    return out


def conv_backward(x, w, gout):
    """Gradients of sum(gout * conv(x, w, b)) with respect to x, w, b."""
    ci, D, H, W = x.shape
    taps = _taps(w.shape[2])
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1)))
    gxp = np.zeros_like(xp)
    gw = np.zeros_like(w)
    for t, (dz, dy, dx) in enumerate(taps):
        sh = xp[:, 1 + dz:1 + dz + D, 1 + dy:1 + dy + H, 1 + dx:1 + dx + W]
        gw[:, :, t] = np.einsum("ozyx,czyx->oc", gout, sh)
        gxp[:, 1 + dz:1 + dz + D, 1 + dy:1 + dy + H, 1 + dx:1 + dx + W] += np.einsum("oc,ozyx->czyx", w[:, :, t], gout)
    gb = gout.sum(axis=(1, 2, 3))
    return gxp[:, 1:-1, 1:-1, 1:-1], gw, gb


def pool(x):
    c, D, H, W = x.shape
    return x.reshape(c, D // 2, 2, H // 2, 2, W // 2, 2).mean(axis=(2, 4, 6))


def pool_backward(g):
    return np.repeat(np.repeat(np.repeat(g, 2, axis=1), 2, axis=2), 2, axis=3) / 8.0


def upsample(x):
    return np.repeat(np.repeat(np.repeat(x, 2, axis=1), 2, axis=2), 2, axis=3)


def upsample_backward(g):
    c, D, H, W = g.shape
    return g.reshape(c, D // 2, 2, H // 2, 2, W // 2, 2).sum(axis=(2, 4, 6))


def forward(theta, x, dims):
    cin, c1, c2, cout = dims
    (wa, ba), (wb, bb), (wc, bc), (wd, bd) = unpack(theta, cin, c1, c2, cout)
    a1 = conv(x, wa, ba)
    e1 = np.maximum(a1, 0)
    p1 = pool(e1)
    a2 = conv(p1, wb, bb)
    e2 = np.maximum(a2, 0)
    u2 = upsample(e2)
    cat = np.concatenate([e1, u2], axis=0)
    a3 = conv(cat, wc, bc)
    d1 = np.maximum(a3, 0)
    y = conv(d1, wd, bd)
    cache = (x, a1, e1, p1, a2, e2, cat, a3, d1)
    return y, cache


def loss_and_grad(theta, x, target, dims):
    """MSE loss and its gradient with respect to the flat parameter vector."""
    cin, c1, c2, cout = dims
    (wa, ba), (wb, bb), (wc, bc), (wd, bd) = unpack(theta, cin, c1, c2, cout)
    y, (x, a1, e1, p1, a2, e2, cat, a3, d1) = forward(theta, x, dims)
    diff = y - target
    loss = float(np.mean(diff ** 2))
    gy = 2.0 * diff / diff.size
    gd1, gwd, gbd = conv_backward(d1, wd, gy)
    ga3 = gd1 * (a3 > 0)
    gcat, gwc, gbc = conv_backward(cat, wc, ga3)
    ge1 = gcat[:c1].copy()
    gu2 = gcat[c1:]
    ge2 = upsample_backward(gu2)
    ga2 = ge2 * (a2 > 0)
    gp1, gwb, gbb = conv_backward(p1, wb, ga2)
    ge1 += pool_backward(gp1)
    ga1 = ge1 * (a1 > 0)
    _, gwa, gba = conv_backward(x, wa, ga1)
    g = np.concatenate([gwa.ravel(), gba, gwb.ravel(), gbb, gwc.ravel(), gbc, gwd.ravel(), gbd])
    return loss, g


def bf16_round(a):
    """Round FP64 values to the nearest bfloat16 (ties to even), as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rounding = ((u >> 16) & 1) + 0x7FFF
    u = ((u + rounding) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
