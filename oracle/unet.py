"""FP64 reference of the 3D U-Net used as a learned Krylov initial guess.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain numpy, written from
the definitions of the layers; it shares no code with the CUDA kernels.

Architecture: four levels of widths C = (C1, C2, C3, C4) = (16, 32, 48, 64),
every 3x3x3 convolution 'same' with zero padding and stride 1, ReLU after
every convolution but the last, 2x2x2 average pooling down and nearest
upsampling up, the skip joined after the upsampled channels:

    level 1:  a0 = relu(conv3(x; Cin -> C1))      e1 = relu(conv3(a0; C1 -> C1))
    level 2:  a2 = relu(conv3(pool e1; C1 -> C2))  e2 = relu(conv3(a2; C2 -> C2))
    level 3:  a4 = relu(conv3(pool e2; C2 -> C3))  e3 = relu(conv3(a4; C3 -> C3))
    level 4:  a6 = relu(conv3(pool e3; C3 -> C4))  a7 = relu(conv3(a6; C4 -> C4))
    up 3:     d3 = relu(conv3(relu(conv3([up a7, e3]; C4+C3 -> C3)); C3 -> C3))
    up 2:     d2 = relu(conv3(relu(conv3([up d3, e2]; C3+C2 -> C2)); C2 -> C2))
    up 1:     d1 = relu(conv3(relu(conv3([up d2, e1]; C2+C1 -> C1)); C1 -> C1))
    output:   y  = conv1(d1; C1 -> Cout)
Loss: mean squared error over all output elements.

Parameter layout (flat vector), layer by layer in the order above (15
convolutions): weights [taps][Cout][Cin] (tap t = 9 (dz+1) + 3 (dy+1) + (dx+1)
for the 3x3x3 layers, one tap for the last), then biases [Cout].

Mixed precision (bf16=True), the definition the CUDA network follows:
weights, the network input, every stored activation (after ReLU, pooling,
upsampling) and every gradient signal that enters a convolution's backward
pass are rounded to bfloat16 (nearest, ties to even); all sums are exact here
(FP32 on the GPU); biases, the output, the loss and its gradient stay in full
precision.  With bf16=False every rounding is skipped (the exact network,
used to check the gradient by finite differences).
"""
from __future__ import annotations

import numpy as np

WIDTHS = (16, 32, 48, 64)


def bf16_round(a):
    """Round FP64 values to the nearest bfloat16 (ties to even), as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rounding = ((u >> 16) & 1) + 0x7FFF
    u = ((u + rounding) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def layer_shapes(cin, cout, widths=WIDTHS):
    """(Cin, Cout, taps) of the 15 convolutions in order."""
    c1, c2, c3, c4 = widths
    return [(cin, c1, 27), (c1, c1, 27), (c1, c2, 27), (c2, c2, 27), (c2, c3, 27), (c3, c3, 27),
            (c3, c4, 27), (c4, c4, 27), (c4 + c3, c3, 27), (c3, c3, 27), (c3 + c2, c2, 27), (c2, c2, 27),
            (c2 + c1, c1, 27), (c1, c1, 27), (c1, cout, 1)]


def n_params(cin, cout, widths=WIDTHS):
    return sum(k * co * ci + co for ci, co, k in layer_shapes(cin, cout, widths))


def unpack(theta, cin, cout, widths=WIDTHS):
    out, o = [], 0
    for ci, co, k in layer_shapes(cin, cout, widths):
        w = np.asarray(theta[o:o + k * co * ci], dtype=np.float64).reshape(k, co, ci)
        o += k * co * ci
        b = np.asarray(theta[o:o + co], dtype=np.float64)
        o += co
        out.append((w, b))
    return out


def _taps(k):
    if k == 1:
        return [(0, 0, 0)]
    return [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def conv(x, w, b):
    """out[co, z, y, x] = b[co] + sum_t sum_ci w[t, co, ci] x[ci, z+dz, y+dy, x+dx]."""
    ci, D, H, W = x.shape
    co = w.shape[1]
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1)))
    out = np.empty((co, D, H, W))
    out[:] = b[:, None, None, None]
    for t, (dz, dy, dx) in enumerate(_taps(w.shape[0])):
        sh = xp[:, 1 + dz:1 + dz + D, 1 + dy:1 + dy + H, 1 + dx:1 + dx + W]
        out += np.einsum("oc,czyx->ozyx", w[t], sh)
    return out


def conv_backward(x, w, gout):
    """Gradients of sum(gout * conv(x, w, b)) with respect to x, w, b."""
    ci, D, H, W = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1)))
    gxp = np.zeros_like(xp)
    gw = np.zeros_like(w)
    for t, (dz, dy, dx) in enumerate(_taps(w.shape[0])):
        sh = xp[:, 1 + dz:1 + dz + D, 1 + dy:1 + dy + H, 1 + dx:1 + dx + W]
        gw[t] = np.einsum("ozyx,czyx->oc", gout, sh)
        gxp[:, 1 + dz:1 + dz + D, 1 + dy:1 + dy + H, 1 + dx:1 + dx + W] += np.einsum("oc,ozyx->czyx", w[t], gout)
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


def _params(theta, cin, cout, widths, bf16):
    layers = unpack(theta, cin, cout, widths)
    if bf16:
        layers = [(bf16_round(w), b) for w, b in layers]
    return layers


def forward(theta, x, cin, cout, widths=WIDTHS, bf16=True):
    """Output y [Cout, D, H, W] and the activations needed by the backward pass."""
    r = bf16_round if bf16 else (lambda a: a)
    P = _params(theta, cin, cout, widths, bf16)
    relu = lambda a: np.maximum(a, 0.0)    # noqa: E731
    act = {}
    act["x"] = r(np.asarray(x, dtype=np.float64))
    act["a0"] = r(relu(conv(act["x"], *P[0])))
    act["e1"] = r(relu(conv(act["a0"], *P[1])))
    act["p1"] = r(pool(act["e1"]))
    act["a2"] = r(relu(conv(act["p1"], *P[2])))
    act["e2"] = r(relu(conv(act["a2"], *P[3])))
    act["p2"] = r(pool(act["e2"]))
    act["a4"] = r(relu(conv(act["p2"], *P[4])))
    act["e3"] = r(relu(conv(act["a4"], *P[5])))
    act["p3"] = r(pool(act["e3"]))
    act["a6"] = r(relu(conv(act["p3"], *P[6])))
    act["a7"] = r(relu(conv(act["a6"], *P[7])))
    act["c3"] = np.concatenate([upsample(act["a7"]), act["e3"]], axis=0)
    act["d3a"] = r(relu(conv(act["c3"], *P[8])))
    act["d3"] = r(relu(conv(act["d3a"], *P[9])))
    act["c2"] = np.concatenate([upsample(act["d3"]), act["e2"]], axis=0)
    act["d2a"] = r(relu(conv(act["c2"], *P[10])))
    act["d2"] = r(relu(conv(act["d2a"], *P[11])))
    act["c1"] = np.concatenate([upsample(act["d2"]), act["e1"]], axis=0)
    act["d1a"] = r(relu(conv(act["c1"], *P[12])))
    act["d1"] = r(relu(conv(act["d1a"], *P[13])))
    y = conv(act["d1"], *P[14])
    return y, (act, P)


def loss_and_grad(theta, x, target, cin, cout, widths=WIDTHS, bf16=True):
    """MSE loss and its gradient with respect to the flat parameter vector."""
    r = bf16_round if bf16 else (lambda a: a)
    y, (act, P) = forward(theta, x, cin, cout, widths, bf16)
    diff = y - np.asarray(target, dtype=np.float64)
    loss = float(np.mean(diff ** 2))
    gy = 2.0 * diff / diff.size
    grads = [None] * 15

    def back(l, inp, g_signal):
        """Layer l's parameter gradients from its input and the (rounded)
        gradient signal at its output; returns the input gradient."""
        gin, gw, gb = conv_backward(inp, P[l][0], g_signal)
        grads[l] = (gw, gb)
        return gin

    mask = lambda g, a: r(g * (a > 0))    # noqa: E731
    g = back(14, act["d1"], gy)                      # 1x1 output layer (full-precision signal)
    g = back(13, act["d1a"], mask(g, act["d1"]))
    g_c1 = back(12, act["c1"], mask(g, act["d1a"]))
    c1, c2, c3, _ = widths
    g_e1 = g_c1[c2:].copy()
    g = upsample_backward(g_c1[:c2])
    g = back(11, act["d2a"], mask(g, act["d2"]))
    g_c2 = back(10, act["c2"], mask(g, act["d2a"]))
    g_e2 = g_c2[c3:].copy()
    g = upsample_backward(g_c2[:c3])
    g = back(9, act["d3a"], mask(g, act["d3"]))
    g_c3 = back(8, act["c3"], mask(g, act["d3a"]))
    g_e3 = g_c3[widths[3]:].copy()
    g = upsample_backward(g_c3[:widths[3]])
    g = back(7, act["a6"], mask(g, act["a7"]))
    g = back(6, act["p3"], mask(g, act["a6"]))
    g_e3 += pool_backward(g)
    g = back(5, act["a4"], mask(g_e3, act["e3"]))
    g = back(4, act["p2"], mask(g, act["a4"]))
    g_e2 += pool_backward(g)
    g = back(3, act["a2"], mask(g_e2, act["e2"]))
    g = back(2, act["p1"], mask(g, act["a2"]))
    g_e1 += pool_backward(g)
    g = back(1, act["a0"], mask(g_e1, act["e1"]))
    back(0, act["x"], mask(g, act["a0"]))
    flat = np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in grads])
    return loss, flat
