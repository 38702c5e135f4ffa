"""Plain numpy FP64 reference for the warm-start U-Net (forward, loss, gradients, Adam).

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark baseline).  It shares no
code with the CUDA library.  Same architecture and parameter layout as the
library's network: for width w, layers
    enc1a 1->w, enc1b w->w, enc2a w->2w, enc2b 2w->2w, bota 2w->4w, botb 4w->4w,
    dec2a 6w->2w, dec2b 2w->2w, dec1a 3w->w, dec1b w->w, out w->1,
each a 3x3 convolution with zero padding 1 (ReLU except `out`), stored as
W[out][in][3][3] then b[out] in one flat array; 2x2 average pooling after enc1b
and enc2b, nearest 2x upsampling before dec2a (concat [up(botb), enc2b]) and
dec1a (concat [up(dec2b), enc1b]); X0 = C + out.  The convolutions use the
weights rounded to BF16 (round to nearest even), as the library does.

Pins (tests/test_unet_oracle.py): convolution vs torch.nn.functional.conv2d on
the CPU, pooling/upsampling adjoint identities, full gradient vs central finite
differences, one Adam step vs torch.optim.Adam.
"""
from __future__ import annotations

import numpy as np

LAYERS = ["enc1a", "enc1b", "enc2a", "enc2b", "bota", "botb", "dec2a", "dec2b", "dec1a", "dec1b", "out"]


def layer_io(w):
    return [(1, w), (w, w), (w, 2 * w), (2 * w, 2 * w), (2 * w, 4 * w), (4 * w, 4 * w), (6 * w, 2 * w),
            (2 * w, 2 * w), (3 * w, w), (w, w), (w, 1)]


def num_params(w):
    return sum(ci * co * 9 + co for ci, co in layer_io(w))


def unpack(params, w):
    """Flat array -> list of (W [co, ci, 3, 3], b [co])."""
    out, off = [], 0
    for ci, co in layer_io(w):
        W = params[off:off + ci * co * 9].reshape(co, ci, 3, 3)
        off += ci * co * 9
        b = params[off:off + co]
        off += co
        out.append((W, b))
    assert off == len(params)
    return out


def bf16_round(x):
    """Round FP32 values to the nearest BF16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def conv3x3(x, W, b):
    """out[n, o, y, x] = b[o] + sum_{i, ky, kx} W[o, i, ky, kx] x[n, i, y + ky - 1, x + kx - 1]."""
    N, Ci, H, Wd = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    out = np.zeros((N, W.shape[0], H, Wd))
    for ky in range(3):
        for kx in range(3):
            out += np.einsum("oi,nihw->nohw", W[:, :, ky, kx], xp[:, :, ky:ky + H, kx:kx + Wd])
    return out + b[None, :, None, None]


def conv3x3_grads(x, W, g):
    """Gradients of sum(g * conv3x3(x, W, b)) w.r.t. x, W and b."""
    N, Ci, H, Wd = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    dW = np.zeros_like(W)
    dxp = np.zeros_like(xp)
    for ky in range(3):
        for kx in range(3):
            dW[:, :, ky, kx] = np.einsum("nohw,nihw->oi", g, xp[:, :, ky:ky + H, kx:kx + Wd])
            dxp[:, :, ky:ky + H, kx:kx + Wd] += np.einsum("oi,nohw->nihw", W[:, :, ky, kx], g)
    return dxp[:, :, 1:-1, 1:-1], dW, g.sum(axis=(0, 2, 3))


def pool(x):
    N, C, H, W = x.shape
    return x.reshape(N, C, H // 2, 2, W // 2, 2).mean(axis=(3, 5))


def pool_adj(g):
    return np.repeat(np.repeat(g, 2, axis=2), 2, axis=3) / 4.0


def up(x):
    return np.repeat(np.repeat(x, 2, axis=2), 2, axis=3)


def up_adj(g):
    N, C, H, W = g.shape
    return g.reshape(N, C, H // 2, 2, W // 2, 2).sum(axis=(3, 5))


def forward(params, w, C, keep=False, bf16=True):
    """C: [N, H, W] -> X0 [N, H, W] (and the activations when keep).  bf16=False
    keeps the weights exact (used by the finite-difference pin)."""
    if bf16:
        P = [(bf16_round(W), b.astype(np.float64)) for W, b in unpack(np.asarray(params, dtype=np.float32), w)]
    else:
        P = [(W.astype(np.float64), b.astype(np.float64)) for W, b in unpack(np.asarray(params, dtype=np.float64), w)]
    relu = lambda z: np.maximum(z, 0.0)
    x = C[:, None].astype(np.float64)
    a = {}
    a["x"] = x
    a["enc1a"] = relu(conv3x3(x, *P[0]))
    a["enc1b"] = relu(conv3x3(a["enc1a"], *P[1]))
    a["p1"] = pool(a["enc1b"])
    a["enc2a"] = relu(conv3x3(a["p1"], *P[2]))
    a["enc2b"] = relu(conv3x3(a["enc2a"], *P[3]))
    a["p2"] = pool(a["enc2b"])
    a["bota"] = relu(conv3x3(a["p2"], *P[4]))
    a["botb"] = relu(conv3x3(a["bota"], *P[5]))
    a["cat2"] = np.concatenate([up(a["botb"]), a["enc2b"]], axis=1)
    a["dec2a"] = relu(conv3x3(a["cat2"], *P[6]))
    a["dec2b"] = relu(conv3x3(a["dec2a"], *P[7]))
    a["cat1"] = np.concatenate([up(a["dec2b"]), a["enc1b"]], axis=1)
    a["dec1a"] = relu(conv3x3(a["cat1"], *P[8]))
    a["dec1b"] = relu(conv3x3(a["dec1a"], *P[9]))
    a["out"] = conv3x3(a["dec1b"], *P[10])
    X0 = C + a["out"][:, 0]
    return (X0, a, P) if keep else X0


def loss_grad(params, w, C, T, bf16=True):
    """loss = mean((X0 - T)^2) and its gradient w.r.t. the flat parameters (taken
    w.r.t. the BF16-rounded weights the forward pass uses)."""
    X0, a, P = forward(params, w, C, keep=True, bf16=bf16)
    d = X0 - T
    loss = float(np.mean(d * d))
    g_out = (2.0 * d / d.size)[:, None]
    grads = [None] * len(P)

    def back(idx, inp, outv, g, relu_layer=True):
        if relu_layer:
            g = g * (outv > 0)
        dx, dW, db = conv3x3_grads(inp, P[idx][0], g)
        grads[idx] = (dW, db)
        return dx

    w_ = w
    g = back(10, a["dec1b"], a["out"], g_out, relu_layer=False)
    g = back(9, a["dec1a"], a["dec1b"], g)
    g_cat1 = back(8, a["cat1"], a["dec1a"], g)
    g_dec2b = up_adj(g_cat1[:, :2 * w_])
    g_enc1b = g_cat1[:, 2 * w_:]
    g = back(7, a["dec2a"], a["dec2b"], g_dec2b)
    g_cat2 = back(6, a["cat2"], a["dec2a"], g)
    g_botb = up_adj(g_cat2[:, :4 * w_])
    g_enc2b = g_cat2[:, 4 * w_:]
    g = back(5, a["bota"], a["botb"], g_botb)
    g_p2 = back(4, a["p2"], a["bota"], g)
    g_enc2b = g_enc2b + pool_adj(g_p2)
    g = back(3, a["enc2a"], a["enc2b"], g_enc2b)
    g_p1 = back(2, a["p1"], a["enc2a"], g)
    g_enc1b = g_enc1b + pool_adj(g_p1)
    g = back(1, a["enc1a"], a["enc1b"], g_enc1b)
    back(0, a["x"], a["enc1a"], g)
    flat = np.concatenate([np.concatenate([dW.ravel(), db.ravel()]) for dW, db in grads])
    return loss, flat


def adam_step(params, grad, m1, m2, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba) with bias correction; returns new (params, m1, m2)."""
    m1 = b1 * m1 + (1 - b1) * grad
    m2 = b2 * m2 + (1 - b2) * grad * grad
    c1, c2 = 1 - b1 ** step, 1 - b2 ** step
    return params - lr * (m1 / c1) / (np.sqrt(m2 / c2) + eps), m1, m2
