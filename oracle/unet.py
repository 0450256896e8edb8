"""FP64 reference of the learned warm start's network (a small 3-D U-Net).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The DDSCAT guide has no learned component; this network exists to give the
Krylov solver an initial guess.  It maps per-voxel features of a target on its
lattice box (occupancy, permittivity, incident field) to the local field
E_loc = alpha^{-1} P, from which the warm start is P0 = alpha E_loc.

Architecture (channels C1..C4, all 3x3x3 convolutions zero-padded, ReLU after
each, average pooling 2x2x2 down, nearest-neighbour upsampling x2, skip
connections concatenated as [upsampled, skip]):
  enc1: cin->C1, C1->C1          pool
  enc2: C1->C2, C2->C2           pool
  enc3: C2->C3, C3->C3           pool
  bot : C3->C4, C4->C4           up
  dec3: C4+C3->C3, C3->C3        up
  dec2: C3+C2->C2, C2->C2        up
  dec1: C2+C1->C1, C1->C1
  head: 1x1x1 C1->cout (linear)
Tensors are channels-last: [B][Z][Y][X][C].  Convolution weights are
[tap][cin][cout] with tap = (dz+1)*9 + (dy+1)*3 + (dx+1).  The flat parameter
vector lists, layer by layer, W then b.

`quant=True` rounds each convolution's input, its weights and (in the backward
pass) the incoming gradient to bfloat16 (round to nearest, ties to even),
which is where the GPU kernels round before their tensor-core products; the
arithmetic itself is FP64.  Parity of this file is pinned by finite
differences and by torch's CPU conv3d in the tests.
"""
from __future__ import annotations

import numpy as np


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round FP64/FP32 values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    bits = (bits + 0x7FFF + lsb) & 0xFFFF0000
    return bits.astype(np.uint32).view(np.float32).astype(np.float64)


def layer_shapes(cin: int, cout: int, ch):
    c1, c2, c3, c4 = ch
    convs = [(cin, c1), (c1, c1), (c1, c2), (c2, c2), (c2, c3), (c3, c3), (c3, c4), (c4, c4),
             (c4 + c3, c3), (c3, c3), (c3 + c2, c2), (c2, c2), (c2 + c1, c1), (c1, c1)]
    shapes = [(27, a, b) for a, b in convs] + [(1, c1, cout)]
    return shapes


def n_params(cin, cout, ch):
    return sum(t * a * b + b for t, a, b in layer_shapes(cin, cout, ch))


def unpack(theta, cin, cout, ch):
    out, o = [], 0
    for t, a, b in layer_shapes(cin, cout, ch):
        w = theta[o:o + t * a * b].reshape(t, a, b)
        o += t * a * b
        bias = theta[o:o + b]
        o += b
        out.append((w, bias))
    return out


def _shift(x, dz, dy, dx):
    """x[b, z+dz, y+dy, x+dx, c] with zeros outside."""
    out = np.zeros_like(x)
    B, Z, Y, X, C = x.shape
    zs, ze = max(0, -dz), min(Z, Z - dz)
    ys, ye = max(0, -dy), min(Y, Y - dy)
    xs, xe = max(0, -dx), min(X, X - dx)
    out[:, zs:ze, ys:ye, xs:xe] = x[:, zs + dz:ze + dz, ys + dy:ye + dy, xs + dx:xe + dx]
    return out


TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def conv3(x, w, b):
    """3x3x3 convolution (cross-correlation), zero padding: y = sum_tap shift(x, tap) @ w[tap] + b."""
    y = np.zeros(x.shape[:4] + (w.shape[2],))
    for t, (dz, dy, dx) in enumerate(TAPS):
        y += _shift(x, dz, dy, dx) @ w[t]
    return y + b


def conv3_backward(x, w, gy):
    """Gradients of conv3 w.r.t. x, w, b given dL/dy."""
    gx = np.zeros_like(x)
    gw = np.zeros_like(w)
    for t, (dz, dy, dx) in enumerate(TAPS):
        xs = _shift(x, dz, dy, dx)
        gw[t] = np.einsum("bzyxi,bzyxo->io", xs, gy)
        gx += _shift(gy @ w[t].T, -dz, -dy, -dx)
    return gx, gw, gy.sum(axis=(0, 1, 2, 3))


def pool2(x):
    B, Z, Y, X, C = x.shape
    return x.reshape(B, Z // 2, 2, Y // 2, 2, X // 2, 2, C).mean(axis=(2, 4, 6))


def pool2_backward(g, shape):
    return np.repeat(np.repeat(np.repeat(g, 2, axis=1), 2, axis=2), 2, axis=3) / 8.0


def up2(x):
    return np.repeat(np.repeat(np.repeat(x, 2, axis=1), 2, axis=2), 2, axis=3)


def up2_backward(g):
    B, Z, Y, X, C = g.shape
    return g.reshape(B, Z // 2, 2, Y // 2, 2, X // 2, 2, C).sum(axis=(2, 4, 6))


def forward(theta, x, cin, cout, ch, quant=False, keep=False):
    """Network output for input x [B,Z,Y,X,cin]; keep=True also returns the tape for backward."""
    layers = unpack(theta, cin, cout, ch)
    q = bf16_round if quant else (lambda a: a)
    tape = []

    def conv_relu(h, li):
        w, b = layers[li]
        hin = q(h)
        pre = conv3(hin, q(w), b)
        out = np.maximum(pre, 0.0)
        tape.append(("conv", li, hin, out))
        return out

    h = conv_relu(x, 0); s1 = conv_relu(h, 1)
    h = pool2(s1)
    h = conv_relu(h, 2); s2 = conv_relu(h, 3)
    h = pool2(s2)
    h = conv_relu(h, 4); s3 = conv_relu(h, 5)
    h = pool2(s3)
    h = conv_relu(h, 6); h = conv_relu(h, 7)
    h = np.concatenate([up2(h), s3], axis=-1)
    h = conv_relu(h, 8); h = conv_relu(h, 9)
    h = np.concatenate([up2(h), s2], axis=-1)
    h = conv_relu(h, 10); h = conv_relu(h, 11)
    h = np.concatenate([up2(h), s1], axis=-1)
    h = conv_relu(h, 12); h = conv_relu(h, 13)
    w, b = layers[14]
    hin = q(h)
    y = hin @ q(w[0]) + b
    tape.append(("head", 14, hin, y))
    return (y, tape) if keep else y


def loss(y, t, mask):
    """Masked mean squared error over occupied voxels and output channels."""
    m = mask[..., None]
    cnt = mask.sum() * y.shape[-1]
    return float(np.sum(m * (y - t) ** 2) / cnt)


def loss_and_grad(theta, x, t, mask, cin, cout, ch, quant=False):
    """Loss and dLoss/dtheta by reverse-mode differentiation of `forward`."""
    layers = unpack(theta, cin, cout, ch)
    q = bf16_round if quant else (lambda a: a)
    y, tape = forward(theta, x, cin, cout, ch, quant=quant, keep=True)
    m = mask[..., None]
    cnt = mask.sum() * y.shape[-1]
    L = float(np.sum(m * (y - t) ** 2) / cnt)
    gy = 2.0 * m * (y - t) / cnt
    grads = [None] * len(layers)
    # head
    _, li, hin, _ = tape[-1]
    w, b = layers[li]
    gq = q(gy)
    grads[li] = (np.einsum("bzyxi,bzyxo->io", hin, gq)[None], gy.sum(axis=(0, 1, 2, 3)))
    g = gq @ q(w[0]).T

    def conv_back(g, k):
        kind, li, hin, out = tape[k]
        w, b = layers[li]
        gpre = g * (out > 0)
        gq = q(gpre)
        gx, gw, _ = conv3_backward(hin, q(w), gq)
        grads[li] = (gw, gpre.sum(axis=(0, 1, 2, 3)))
        return gx

    c1, c2, c3, c4 = ch
    # tape indices: 0 e1a 1 e1b 2 e2a 3 e2b 4 e3a 5 e3b 6 ba 7 bb 8 d3a 9 d3b 10 d2a 11 d2b 12 d1a 13 d1b 14 head
    g = conv_back(g, 13)
    g = conv_back(g, 12)
    g_up, g_s1 = g[..., :c2], g[..., c2:]
    g = up2_backward(g_up)
    g = conv_back(g, 11)
    g = conv_back(g, 10)
    g_up, g_s2 = g[..., :c3], g[..., c3:]
    g = up2_backward(g_up)
    g = conv_back(g, 9)
    g = conv_back(g, 8)
    g_up, g_s3 = g[..., :c4], g[..., c4:]
    g = up2_backward(g_up)
    g = conv_back(g, 7)
    g = conv_back(g, 6)
    g = pool2_backward(g, None) + g_s3
    g = conv_back(g, 5)
    g = conv_back(g, 4)
    g = pool2_backward(g, None) + g_s2
    g = conv_back(g, 3)
    g = conv_back(g, 2)
    g = pool2_backward(g, None) + g_s1
    g = conv_back(g, 1)
    conv_back(g, 0)
    flat = np.concatenate([np.concatenate([gw.reshape(-1), gb]) for gw, gb in grads])
    return L, flat


def adamw(theta, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0):
    """One AdamW update (Loshchilov & Hutter): decoupled weight decay, bias-corrected moments."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    theta = theta - lr * (mh / (np.sqrt(vh) + eps) + wd * theta)
    return theta, m, v
