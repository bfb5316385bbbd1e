"""FP64 CPU oracle of the learned warm start's network (a 2D U-Net over the
N phases as channels) and of its training step.

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): the GPU kernels are
checked against it; the product path never imports it.

The network (all convolutions zero-padded, with bias):
  encoder level l = 0..L-1, c_l = base * 2^l channels:
      x_0 = input, x_l = maxpool2(e_{l-1});  e_l = relu(conv3(relu(conv3(x_l))))
  decoder level l = L-2..0:
      u = upsample_nearest2(d_{l+1}) (d_{L-1} = e_{L-1});  c = concat(u, e_l)
      d_l = relu(conv3(relu(conv3(c))))
  output = input + conv1(d_0)          (the net predicts a correction)
Loss: mean squared error against the target.

Storage emulation: the GPU keeps the input, the weights used in the
convolutions and every post-ReLU activation in BF16 (round to nearest
even), accumulates in FP32 and keeps gradients in FP32, except that a
gradient entering a 3x3 convolution's backward products (input and weight
gradients) is rounded to BF16 (the bias gradient and the final 1x1 layer
use it unrounded).  With bf16=True the oracle rounds the same values at the
same points (and nothing else), so the two differ only by accumulation
order.

Parameter order (flat list of (weight, bias)): encoder l = 0..L-1 conv a, b;
decoder l = L-2..0 conv a, b; the final 1x1 convolution.  Weights are
[cout][cin][3][3] ([cout][cin] for the 1x1).
"""
from __future__ import annotations

from typing import List, Tuple

import numpy as np


def bf16(a: np.ndarray) -> np.ndarray:
    """Round FP32 values to BF16 (nearest, ties to even) and back (FP64 out)."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def layer_shapes(in_ch: int, out_ch: int, base: int, levels: int) -> List[Tuple[int, int, int]]:
    """(cout, cin, k) of every convolution in parameter order."""
    s = []
    cin = in_ch
    for l in range(levels):
        c = base << l
        s += [(c, cin, 3), (c, c, 3)]
        cin = c
    for l in range(levels - 2, -1, -1):
        c = base << l
        s += [(c, (base << (l + 1)) + c, 3), (c, c, 3)]
    s.append((out_ch, base, 1))
    return s


def init_params(in_ch, out_ch, base, levels, seed):
    """He-normal weights, zero biases, a zero final layer (the net starts as
    the identity map of its input)."""
    rng = np.random.default_rng(seed)
    ps = []
    shapes = layer_shapes(in_ch, out_ch, base, levels)
    for i, (co, ci, k) in enumerate(shapes):
        if i == len(shapes) - 1:
            w = np.zeros((co, ci))
        else:
            w = rng.standard_normal((co, ci, k, k)) * np.sqrt(2.0 / (ci * k * k))
        ps.append((w.astype(np.float32).astype(np.float64), np.zeros(co)))
    return ps


# ---------------------------------------------------------------- primitives
def conv3(x, w, b):
    """x [B][C][H][W], w [O][C][3][3] -> [B][O][H][W], zero padding 1."""
    B, C, H, W = x.shape
    xp = np.zeros((B, C, H + 2, W + 2))
    xp[:, :, 1:-1, 1:-1] = x
    out = np.zeros((B, w.shape[0], H, W))
    for ky in range(3):
        for kx in range(3):
            out += np.einsum("bchw,oc->bohw", xp[:, :, ky:ky + H, kx:kx + W], w[:, :, ky, kx])
    return out + b[None, :, None, None]


def conv3_backward(x, w, gout):
    """Gradients of conv3 w.r.t. its input, weights and bias."""
    B, C, H, W = x.shape
    xp = np.zeros((B, C, H + 2, W + 2))
    xp[:, :, 1:-1, 1:-1] = x
    gw = np.zeros_like(w)
    gxp = np.zeros_like(xp)
    for ky in range(3):
        for kx in range(3):
            gw[:, :, ky, kx] = np.einsum("bohw,bchw->oc", gout, xp[:, :, ky:ky + H, kx:kx + W])
            gxp[:, :, ky:ky + H, kx:kx + W] += np.einsum("bohw,oc->bchw", gout, w[:, :, ky, kx])
    return gxp[:, :, 1:-1, 1:-1], gw, gout.sum(axis=(0, 2, 3))


def maxpool2(x):
    B, C, H, W = x.shape
    v = x.reshape(B, C, H // 2, 2, W // 2, 2)
    return v.max(axis=(3, 5))


def maxpool2_backward(x, gout):
    """The gradient goes to the first maximum of each 2x2 window in the order
    (0,0), (0,1), (1,0), (1,1)."""
    B, C, H, W = x.shape
    g = np.zeros_like(x)
    m = maxpool2(x)
    taken = np.zeros(gout.shape, dtype=bool)
    for dy in range(2):
        for dx in range(2):
            hit = (x[:, :, dy::2, dx::2] == m) & ~taken
            g[:, :, dy::2, dx::2] = np.where(hit, gout, 0.0)
            taken |= hit
    return g


def up2(x):
    return x.repeat(2, axis=2).repeat(2, axis=3)


def up2_backward(g):
    B, C, H, W = g.shape
    return g.reshape(B, C, H // 2, 2, W // 2, 2).sum(axis=(3, 5))


# ---------------------------------------------------------------- network
def forward(params, x, levels, bf16_storage=True):
    """Returns (output, cache) ; cache holds what the backward pass needs."""
    q = bf16 if bf16_storage else (lambda a: np.asarray(a, np.float64))
    W = [(q(w), b) for w, b in params]
    xin = q(x)
    cache = {"x": xin, "acts": []}
    enc = []
    h = xin
    k = 0
    for l in range(levels):
        if l > 0:
            h = maxpool2(enc[-1])
        a_in = h
        z1 = conv3(a_in, *W[k]); a1 = q(np.maximum(z1, 0)); k += 1
        z2 = conv3(a1, *W[k]); a2 = q(np.maximum(z2, 0)); k += 1
        cache["acts"].append((a_in, a1, a2))
        enc.append(a2)
    d = enc[-1]
    for l in range(levels - 2, -1, -1):
        c = np.concatenate([up2(d), enc[l]], axis=1)
        z1 = conv3(c, *W[k]); a1 = q(np.maximum(z1, 0)); k += 1
        z2 = conv3(a1, *W[k]); a2 = q(np.maximum(z2, 0)); k += 1
        cache["acts"].append((c, a1, a2))
        d = a2
    wf, bf = W[k]
    out = xin + np.einsum("bchw,oc->bohw", d, wf) + bf[None, :, None, None]
    cache["d0"] = d
    cache["W"] = W
    return out, cache


def loss_and_grads(params, x, target, levels, bf16_storage=True):
    """MSE loss and its gradients w.r.t. every (weight, bias), FP64."""
    out, cache = forward(params, x, levels, bf16_storage)
    q = bf16 if bf16_storage else (lambda a: a)

    def conv3_bwd(xin, w, gz):
        gx, gw, _ = conv3_backward(xin, w, q(gz))
        return gx, gw, gz.sum(axis=(0, 2, 3))

    n = out.size
    loss = float(np.sum((out - target) ** 2) / n)
    g_out = 2.0 * (out - target) / n
    W = cache["W"]
    grads = [None] * len(W)
    k = len(W) - 1
    d0 = cache["d0"]
    grads[k] = (np.einsum("bohw,bchw->oc", g_out, d0), g_out.sum(axis=(0, 2, 3)))
    g = np.einsum("bohw,oc->bchw", g_out, W[k][0])
    k -= 1
    acts = cache["acts"]
    enc_grads = [None] * levels
    # decoder, last built first
    for l in range(0, levels - 1):
        c, a1, a2 = acts[levels + (levels - 2 - l)]
        g2 = g * (a2 > 0)
        ga1, gw, gb = conv3_bwd(a1, W[k][0], g2); grads[k] = (gw, gb); k -= 1
        g1 = ga1 * (a1 > 0)
        gc, gw, gb = conv3_bwd(c, W[k][0], g1); grads[k] = (gw, gb); k -= 1
        cu = acts[l + 1][2].shape[1]        # channels of the upsampled part (those of e_{l+1})
        g_up, g_skip = gc[:, :cu], gc[:, cu:]
        enc_grads[l] = g_skip
        g = up2_backward(g_up)
    # encoder, deepest first (g is the gradient w.r.t. e_{L-1})
    for l in range(levels - 1, -1, -1):
        if enc_grads[l] is not None and l < levels - 1:
            g = g + enc_grads[l]
        a_in, a1, a2 = acts[l]
        g2 = g * (a2 > 0)
        ga1, gw, gb = conv3_bwd(a1, W[k][0], g2); grads[k] = (gw, gb); k -= 1
        g1 = ga1 * (a1 > 0)
        gin, gw, gb = conv3_bwd(a_in, W[k][0], g1); grads[k] = (gw, gb); k -= 1
        if l > 0:
            g = maxpool2_backward(acts[l - 1][2], gin)
    return loss, grads, out
