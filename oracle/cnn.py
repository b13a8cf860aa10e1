"""Residual CNN of the learned warm start, forward and backward in float64
(oracle; test infrastructure only).

The network maps the density-compensated adjoint u = T^H y, as a 2-channel
image (real, imaginary part; pixel (j, i) = coefficient i + N j), to
x0 = u + f(u), where f is a stack of 3x3 convolutions (zero padding 1) with
ReLU between them and none after the last.  Loss: mean squared error
L = sum (x0 - target)^2 / (B * 2 * H * W).

Parameters per layer l: weight W[l] of shape (C_out, C_in, 3, 3), bias b[l] of
shape (C_out,).  Convolution (cross-correlation, as in every CNN library):
    out[o, y, x] = b[o] + sum_{c, dy, dx} W[o, c, dy, dx] in[c, y + dy - 1, x + dx - 1].
Every operation is written out with numpy loops over the 9 taps; gradients are
the textbook backpropagation of these formulas.
"""
import numpy as np


def conv3(inp, W, b):
    """inp (B, C, H, W) -> (B, O, H, W)."""
    B, C, H, Wd = inp.shape
    O = W.shape[0]
    pad = np.zeros((B, C, H + 2, Wd + 2))
    pad[:, :, 1:-1, 1:-1] = inp
    out = np.zeros((B, O, H, Wd)) + b[None, :, None, None]
    for dy in range(3):
        for dx in range(3):
            patch = pad[:, :, dy:dy + H, dx:dx + Wd]  # (B, C, H, W)
            out += np.einsum("oc,bchw->bohw", W[:, :, dy, dx], patch)
    return out


def conv3_backward(inp, W, gout):
    """Gradients of conv3 w.r.t. its input, weight and bias."""
    B, C, H, Wd = inp.shape
    pad = np.zeros((B, C, H + 2, Wd + 2))
    pad[:, :, 1:-1, 1:-1] = inp
    gW = np.zeros_like(W)
    gpad = np.zeros_like(pad)
    for dy in range(3):
        for dx in range(3):
            patch = pad[:, :, dy:dy + H, dx:dx + Wd]
            gW[:, :, dy, dx] = np.einsum("bohw,bchw->oc", gout, patch)
            gpad[:, :, dy:dy + H, dx:dx + Wd] += np.einsum("oc,bohw->bchw", W[:, :, dy, dx], gout)
    gb = gout.sum(axis=(0, 2, 3))
    return gpad[:, :, 1:-1, 1:-1], gW, gb


def forward(params, u):
    """params: list of (W, b); returns x0 and the per-layer activations."""
    acts = [u]
    h = u
    for l, (W, b) in enumerate(params):
        z = conv3(h, W, b)
        h = np.maximum(z, 0.0) if l < len(params) - 1 else z
        acts.append(h)
    return u + h, acts


def loss_and_grads(params, u, target):
    x0, acts = forward(params, u)
    n = x0.size
    diff = x0 - target
    loss = np.sum(diff * diff) / n
    g = 2.0 * diff / n  # dL/dx0 = dL/df (the residual path u has no parameters)
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W, b = params[l]
        if l < len(params) - 1:
            g = g * (acts[l + 1] > 0)  # through the ReLU of layer l
        gin, gW, gb = conv3_backward(acts[l], W, g)
        grads[l] = (gW, gb)
        g = gin
    return loss, grads
