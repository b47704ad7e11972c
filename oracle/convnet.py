"""Learned preconditioner network (oracle, FP64): forward and backward.

The learned replacement of the Teter preconditioner is a 3-D convolutional
network on the extended element's grid: inputs are the residual (scaled to
unit RMS) and the local potential, 4 layers of 3x3x3 convolutions with
circular padding (the grid is periodic), 2 -> 16 -> 16 -> 16 -> 1 channels,
ReLU between layers and none on the output; the correction is the output
times the residual's RMS, which makes the map scale-equivariant.  It is
trained on (residual, exact correction) pairs, the correction solving
(H - sigma I) t = r, by mean squared error on the unit-RMS target.

Layout: fields are (C, nz, ny, nx); weights (C_out, C_in, 3, 3, 3) indexed
[dz, dy, dx] with the tap at offset (d - 1) along each axis:

    out[o, z, y, x] = b[o] + sum_{i, dz, dy, dx} w[o, i, dz, dy, dx]
                      * in[i, z + dz - 1, y + dy - 1, x + dx - 1]   (mod n)

This module is plain NumPy: one shifted copy per tap, no blocking.
"""

from __future__ import annotations

import numpy as np

CHANNELS = (2, 16, 16, 16, 1)


def _shift(x: np.ndarray, dz: int, dy: int, dx: int) -> np.ndarray:
    """y[..., z, y, x] = x[..., z + dz - 1, y + dy - 1, x + dx - 1] (periodic)."""
    return np.roll(x, shift=(1 - dz, 1 - dy, 1 - dx), axis=(-3, -2, -1))


def conv3d(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Circular 3x3x3 convolution (cross-correlation) with bias."""
    co = w.shape[0]
    out = np.zeros((co,) + x.shape[1:])
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                xs = _shift(x, dz, dy, dx)
                out += np.einsum("oi,izyx->ozyx", w[:, :, dz, dy, dx], xs)
    return out + b[:, None, None, None]


def conv3d_backward(x: np.ndarray, w: np.ndarray, gout: np.ndarray):
    """Gradients of sum(gout * conv3d(x, w, b)) w.r.t. x, w, b."""
    gx = np.zeros_like(x)
    gw = np.zeros_like(w)
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                xs = _shift(x, dz, dy, dx)
                gw[:, :, dz, dy, dx] = np.einsum("ozyx,izyx->oi", gout, xs)
                # adjoint of the shift: move gout back by the same offset
                g = np.einsum("oi,ozyx->izyx", w[:, :, dz, dy, dx], gout)
                gx += np.roll(g, shift=(dz - 1, dy - 1, dx - 1), axis=(-3, -2, -1))
    gb = gout.sum(axis=(1, 2, 3))
    return gx, gw, gb


def init_params(gen: np.random.Generator, channels=CHANNELS):
    """He-normal weights, zero biases."""
    params = []
    for ci, co in zip(channels[:-1], channels[1:]):
        w = gen.standard_normal((co, ci, 3, 3, 3)) * np.sqrt(2.0 / (27 * ci))
        params.append((w, np.zeros(co)))
    return params


def forward(params, inp: np.ndarray):
    """Network output and the per-layer activations needed for backward."""
    acts = [inp]
    h = inp
    for k, (w, b) in enumerate(params):
        z = conv3d(h, w, b)
        h = np.maximum(z, 0.0) if k + 1 < len(params) else z
        acts.append(h)
    return h, acts


def backward(params, acts, gout: np.ndarray):
    """Parameter gradients of sum(gout * output) (ReLU masks from acts)."""
    grads = [None] * len(params)
    g = gout
    for k in range(len(params) - 1, -1, -1):
        w, _ = params[k]
        if k + 1 < len(params):
            g = g * (acts[k + 1] > 0.0)
        gx, gw, gb = conv3d_backward(acts[k], w, g)
        grads[k] = (gw, gb)
        g = gx
    return grads


def network_input(r: np.ndarray, v: np.ndarray):
    """(2, nz, ny, nx) input and the RMS scale of the residual r."""
    rms = float(np.sqrt(np.mean(r * r)))
    rms = rms if rms > 0.0 else 1.0
    return np.stack([r / rms, v]), rms


def precondition(params, r: np.ndarray, v: np.ndarray) -> np.ndarray:
    """w = rms(r) * net(r / rms(r), V) for one residual field (nz, ny, nx)."""
    inp, rms = network_input(r, v)
    out, _ = forward(params, inp)
    return rms * out[0]


def loss_and_grads(params, r: np.ndarray, v: np.ndarray, t: np.ndarray):
    """Mean squared error of net(r/rms, V) against t/rms and its gradients."""
    inp, rms = network_input(r, v)
    out, acts = forward(params, inp)
    diff = out[0] - t / rms
    n = diff.size
    loss = float(np.sum(diff * diff) / n)
    gout = (2.0 / n) * diff[None]
    return loss, backward(params, acts, gout)
