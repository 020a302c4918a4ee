"""Convolutional network of the learned warm start, FP64 (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The warm start is not part of the paper: a small fully convolutional network
maps an observation to a per-pixel guess of the EP posterior mean and
log-variance, from which the prior sites are initialised before plain EP
sweeps.  This module is the reference the GPU kernels are checked against:
forward pass, backward pass and the Adam step, written from their definitions.

Layers: L convolutions with 3x3 kernels on a torus (circular padding, like the
periodic image model), each followed by a ReLU except the last.  Arrays are
(batch, channels, height, width).  A convolution is the cross-correlation

    out[n, o, i, j] = b[o] + sum_{c, a, e} W[o, c, a, e] x[n, c, (i + a - 1) mod H, (j + e - 1) mod W]

with a, e in {0, 1, 2}.
"""
from __future__ import annotations

import numpy as np


def conv3x3(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Circular 3x3 cross-correlation; x (N, C, H, W), w (O, C, 3, 3), b (O,)."""
    n, c, h, wd = x.shape
    o = w.shape[0]
    out = np.empty((n, o, h, wd))
    out[:] = b[None, :, None, None]
    for a in range(3):
        for e in range(3):
            # shifted[..., i, j] = x[..., i + a - 1, j + e - 1]
            shifted = np.roll(x, shift=(1 - a, 1 - e), axis=(2, 3))
            out += np.einsum("oc,nchw->nohw", w[:, :, a, e], shifted)
    return out


def conv3x3_backward(x: np.ndarray, w: np.ndarray, dout: np.ndarray):
    """Gradients of a loss through conv3x3 given dL/dout: (dx, dw, db)."""
    dx = np.zeros_like(x)
    dw = np.zeros_like(w)
    for a in range(3):
        for e in range(3):
            shifted = np.roll(x, shift=(1 - a, 1 - e), axis=(2, 3))
            dw[:, :, a, e] = np.einsum("nohw,nchw->oc", dout, shifted)
            # out[i, j] uses x[i + a - 1, j + e - 1]: send dout back by the same shift
            back = np.einsum("oc,nohw->nchw", w[:, :, a, e], dout)
            dx += np.roll(back, shift=(a - 1, e - 1), axis=(2, 3))
    db = dout.sum(axis=(0, 2, 3))
    return dx, dw, db


def forward(params, x: np.ndarray):
    """All layers; params is a list of (w, b).  Returns the output and the list
    of layer inputs and pre-activations needed by backward."""
    acts = [x]
    pres = []
    h = x
    for li, (w, b) in enumerate(params):
        z = conv3x3(h, w, b)
        pres.append(z)
        h = np.maximum(z, 0.0) if li + 1 < len(params) else z
        acts.append(h)
    return h, acts, pres


def backward(params, acts, pres, dout: np.ndarray):
    """Gradients of all layers' (w, b) given dL/d(network output)."""
    grads = [None] * len(params)
    g = dout
    for li in range(len(params) - 1, -1, -1):
        if li + 1 < len(params):
            g = g * (pres[li] > 0.0)
        w, _ = params[li]
        dx, dw, db = conv3x3_backward(acts[li], w, g)
        grads[li] = (dw, db)
        g = dx
    return grads


def adam_step(p, g, m, v, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, Algorithm 1) in place; t counts from 1."""
    m *= beta1
    m += (1.0 - beta1) * g
    v *= beta2
    v += (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    p -= lr * mhat / (np.sqrt(vhat) + eps)


def warmstart_loss(out: np.ndarray, y: np.ndarray, mean: np.ndarray, tau: np.ndarray,
                   log_xi: np.ndarray, w_mu: float):
    """Training loss of the warm start against a converged EP state and its
    gradient w.r.t. the output (n, 6, h, w).

    Targets: out0 -> mean - y (posterior mean minus observation), out[1 + s] ->
    log(tau_s) + log(xi) (site precisions, site 0 first, tau (n, 5, h, w));
    L = mean over images and pixels of w_mu (out0 - t0)^2 + (1/5) sum_s (out[1+s] - t[1+s])^2.
    """
    n = out.shape[0] * out.shape[2] * out.shape[3]
    t = np.empty_like(out)
    t[:, 0] = mean - y
    t[:, 1:] = np.log(tau) + np.asarray(log_xi)[:, None, None, None]
    r = out - t
    wts = np.array([w_mu] + [0.2] * 5)[None, :, None, None]
    loss = float((wts * r * r).sum() / n)
    return loss, 2.0 * wts * r / n
