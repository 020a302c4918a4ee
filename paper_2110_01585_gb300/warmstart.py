"""Learned warm start (not in the paper).

A small fully convolutional network maps an observation to a per-pixel guess of
the converged EP state: the posterior mean and the precision of each of the five
sites.  ``ep_tv_warm_start`` sets the sites from it, and plain EP sweeps take
over from there (and correct the guess: a context that is not warm-started is the
cold-start fallback).  Predicting the site precisions, not only the posterior,
starts EP near the fixed point the cold start reaches.

The network: L = 6 convolutions with 3x3 kernels on the torus, 32 channels,
ReLU between them.  Input channels: the observation y, log10(xi)/4 and the blur
standard deviation / 4 (constant planes).  Six outputs:
    mean = y + out0,      tau_s = exp(out[1 + s]) / xi   (sites s = 0..4).
Training minimises mean(w_mean (out0 - (mu_EP - y))^2 + (1/5) sum_s (out[1+s] - log(tau_s xi))^2)
against converged states of plain cold-start EP, with Adam.  Inputs, targets and
the prediction stay on the device.

Everything here is argument marshalling around the C ABI: the forward and
backward passes, the loss and the optimiser step run in libeptv's kernels.
"""
from __future__ import annotations

import ctypes
import math
from typing import List, Optional, Tuple

import numpy as np

from . import _lib

CHANNELS = 32
LAYERS = 6
IN_CHANNELS = 3
OUT_CHANNELS = 6
W_MEAN = 100.0


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p()


def _check(code, where):
    _lib.check(code, where)


class WarmStartNet:
    """The warm-start network on one CUDA device."""

    def __init__(self, seed: int = 0, channels: int = CHANNELS, layers: int = LAYERS,
                 device: str = "cuda", stream=None):
        import torch
        self.torch = torch
        self.lib = _lib.load()
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        rng = np.random.default_rng(seed)
        dims = [IN_CHANNELS] + [channels] * (layers - 1) + [OUT_CHANNELS]
        self.params: List[Tuple[object, object]] = []
        for i in range(layers):
            cin, cout = dims[i], dims[i + 1]
            scale = math.sqrt(2.0 / (cin * 9)) if i + 1 < layers else 0.1 * math.sqrt(1.0 / (cin * 9))
            w = rng.standard_normal((cout, cin, 3, 3)) * scale
            self.params.append((torch.tensor(w, dtype=torch.float32, device=self.device),
                                torch.zeros(cout, dtype=torch.float32, device=self.device)))
        self.dims = dims
        self._adam = None
        self.step_count = 0

    # -- parameters
    def state(self) -> dict:
        out = {}
        for i, (w, b) in enumerate(self.params):
            out[f"w{i}"] = w.cpu().numpy()
            out[f"b{i}"] = b.cpu().numpy()
        return out

    def load_state(self, state: dict):
        torch = self.torch
        for i in range(len(self.params)):
            self.params[i] = (torch.tensor(np.asarray(state[f"w{i}"]), dtype=torch.float32, device=self.device),
                              torch.tensor(np.asarray(state[f"b{i}"]), dtype=torch.float32, device=self.device))

    def save(self, path: str, **meta):
        np.savez(path, **self.state(), **{k: np.asarray(v) for k, v in meta.items()})

    @classmethod
    def load(cls, path: str, device: str = "cuda"):
        data = np.load(path)
        layers = sum(1 for k in data.files if k.startswith("w"))
        net = cls(layers=layers, channels=int(data["w0"].shape[0]), device=device)
        net.load_state({k: data[k] for k in data.files})
        meta = {k: data[k] for k in data.files if not (k[0] in "wb" and k[1:].isdigit())}
        return net, meta

    # -- features
    def features(self, y, xi, blur_std: float):
        """Input planes (n, 3, h, w) from observations y (n, h, w) and noise
        variances xi (n,)."""
        torch = self.torch
        n, h, w = y.shape
        x = torch.empty((n, IN_CHANNELS, h, w), dtype=torch.float32, device=self.device)
        x[:, 0] = y
        x[:, 1] = torch.as_tensor(np.log10(np.asarray(xi, np.float64)) / 4.0, dtype=torch.float32,
                                  device=self.device).view(n, 1, 1)
        x[:, 2] = blur_std / 4.0
        return x

    # -- passes
    def forward(self, x, keep: bool = False):
        """Network output (n, 2, h, w); with keep the layer outputs are kept for
        backward."""
        torch = self.torch
        n, _, h, w = x.shape
        acts = [x]
        cur = x
        for i, (wt, b) in enumerate(self.params):
            cout = wt.shape[0]
            out = torch.empty((n, cout, h, w), dtype=torch.float32, device=self.device)
            relu = 1 if i + 1 < len(self.params) else 0
            _check(self.lib.ep_tv_conv3x3_forward(n, cur.shape[1], cout, h, w, _ptr(cur), _ptr(wt),
                                                  _ptr(b), relu, _ptr(out),
                                                  ctypes.c_void_p(self.stream.cuda_stream)),
                   "ep_tv_conv3x3_forward")
            if keep:
                acts.append(out)
            cur = out
        if keep:
            self._acts = acts
        return cur

    def backward(self, dout):
        """Gradients [(dw, db)] of all layers for dL/dout, after forward(keep=True)."""
        torch = self.torch
        acts = self._acts
        n, _, h, w = dout.shape
        grads = [None] * len(self.params)
        g = dout
        for i in range(len(self.params) - 1, -1, -1):
            wt, b = self.params[i]
            cout, cin = wt.shape[0], wt.shape[1]
            work_bytes = self.lib.ep_tv_conv3x3_backward_work(n, cin, cout, h, w)
            work = torch.empty(int(work_bytes) // 4 + 1, dtype=torch.float32, device=self.device)
            dw = torch.empty_like(wt)
            db = torch.empty_like(b)
            dx = torch.empty((n, cin, h, w), dtype=torch.float32, device=self.device) if i > 0 else None
            y = acts[i + 1] if i + 1 < len(self.params) else None
            _check(self.lib.ep_tv_conv3x3_backward(n, cin, cout, h, w, _ptr(acts[i]), _ptr(wt), _ptr(y),
                                                   _ptr(g), _ptr(dx), _ptr(dw), _ptr(db), _ptr(work),
                                                   ctypes.c_size_t(work.numel() * 4),
                                                   ctypes.c_void_p(self.stream.cuda_stream)),
                   "ep_tv_conv3x3_backward")
            grads[i] = (dw, db)
            g = dx
        return grads

    def loss(self, out, y, mean, tau, log_xi, w_mean: float = W_MEAN):
        """Loss (device double tensor) and dL/dout against converged EP states
        (posterior mean (n, h, w), site precisions tau (n, 5, h, w)), for
        observations y (n, h, w) with log noise variances log_xi (n,)."""
        torch = self.torch
        n, _, h, w = out.shape
        dout = torch.empty_like(out)
        loss = torch.empty(1, dtype=torch.float64, device=self.device)
        _check(self.lib.ep_tv_warmstart_loss(n, h, w, _ptr(out), _ptr(y.contiguous()),
                                             _ptr(mean.contiguous()), _ptr(tau.contiguous()),
                                             _ptr(log_xi.contiguous()), ctypes.c_float(w_mean),
                                             _ptr(dout), _ptr(loss),
                                             ctypes.c_void_p(self.stream.cuda_stream)),
               "ep_tv_warmstart_loss")
        return loss, dout

    def adam(self, grads, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999,
             eps: float = 1e-8):
        torch = self.torch
        if self._adam is None:
            self._adam = [(torch.zeros_like(w), torch.zeros_like(w), torch.zeros_like(b), torch.zeros_like(b))
                          for w, b in self.params]
        self.step_count += 1
        for (w, b), (dw, db), (mw, vw, mb, vb) in zip(self.params, grads, self._adam):
            for p, g, m, v in ((w, dw, mw, vw), (b, db, mb, vb)):
                _check(self.lib.ep_tv_adam_step(p.numel(), _ptr(p), _ptr(g), _ptr(m), _ptr(v),
                                                self.step_count, ctypes.c_float(lr),
                                                ctypes.c_float(beta1), ctypes.c_float(beta2),
                                                ctypes.c_float(eps),
                                                ctypes.c_void_p(self.stream.cuda_stream)),
                       "ep_tv_adam_step")

    # -- use
    def predict(self, y, xi: float, blur_std: float):
        """Network output (6, h, w) for one observation y (h, w): predicted
        posterior mean y + out[0] and site precisions exp(out[1 + s]) / xi, which
        ``ep_tv_warm_start`` applies."""
        x = self.features(y.unsqueeze(0), [xi], blur_std)
        return self.forward(x)[0]
