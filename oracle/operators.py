"""Degradation operators H of Sec. II-A (oracle, FP64, test infrastructure).

(i) identity (denoising), (ii) convolution (deconvolution; periodic boundary,
centred odd kernel), (iii) a dense M x N sensing matrix (compressive sensing).
The convolution is written from its definition as a double sum, and its
transpose as the same sum with the kernel mirrored.
"""
from __future__ import annotations

import numpy as np


def conv_periodic(x: np.ndarray, kernel: np.ndarray) -> np.ndarray:
    """(H x)[r, c] = sum_{a, b} k[a, b] x[(r - a + kh//2) mod H, (c - b + kw//2) mod W]."""
    kh, kw = kernel.shape
    out = np.zeros_like(x, dtype=np.float64)
    for a in range(kh):
        for b in range(kw):
            # np.roll(x, t)[r] = x[r - t]
            out += kernel[a, b] * np.roll(x, (a - kh // 2, b - kw // 2), axis=(0, 1))
    return out


def conv_periodic_t(x: np.ndarray, kernel: np.ndarray) -> np.ndarray:
    """Adjoint of :func:`conv_periodic`: (H^T z)[r, c] = sum k[a, b] z[r + a - kh//2, c + b - kw//2]."""
    kh, kw = kernel.shape
    out = np.zeros_like(x, dtype=np.float64)
    for a in range(kh):
        for b in range(kw):
            out += kernel[a, b] * np.roll(x, (-(a - kh // 2), -(b - kw // 2)), axis=(0, 1))
    return out


def conv_matrix(height: int, width: int, kernel: np.ndarray) -> np.ndarray:
    """Dense N x N matrix of the periodic convolution (small images only)."""
    n = height * width
    mat = np.zeros((n, n))
    for p in range(n):
        e = np.zeros(n)
        e[p] = 1.0
        mat[:, p] = conv_periodic(e.reshape(height, width), kernel).reshape(-1)
    return mat
