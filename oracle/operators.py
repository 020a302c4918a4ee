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


def _popcount(a: np.ndarray) -> np.ndarray:
    """Set bits of each uint64 (NumPy's own routine where it has one)."""
    if hasattr(np, "bitwise_count"):
        return np.bitwise_count(a)
    a = a.astype(np.uint64)
    out = np.zeros(a.shape, dtype=np.uint64)
    while np.any(a):
        out += a & np.uint64(1)
        a = a >> np.uint64(1)
    return out


def paley_to_sylvester(k: int, bits: int) -> int:
    """Row of the Sylvester-ordered Hadamard matrix that holds the Paley-ordered
    Walsh function k: the Paley index with its bits reversed."""
    out = 0
    for i in range(bits):
        if k >> i & 1:
            out |= 1 << (bits - 1 - i)
    return out


def hadamard_matrix(height: int, width: int, patterns) -> np.ndarray:
    """Sec. II-A (iii): M rows of the 2-D Hadamard matrix (the Kronecker product
    of the 1-D matrices of sizes height and width, both powers of two), scaled
    by 1 / sqrt(M) so that every column has unit norm like the Gaussian sensing
    matrix with entries N(0, 1/M).  patterns: M pattern indices p = kr * width + kc,
    kr and kc Paley-ordered Walsh indices along rows and columns.  Entry
    (a, b) of the Sylvester-ordered matrix is (-1)^popcount(a & b)."""
    hb, wb = int(height).bit_length() - 1, int(width).bit_length() - 1
    if (1 << hb) != height or (1 << wb) != width:
        raise ValueError("the Hadamard operator needs power-of-two sides")
    n = height * width
    cols = np.arange(n, dtype=np.uint64)
    rows = np.empty((len(patterns), n))
    for i, p in enumerate(patterns):
        kr, kc = divmod(int(p), width)
        s = np.uint64((paley_to_sylvester(kr, hb) << wb) | paley_to_sylvester(kc, wb))
        rows[i] = 1.0 - 2.0 * (_popcount(cols & s) & 1)
    return rows / np.sqrt(len(patterns))
