"""Seeded synthetic restoration problems.

This module only draws inputs: ground-truth images, blur kernels, sensing
matrices, noisy observations and the standard-normal probe vectors that the
Rao-Blackwellised Monte Carlo variance estimator consumes.  It contains none of
the expectation-propagation arithmetic, so both the FP64 oracle and the CUDA
path can take their inputs from here without sharing any of the method.

The paper's own test images (Cameraman, Flinstones, Mandrill, Shepp-Logan) are
not available; these generators stand in for them with the same sizes and the
same kind of structure (piecewise-constant objects, smooth background), see the
experimental section of the paper (Sec. V).

All draws use ``numpy.random.default_rng(seed)`` so a seed fixes a problem.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

__all__ = [
    "Problem",
    "piecewise_image",
    "uniform_kernel",
    "gaussian_kernel",
    "circular_blur",
    "denoise_problem",
    "deconv_problem",
    "cs_problem",
    "batched_problems",
    "rbmc_probes",
]


@dataclasses.dataclass
class Problem:
    """One restoration problem y = H x + n, n ~ N(0, xi I)."""

    kind: str                      # "denoise", "deconv" or "cs"
    x: np.ndarray                  # ground truth, (H, W) float64
    y: np.ndarray                  # observation: (H, W) for denoise/deconv, (M,) for cs
    xi: float                      # noise variance
    beta: float                    # TV parameter (lambda in the paper) or its EM start
    kernel: Optional[np.ndarray] = None   # (kh, kw) blur kernel, deconv only
    A: Optional[np.ndarray] = None        # (M, N) sensing matrix, cs only
    seed: int = 0
    patterns: Optional[np.ndarray] = None  # Hadamard CS: the M selected pattern indices

    @property
    def shape(self):
        return self.x.shape

    @property
    def n_pixels(self):
        return int(self.x.size)


def piecewise_image(h: int, w: int, rng: np.random.Generator, n_rect: int = 8,
                    n_disc: int = 0, grf_length: Optional[float] = None,
                    grf_std: float = 0.1, background: float = 0.5) -> np.ndarray:
    """Piecewise-constant test image.

    ``n_rect`` axis-aligned rectangles with intensities U[0,1] are painted on a
    constant background, then ``n_disc`` discs (radius U[w/32, w/8], intensity
    U[0,1]), then, if ``grf_length`` is given, a zero-mean Gaussian random field
    with a Gaussian spectral envelope of that length scale (pixels) and standard
    deviation ``grf_std`` is added.
    """
    img = np.full((h, w), background, dtype=np.float64)
    for _ in range(n_rect):
        r0, r1 = np.sort(rng.integers(0, h + 1, size=2))
        c0, c1 = np.sort(rng.integers(0, w + 1, size=2))
        if r1 == r0:
            r1 = min(h, r0 + 1)
        if c1 == c0:
            c1 = min(w, c0 + 1)
        img[r0:r1, c0:c1] = rng.uniform(0.0, 1.0)
    if n_disc:
        rr, cc = np.mgrid[0:h, 0:w]
        for _ in range(n_disc):
            cy, cx = rng.uniform(0, h), rng.uniform(0, w)
            rad = rng.uniform(w / 32.0, w / 8.0)
            img[(rr - cy) ** 2 + (cc - cx) ** 2 <= rad * rad] = rng.uniform(0.0, 1.0)
    if grf_length is not None:
        white = rng.standard_normal((h, w))
        fy = np.fft.fftfreq(h)[:, None]
        fx = np.fft.fftfreq(w)[None, :]
        envelope = np.exp(-2.0 * (math.pi * grf_length) ** 2 * (fy ** 2 + fx ** 2))
        field = np.real(np.fft.ifft2(np.fft.fft2(white) * envelope))
        sd = field.std()
        if sd > 0:
            img += grf_std * field / sd
    return img


def uniform_kernel(width: int) -> np.ndarray:
    """width x width box blur, normalised to unit sum."""
    return np.full((width, width), 1.0 / (width * width), dtype=np.float64)


def gaussian_kernel(width: int, std: float) -> np.ndarray:
    """width x width sampled Gaussian blur, normalised to unit sum."""
    r = np.arange(width) - (width - 1) / 2.0
    g = np.exp(-0.5 * (r / std) ** 2)
    k = np.outer(g, g)
    return k / k.sum()


def circular_blur(x: np.ndarray, kernel: np.ndarray) -> np.ndarray:
    """Periodic (circular) convolution of an image with a centred odd kernel.

    Used only to synthesise observations.  Computed with the FFT so that it is
    independent of both the oracle's and the CUDA path's operator code.
    """
    h, w = x.shape
    kh, kw = kernel.shape
    pad = np.zeros((h, w))
    pad[:kh, :kw] = kernel
    pad = np.roll(pad, (-(kh // 2), -(kw // 2)), axis=(0, 1))
    return np.real(np.fft.ifft2(np.fft.fft2(x) * np.fft.fft2(pad)))


def denoise_problem(h: int = 64, w: int = 64, sigma: float = 0.1, beta: float = 20.0,
                    seed: int = 0, n_rect: int = 8) -> Problem:
    """Denoising: 8 rectangles U[0,1] on a 0.5 background, Gaussian noise."""
    rng = np.random.default_rng(seed)
    x = piecewise_image(h, w, rng, n_rect=n_rect)
    y = x + sigma * rng.standard_normal((h, w))
    return Problem("denoise", x, y, sigma * sigma, beta, seed=seed)


def deconv_problem(h: int = 512, w: int = 512, kernel: Optional[np.ndarray] = None,
                   bsnr_db: Optional[float] = 40.0, beta0: float = 1.0, seed: int = 0,
                   n_rect: int = 8, n_disc: int = 4, grf_length: float = 32.0,
                   grf_std: float = 0.1, sigma: Optional[float] = None) -> Problem:
    """Deconvolution with a periodic blur.

    Unless ``sigma`` is given, the noise variance follows from the blurred
    signal-to-noise ratio, BSNR = 10 log10(var(Hx) / xi), with the
    mean-subtracted variance of Hx.
    """
    rng = np.random.default_rng(seed)
    if kernel is None:
        kernel = uniform_kernel(9)
    x = piecewise_image(h, w, rng, n_rect=n_rect, n_disc=n_disc,
                        grf_length=grf_length, grf_std=grf_std)
    hx = circular_blur(x, kernel)
    if sigma is not None:
        xi = float(sigma) ** 2
    else:
        xi = float(np.var(hx) / 10.0 ** (bsnr_db / 10.0))
    y = hx + math.sqrt(xi) * rng.standard_normal((h, w))
    return Problem("deconv", x, y, xi, beta0, kernel=np.asarray(kernel, np.float64), seed=seed)


def pixel_scale_image(h: int, w: int, rng: np.random.Generator, background: float = 0.5,
                      grf_length: float = 8.0, grf_std: float = 0.05) -> np.ndarray:
    """Piecewise-constant image whose features are sized in pixels, not relative
    to the image, so that small and large images share their local statistics:
    one rectangle per 64^2 pixels (sides U[4, 48]), one disc per 128^2 pixels
    (radius U[4, 16]), intensities U[0, 1], plus a Gaussian random field of
    length scale ``grf_length`` pixels and standard deviation ``grf_std``.  Shapes
    wrap around the torus."""
    img = np.full((h, w), background, dtype=np.float64)
    n_rect = max(1, (h * w) // (64 * 64))
    n_disc = max(1, (h * w) // (128 * 128))
    for _ in range(n_rect):
        r0, c0 = int(rng.integers(0, h)), int(rng.integers(0, w))
        rh, rw = int(rng.integers(4, 49)), int(rng.integers(4, 49))
        rows = np.arange(r0, r0 + rh) % h
        cols = np.arange(c0, c0 + rw) % w
        img[np.ix_(rows, cols)] = rng.uniform(0.0, 1.0)
    for _ in range(n_disc):
        cy, cx = rng.uniform(0, h), rng.uniform(0, w)
        rad = rng.uniform(4.0, 16.0)
        rr = np.arange(int(cy - rad) - 1, int(cy + rad) + 2)
        cc = np.arange(int(cx - rad) - 1, int(cx + rad) + 2)
        inside = (rr[:, None] + 0.0 - cy) ** 2 + (cc[None, :] + 0.0 - cx) ** 2 <= rad * rad
        value = rng.uniform(0.0, 1.0)
        sub = img[np.ix_(rr % h, cc % w)]
        sub[inside] = value
        img[np.ix_(rr % h, cc % w)] = sub
    white = rng.standard_normal((h, w))
    fy = np.fft.fftfreq(h)[:, None]
    fx = np.fft.fftfreq(w)[None, :]
    envelope = np.exp(-2.0 * (math.pi * grf_length) ** 2 * (fy ** 2 + fx ** 2))
    field = np.real(np.fft.ifft2(np.fft.fft2(white) * envelope))
    sd = field.std()
    if sd > 0:
        img += grf_std * field / sd
    return img


WARMSTART_BLUR_STD = 2.0


def warmstart_problem(h: int, w: int, seed: int, bsnr_db: float = 30.0,
                      beta: float = 1.0) -> Problem:
    """Deconvolution workload of the learned warm start: 15 x 15 Gaussian blur of
    standard deviation 2 pixels, BSNR 30 dB, image features sized in pixels
    (``pixel_scale_image``) so that networks trained on small images apply to
    large ones."""
    rng = np.random.default_rng(seed)
    kernel = gaussian_kernel(15, WARMSTART_BLUR_STD)
    x = pixel_scale_image(h, w, rng)
    hx = circular_blur(x, kernel)
    xi = float(np.var(hx) / 10.0 ** (bsnr_db / 10.0))
    y = hx + math.sqrt(xi) * rng.standard_normal((h, w))
    return Problem("deconv", x, y, xi, beta, kernel=kernel, seed=seed)


def cs_problem(h: int = 128, w: int = 128, ratio: float = 0.3, sigma: float = 0.01,
               beta0: float = 1.0, seed: int = 0, m: Optional[int] = None) -> Problem:
    """Compressive sensing with a dense Gaussian matrix, entries N(0, 1/M)."""
    rng = np.random.default_rng(seed)
    x = piecewise_image(h, w, rng, n_rect=8, n_disc=4, grf_length=h / 16.0)
    n = h * w
    if m is None:
        m = int(math.floor(ratio * n))
    A = rng.standard_normal((m, n)) / math.sqrt(m)
    y = A @ x.reshape(-1) + sigma * rng.standard_normal(m)
    return Problem("cs", x, y, sigma * sigma, beta0, A=A, seed=seed)


def _fwht(v: np.ndarray) -> np.ndarray:
    """Unnormalised Walsh-Hadamard transform of a vector of power-of-two length
    (Sylvester order): out[a] = sum_b (-1)^popcount(a & b) v[b]."""
    out = np.array(v, dtype=np.float64)
    n, h = out.size, 1
    while h < n:
        out = out.reshape(-1, 2, h)
        out = np.stack([out[:, 0] + out[:, 1], out[:, 0] - out[:, 1]], axis=1).reshape(-1)
        h *= 2
    return out


def _bitrev(k: int, bits: int) -> int:
    return int(format(k, f"0{bits}b")[::-1], 2) if bits else 0


def hadamard_cs_problem(h: int = 128, w: int = 128, ratio: float = 0.3, sigma: float = 0.01,
                        beta0: float = 1.0, seed: int = 0) -> Problem:
    """Compressive sensing with M uniformly chosen patterns of the 2-D Hadamard
    matrix (Paley-ordered indices p = kr * w + kc), scaled by 1/sqrt(M): the
    observation y = H x + n computed with a fast transform (Sylvester row =
    bit-reversed Paley index along each axis)."""
    rng = np.random.default_rng(seed)
    x = piecewise_image(h, w, rng, n_rect=8, n_disc=4, grf_length=h / 16.0)
    n = h * w
    m = int(math.floor(ratio * n))
    patterns = np.sort(rng.choice(n, size=m, replace=False))
    hb, wb = h.bit_length() - 1, w.bit_length() - 1
    sylv = np.array([(_bitrev(int(p) // w, hb) << wb) | _bitrev(int(p) % w, wb) for p in patterns])
    y = _fwht(x.reshape(-1))[sylv] / math.sqrt(m) + sigma * rng.standard_normal(m)
    return Problem("cs", x, y, sigma * sigma, beta0, seed=seed, patterns=patterns)


def batched_problems(n: int = 256, seed: int = 0, min_side: int = 64, max_side: int = 1024):
    """Uneven batch: sides log-uniform in [min_side, max_side] rounded to even,
    sigma U[0.02, 0.2], blur widths from {1, 5, 9, 15} (1 means denoising)."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(n):
        side = int(round(math.exp(rng.uniform(math.log(min_side), math.log(max_side)))))
        side += side % 2
        sigma = float(rng.uniform(0.02, 0.2))
        width = int(rng.choice([1, 5, 9, 15]))
        sub = int(rng.integers(0, 2 ** 31))
        if width == 1:
            p = denoise_problem(side, side, sigma=sigma, beta=1.0, seed=sub)
        else:
            p = deconv_problem(side, side, kernel=uniform_kernel(width), sigma=sigma,
                               seed=sub, grf_length=side / 16.0)
        out.append(p)
    return out


def rbmc_probes(n_samples: int, m: int, n: int, seed: int = 1234):
    """Standard-normal probe vectors for the perturbation sampler.

    Returns (eps1, eps2) with shapes (S, M) and (S, N): eps1 perturbs the
    observations, eps2 the cavity prior.  They are drawn once and kept fixed
    across sweeps.
    """
    rng = np.random.default_rng(seed)
    eps1 = rng.standard_normal((n_samples, m))
    eps2 = rng.standard_normal((n_samples, n))
    return eps1, eps2
