"""Moments of the Laplace-tilted edge marginal (oracle, FP64, test infrastructure).

Sec. III-C, Eq. marginal_tilted_un: for an edge n = (i, j) of V_k the tilted
marginal of u_n = x_i - x_j is

    P_k(u) ~ N(u; mu, s2) * phi(u),   mu = m_i - m_j,  s2 = c_i + c_j,

and for the l1-TV prior (Eq. L1_TV) phi(u) = exp(-lam |u|).  The paper states
that this is a mixture of two truncated Gaussians and omits the formulas; they
follow by completing the square on each half line:

  u >= 0:  N(u; mu, s2) e^{-lam u} = N(u; mu - lam s2, s2) * exp(-lam mu + lam^2 s2 / 2)
  u <  0:  N(u; mu, s2) e^{+lam u} = N(u; mu + lam s2, s2) * exp(+lam mu + lam^2 s2 / 2)

With s = sqrt(s2), a_plus = lam s - mu / s and a_minus = lam s + mu / s the
mass of each half is exp(-mu^2 / (2 s2)) * erfcx(a / sqrt 2) / 2, so the common
factor cancels and the mixture weights are

  w_plus = erfcx(a_plus / sqrt2) / (erfcx(a_plus / sqrt2) + erfcx(a_minus / sqrt2)).

Each half is a Gaussian truncated at 0; with the inverse Mills ratio
h(a) = phi(a) / Phi(-a) = sqrt(2/pi) / erfcx(a / sqrt2) its moments are

  E_plus  = (mu - lam s2) + s h(a_plus),   V_plus  = s2 [1 - h(a_plus)(h(a_plus) - a_plus)]
  E_minus = (mu + lam s2) - s h(a_minus),  V_minus = s2 [1 - h(a_minus)(h(a_minus) - a_minus)]

and the mixture moments are

  mean = w+ E+ + w- E-,  var = w+ V+ + w- V- + w+ w- (E+ - E-)^2,  E|u| = w+ E+ - w- E-.

For large a, h(a) - a and 1 - h(a)(h(a) - a) cancel.  There the oracle uses
Laplace's continued fraction for the Mills ratio, Phi(-a)/phi(a) =
1/(a + 1/(a + 2/(a + 3/(a + ...)))), so that g = h - a = t_1 with
t_k = k / (a + t_{k+1}), and 1 - h g = t_1 (t_2 - t_1), which has no
cancellation.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erfc, erfcx

SQRT2 = math.sqrt(2.0)
SQRT_2_OVER_PI = math.sqrt(2.0 / math.pi)

# Above this argument the continued fraction replaces the direct formulas.
CF_SWITCH = 5.0
CF_TERMS = 64


def _mills_tail(a: np.ndarray):
    """g(a) = h(a) - a and v(a) = 1 - h(a) g(a) from Laplace's continued fraction."""
    t_next = np.zeros_like(a)
    t2 = np.zeros_like(a)
    for k in range(CF_TERMS, 0, -1):
        t_next = k / (a + t_next)
        if k == 2:
            t2 = t_next.copy()
    t1 = t_next
    return t1, t1 * (t2 - t1)


def _log_erfcx(x: np.ndarray) -> np.ndarray:
    """log erfcx(x); for x < -20 erfcx(x) = exp(x^2) erfc(x) with erfc(x) = 2 - erfc(-x)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    neg = x < -20.0
    out[~neg] = np.log(erfcx(x[~neg]))
    out[neg] = x[neg] ** 2 + np.log(2.0 - erfc(-x[neg]))
    return out


def truncated_moments(a: np.ndarray):
    """For a standard normal truncated to [a, inf): (g, v) with
    mean = a + h(a) = a + g and variance = 1 - h(a)(h(a) - a) = v."""
    a = np.asarray(a, dtype=np.float64)
    g = np.empty_like(a)
    v = np.empty_like(a)
    big = a > CF_SWITCH
    small = ~big
    h = SQRT_2_OVER_PI / erfcx(a[small] / SQRT2)
    g[small] = h - a[small]
    v[small] = 1.0 - h * (h - a[small])
    if np.any(big):
        gb, vb = _mills_tail(a[big])
        g[big] = gb
        v[big] = vb
    return g, v


def laplace_tilted(mu, s2, lam):
    """Mean, variance and E|u| of P(u) ~ N(u; mu, s2) exp(-lam |u|).

    Arrays broadcast.  lam >= 0, s2 > 0.
    """
    mu = np.asarray(mu, dtype=np.float64)
    s2 = np.asarray(s2, dtype=np.float64)
    lam = float(lam)
    s = np.sqrt(s2)
    a_plus = lam * s - mu / s
    a_minus = lam * s + mu / s
    # w_plus = erfcx(a+/sqrt2) / (erfcx(a+/sqrt2) + erfcx(a-/sqrt2)), taken through
    # logarithms because erfcx overflows for arguments below about -26.
    d = _log_erfcx(a_minus / SQRT2) - _log_erfcx(a_plus / SQRT2)
    with np.errstate(over="ignore"):
        w_plus = 1.0 / (1.0 + np.exp(d))
        w_minus = 1.0 / (1.0 + np.exp(-d))
    g_plus, v_plus = truncated_moments(a_plus)
    g_minus, v_minus = truncated_moments(a_minus)
    # E_plus = (mu - lam s2) + s h(a_plus) = s (h(a_plus) - a_plus)
    e_plus = s * g_plus
    e_minus = -s * g_minus
    var_plus = s2 * v_plus
    var_minus = s2 * v_minus
    mean = w_plus * e_plus + w_minus * e_minus
    var = w_plus * var_plus + w_minus * var_minus + w_plus * w_minus * (e_plus - e_minus) ** 2
    eabs = w_plus * e_plus - w_minus * e_minus
    return mean, var, eabs


def gaussian_mixture_tilted(mu, s2, omega, v1, v2):
    """Mean and variance of P(u) ~ N(u; mu, s2) phi(u) for the two-Gaussian
    priors of Sec. II-B (oracle, FP64).

    MoG2-TV (Eq. MoG2_TV_prior): phi(u) = omega N(u; 0, v1) + (1 - omega) N(u; 0, v2).
    BG-TV (Eq. BG_TV) is the limit v2 -> 0, where the second component is the
    point mass delta(u); pass v2 = 0.

    Each product of Gaussians is a scaled Gaussian,
        N(u; 0, v) N(u; mu, s2) = N(mu; 0, v + s2) N(u; mu v / (v + s2), v s2 / (v + s2)),
    so P is a two-component Gaussian mixture with weights proportional to
    omega N(mu; 0, v1 + s2) and (1 - omega) N(mu; 0, v2 + s2) (for v2 = 0 the
    second component is a point mass at 0 with weight (1 - omega) N(mu; 0, s2)).
    Its mean is sum_k W_k m_k and its variance sum_k W_k (c_k + m_k^2) - mean^2.
    """
    mu = np.asarray(mu, dtype=np.float64)
    s2 = np.asarray(s2, dtype=np.float64)
    e1, e2 = v1 + s2, v2 + s2
    # weights from the log densities (normalising constants of each component)
    with np.errstate(divide="ignore"):  # omega = 0 or 1: that component has no weight
        l1 = np.log(omega) - 0.5 * np.log(2 * math.pi * e1) - mu ** 2 / (2 * e1)
        l2 = np.log(1.0 - omega) - 0.5 * np.log(2 * math.pi * e2) - mu ** 2 / (2 * e2)
    lmax = np.maximum(l1, l2)
    w1 = np.exp(l1 - lmax)
    w2 = np.exp(l2 - lmax)
    w1, w2 = w1 / (w1 + w2), w2 / (w1 + w2)
    m1, m2 = mu * v1 / e1, mu * v2 / e2
    c1, c2 = v1 * s2 / e1, v2 * s2 / e2
    mean = w1 * m1 + w2 * m2
    var = w1 * (c1 + m1 ** 2) + w2 * (c2 + m2 ** 2) - mean ** 2
    return mean, var


def folded_normal_mean(m, s2):
    """E|u| for u ~ N(m, s2): s sqrt(2/pi) exp(-m^2 / (2 s2)) + m erf(m / (s sqrt 2))."""
    from scipy.special import erf
    m = np.asarray(m, dtype=np.float64)
    s = np.sqrt(np.asarray(s2, dtype=np.float64))
    return s * SQRT_2_OVER_PI * np.exp(-m * m / (2.0 * s * s)) + m * erf(m / (s * SQRT2))
