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
