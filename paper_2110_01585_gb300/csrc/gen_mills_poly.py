"""Writes mills_poly.cuh: polynomial fits of the truncated-normal functions
used by the FP32 tilted-moment kernel.

For a standard normal Z truncated to [b, inf), b >= 0, with the inverse Mills
ratio h(b) = phi(b) / Q(b) (Q the upper tail), the kernel needs
    g(b) = E[Z | Z > b] - b = h(b) - b          (g -> 1/b   as b -> inf)
    v(b) = Var[Z | Z > b]   = 1 - h(b) g(b)     (v -> 1/b^2 as b -> inf)
On u = (K - b) / (K + b) in (-1, 1] the scaled functions
    G(u) = g(b) (b + K) / K,    V(u) = v(b) ((b + K) / K)^2
are smooth and bounded (G -> 1/K, V -> 1/K^2 at u = -1), so a polynomial
in u of moderate degree reaches near-FP32 accuracy over all of [0, inf)
(degree 12: g within 5e-8, v within 1e-6 relative); the fit
is a least-squares Chebyshev fit at Chebyshev nodes of 40-digit values
(mpmath), converted to monomials for Horner evaluation.  Negative arguments
follow from the reflection Q(-b) = 1 - Q(b) in the kernel.

Run: python gen_mills_poly.py  (needs mpmath; the output is committed).
"""
import os

import mpmath as mp
import numpy as np
from numpy.polynomial import chebyshev as C

K = 2.0
DEGREE = int(os.environ.get("MILLS_DEGREE", "12"))
NODES = 200


def g_v(b):
    b = mp.mpf(b)
    q = mp.erfc(b / mp.sqrt(2)) / 2
    phi = mp.exp(-b * b / 2) / mp.sqrt(2 * mp.pi)
    h = phi / q
    g = h - b
    return g, 1 - h * g


def fit():
    mp.mp.dps = 40
    u = np.cos(np.pi * (np.arange(NODES) + 0.5) / NODES)
    b = K * (1 - u) / (1 + u)
    gv = np.array([[float(x) for x in g_v(bi)] for bi in b])
    G = gv[:, 0] * (b + K) / K
    V = gv[:, 1] * ((b + K) / K) ** 2
    pg = C.cheb2poly(C.chebfit(u, G, DEGREE))
    pv = C.cheb2poly(C.chebfit(u, V, DEGREE))
    return pg, pv


def main():
    pg, pv = fit()
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "mills_poly.cuh")
    with open(out, "w") as f:
        f.write("// Generated by gen_mills_poly.py; do not edit.\n")
        f.write("// g(b) = G(u) K / (b + K), v(b) = V(u) (K / (b + K))^2, u = (K - b) / (K + b), b >= 0;\n")
        f.write("// coefficients of u^0 .. u^%d (literals, so that the packed FMAs take them as\n" % DEGREE)
        f.write("// immediates instead of constant-bank loads).\n#pragma once\n\nnamespace eptv {\n\n")
        f.write("constexpr float kMillsK = %.1ff;\n" % K)
        f.write("constexpr int kMillsDegree = %d;\n\n" % DEGREE)
        for name, p in (("kMillsG", pg), ("kMillsV", pv)):
            f.write("__device__ constexpr float %s[%d] = {\n" % (name, len(p)))
            for c in p:
                f.write("    %.9ef,\n" % c)
            f.write("};\n\n")
        f.write("}  // namespace eptv\n")
    print("wrote", out)


if __name__ == "__main__":
    main()
