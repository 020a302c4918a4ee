"""The four matchings V1..V4 of the 4-neighbour pixel graph (oracle, test infrastructure).

Sec. II-B (Eq. prior0, Eq. prior1 and the caption of Fig. 1): the set V of
4-neighbour pixel pairs is split into four subsets V_k such that no pixel
appears twice inside one V_k, and each pixel is in one edge of every V_k.  The
figure that fixes the geometry is missing from the text; the counts the paper
gives (2N gradients, D_k of size N/2 x N) hold on a torus with even H and W.
The reading used here:

  V1: horizontal (r, 2a)   - (r, 2a + 1)
  V2: horizontal (r, 2a+1) - (r, 2a + 2 mod W)
  V3: vertical   (2b, c)   - (2b + 1, c)
  V4: vertical   (2b+1, c) - (2b + 2 mod H, c)

With ``periodic=False`` the wrap-around edges of V2 and V4 are dropped (and
odd sizes are allowed); pixels with no edge in V_k keep site k at its initial
value.  ``periodic_rows`` (default: ``periodic``) decides the wrap of V4 alone,
so that a band of rows cut from a torus keeps its wrapping columns.  Pixel p = r * W + c (row-major).  The edge difference is
u = x_first - x_second, i.e. left minus right and top minus bottom.
"""
from __future__ import annotations

import numpy as np


def edges(height: int, width: int, k: int, periodic: bool = True, periodic_rows=None):
    """Return (first, second) flat pixel indices of the edges of V_k, k in 1..4."""
    periodic_rows = periodic if periodic_rows is None else periodic_rows
    if (periodic and width % 2) or (periodic_rows and height % 2):
        raise ValueError("periodic boundary needs even height and width")
    first, second = [], []
    for r in range(height):
        for c in range(width):
            if k == 1 and c % 2 == 0 and c + 1 < width:
                first.append(r * width + c)
                second.append(r * width + c + 1)
            elif k == 2 and c % 2 == 1:
                cn = c + 1
                if cn == width:
                    if not periodic:
                        continue
                    cn = 0
                if cn == c:
                    continue
                first.append(r * width + c)
                second.append(r * width + cn)
            elif k == 3 and r % 2 == 0 and r + 1 < height:
                first.append(r * width + c)
                second.append((r + 1) * width + c)
            elif k == 4 and r % 2 == 1:
                rn = r + 1
                if rn == height:
                    if not periodic_rows:
                        continue
                    rn = 0
                if rn == r:
                    continue
                first.append(r * width + c)
                second.append(rn * width + c)
    return np.asarray(first, dtype=np.int64), np.asarray(second, dtype=np.int64)
