"""Fast Léja points on [-2, 2] (oracle; test infrastructure only).

Section 3, Eq. (Léja5) defines a Léja sequence on an interval greedily: each new point
maximises the product of distances to the points already chosen. The paper uses the "fast"
variant of Baglama, Calvetti and Reichel (1998), precomputed once on [-2, 2] and mapped
affinely to the spectral interval (Section 3.1, Eq. z_mapping). The fast variant restricts the
maximisation to the midpoints of the gaps between consecutive chosen points.

Reading fixed by this library (the paper leaves it open):
  * xi_0 = 2 (the right end; the paper starts "usually" at lambda_max), xi_1 = -2;
  * candidates are the midpoints (a + b) / 2 of neighbours in the sorted chosen set;
  * the score of x is prod_{k=0}^{j-1} |x - xi_k|, multiplied left to right in k order, FP64;
  * the largest score wins; scores within a relative 1e-10 of the largest count as tied, and
    the smallest tied x wins. (Symmetric candidates +-x tie exactly in exact arithmetic, and
    floating-point rounding would otherwise break those ties arbitrarily; with the tolerance the
    sequence equals the one computed in exact rational arithmetic.)
"""
from __future__ import annotations

import numpy as np

TIE_RTOL = 1e-10


def fast_leja_points(count: int) -> np.ndarray:
    """First `count` fast Léja points on [-2, 2] (Eq. Léja5 restricted to gap midpoints)."""
    if count < 0:
        raise ValueError("count must be non-negative")
    pts: list[float] = []
    if count >= 1:
        pts.append(2.0)
    if count >= 2:
        pts.append(-2.0)
    while len(pts) < count:
        srt = sorted(pts)
        cand = np.array([(a + b) / 2.0 for a, b in zip(srt[:-1], srt[1:])], dtype=np.float64)
        score = np.ones_like(cand)
        for xk in pts:                      # k = 0 .. j-1, left to right
            score = score * np.abs(cand - xk)
        best = score.max()
        # candidates are ascending, so the first (near-)maximiser is the smallest x
        idx = int(np.flatnonzero(score >= best * (1.0 - TIE_RTOL))[0])
        pts.append(float(cand[idx]))
    return np.array(pts, dtype=np.float64)
