"""Triangle cubature rules (barycentric points, weights summing to one)."""
from __future__ import annotations

import math

import numpy as np


def cowper7():
    """Cowper's 7-point rule, exact for polynomials of degree 5.

    Centroid with weight 9/40; the two orbits (a, a, 1-2a) with
    a = (6 -+ sqrt 15)/21 and weights (155 -+ sqrt 15)/1200.
    Returns ``(bary[7,3], w[7])``.
    """
    s = math.sqrt(15.0)
    a1, a2 = (6.0 - s) / 21.0, (6.0 + s) / 21.0
    w1, w2 = (155.0 - s) / 1200.0, (155.0 + s) / 1200.0
    pts = [(1 / 3, 1 / 3, 1 / 3)]
    wts = [9.0 / 40.0]
    for a, w in ((a1, w1), (a2, w2)):
        b = 1.0 - 2.0 * a
        pts += [(a, a, b), (a, b, a), (b, a, a)]
        wts += [w, w, w]
    return np.asarray(pts), np.asarray(wts)


def collapsed_gauss(n: int):
    """n x n Gauss-Legendre on the square mapped to the triangle (Duffy map).

    (s, t) in [0,1]^2 -> barycentric (s (1 - t), s t, 1 - s), Jacobian 2 s
    relative to the unit triangle's area.  Exact for total degree <= 2n - 2.
    """
    x, w = np.polynomial.legendre.leggauss(n)
    x = 0.5 * (x + 1.0)
    w = 0.5 * w
    S, Tt = np.meshgrid(x, x, indexing="ij")
    WS, WT = np.meshgrid(w, w, indexing="ij")
    S, Tt, W = S.ravel(), Tt.ravel(), (WS * WT).ravel()
    bary = np.stack([S * (1 - Tt), S * Tt, 1 - S], axis=1)
    return bary, W * 2.0 * S


def points(V: np.ndarray, F: np.ndarray, bary: np.ndarray) -> np.ndarray:
    """Cartesian cubature points ``[nt, nq, 3]``."""
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    return (bary[None, :, 0:1] * a[:, None] + bary[None, :, 1:2] * b[:, None]
            + bary[None, :, 2:3] * c[:, None])
