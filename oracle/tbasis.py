"""Causal piecewise-polynomial interpolatory temporal basis (CPPIF), Sec. 3, Eq. 3.

T(u) with u in units of the time step.  Order Q uses, on the interval
(n-1, n] of the time axis, the Lagrange polynomial through the samples
n, n-1, ..., n-Q.  Seen from one sample, the basis is therefore non-zero on
(-1, Q] and, on its piece (j-1, j] (j = 0..Q),

    T(u) = prod_{k=0..Q, k != j} (u - j + k) / (k - j).

Derivatives are those of the local piece (no Dirac terms at the knots); at a knot
the piece (j-1, j] to its left is used, so a value at u = j belongs to piece j.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import polynomial as P


def piece_coeffs(Q: int) -> list[np.ndarray]:
    """Power-series coefficients (ascending) of T on each piece j = 0..Q."""
    out = []
    for j in range(Q + 1):
        c = np.array([1.0])
        for k in range(Q + 1):
            if k == j:
                continue
            # factor (u - j + k) / (k - j)
            c = P.polymul(c, np.array([(k - j), 1.0]) / (k - j))
        out.append(c)
    return out


def T(u, Q: int = 2, deriv: int = 0) -> np.ndarray:
    """Evaluate T^(deriv)(u) elementwise."""
    u = np.asarray(u, dtype=np.float64)
    out = np.zeros_like(u)
    j = np.ceil(u)
    for jj, c in enumerate(piece_coeffs(Q)):
        cd = P.polyder(c, deriv) if deriv else c
        sel = j == jj
        if np.any(sel):
            out[sel] = P.polyval(u[sel], cd)
    return out
