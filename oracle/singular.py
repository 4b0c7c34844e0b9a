"""Closed-form potential integrals over a flat triangle (singularity extraction).

For an observation point r and a triangle T' with vertices (A, B, C) listed
counter-clockwise about its unit normal n:

    I0(r)   = int_T' 1 / |r - r'| dS'
    I1(r)   = int_T' (r' - r) / |r - r'| dS'      (a vector)

written, as in Wilton et al. (IEEE TAP 1984) and Graglia (IEEE TAP 1993), as a
sum over the three edges of T'.  With rho the projection of r on the plane of T',
d = n.(r - A) the signed height, and for an edge running from a to b: unit
tangent t, outward in-plane normal u = t x n, l+- = (b|a - rho).t,
P0 = (a - rho).u (signed), R0^2 = P0^2 + d^2 and R+- = sqrt(R0^2 + l+-^2):

    I0 = sum_edges P0 ln((R+ + l+)/(R- + l-))
               - |d| [atan(P0 l+ / (R0^2 + |d| R+)) - atan(P0 l- / (R0^2 + |d| R-))]
    int_T' (rho' - rho)/R dS' = 1/2 sum_edges u [R0^2 ln((R+ + l+)/(R- + l-)) + l+ R+ - l- R-]
    I1 = int_T' (rho' - rho)/R dS' - d n I0

Used by the Galerkin fill of the impedance matrices; the paper states that the
fill uses singularity extraction (Sec. 3.1) without fixing the scheme.
"""
from __future__ import annotations

import numpy as np


def _dot(a, b):
    return np.sum(a * b, axis=-1)


def _log_ratio(Rp, lp, Rm, lm, R0sq):
    # R + l computed without cancellation: for l < 0, R + l = R0^2 / (R - l)
    def rpl(R, l):
        with np.errstate(divide="ignore", invalid="ignore"):
            return np.where(l >= 0, R + l, R0sq / (R - l))

    num, den = rpl(Rp, lp), rpl(Rm, lm)
    with np.errstate(divide="ignore", invalid="ignore"):
        out = np.log(num / den)
    return np.where((num > 0) & (den > 0), out, 0.0)


def potential_integrals(r, A, B, C):
    """Return ``(I0[...], I1[...,3])``; all inputs broadcast over leading axes."""
    r, A, B, C = (np.asarray(x, dtype=np.float64) for x in (r, A, B, C))
    n = np.cross(B - A, C - A)
    n = n / np.linalg.norm(n, axis=-1, keepdims=True)
    d = _dot(r - A, n)
    rho = r - d[..., None] * n
    ad = np.abs(d)
    scale = np.maximum(np.linalg.norm(B - A, axis=-1), np.linalg.norm(C - A, axis=-1))
    I0 = np.zeros(np.broadcast_shapes(d.shape, scale.shape))
    Iv = np.zeros(I0.shape + (3,))
    for a, b in ((A, B), (B, C), (C, A)):
        e = b - a
        t = e / np.linalg.norm(e, axis=-1, keepdims=True)
        u = np.cross(t, n)
        lp = _dot(b - rho, t)
        lm = _dot(a - rho, t)
        P0 = _dot(a - rho, u)
        R0sq = P0 * P0 + d * d
        Rp = np.sqrt(R0sq + lp * lp)
        Rm = np.sqrt(R0sq + lm * lm)
        tiny = (1e-13 * scale) ** 2
        ok = R0sq > tiny
        L = np.where(ok, _log_ratio(Rp, lp, Rm, lm, R0sq), 0.0)
        with np.errstate(divide="ignore", invalid="ignore"):
            at = (np.arctan(P0 * lp / (R0sq + ad * Rp)) - np.arctan(P0 * lm / (R0sq + ad * Rm)))
        at = np.where(ok, at, 0.0)
        I0 = I0 + P0 * L - ad * at
        Iv = Iv + 0.5 * u * (R0sq * L + lp * Rp - lm * Rm)[..., None]
    I1 = Iv - d[..., None] * n * I0[..., None]
    return I0, I1
