"""The accuracy measure of Sec. 2.4 on the library's RCS (``AimContext.march_spectrum``
followed by ``AimContext.rcs``): observation directions over the whole sphere with the
weights of its surface integral, and the thresholded dB-error norm of Eq. 2.

Host arithmetic on a few thousand RCS values; the march and the far field run in the
library.
"""
from __future__ import annotations

import math

import numpy as np


def sphere_grid(n_theta: int, n_phi: int):
    """Directions for the integrals of Eq. 2: n_theta Gauss-Legendre nodes in cos(theta)
    times n_phi equispaced azimuths.  Returns (rhat [nd, 3], theta-polarisation unit
    vectors [nd, 3], weights [nd] of sin(theta) dtheta dphi, theta [nd], phi [nd])."""
    mu, wmu = np.polynomial.legendre.leggauss(n_theta)
    theta = np.arccos(mu)
    phi = (2.0 * math.pi / n_phi) * np.arange(n_phi)
    th, ph = (a.ravel() for a in np.meshgrid(theta, phi, indexing="ij"))
    st, ct, sp, cp = np.sin(th), np.cos(th), np.sin(ph), np.cos(ph)
    rhat = np.stack([st * cp, st * sp, ct], axis=1)
    e_theta = np.stack([ct * cp, ct * sp, -st], axis=1)
    w = np.repeat(wmu, n_phi) * (2.0 * math.pi / n_phi)
    return rhat, e_theta, w, th, ph


def db_error(sigma, sigma_ref, weights, threshold_db: float = 80.0) -> float:
    """Eq. 2: with s^TH = max(10 log10 s, TH) - TH and TH the reference's peak minus
    ``threshold_db`` dB, sum w (s^TH - s_ref^TH)^2 / sum w (s_ref^TH)^2."""
    s = 10.0 * np.log10(np.maximum(np.asarray(sigma, dtype=np.float64), 1e-300))
    r = 10.0 * np.log10(np.maximum(np.asarray(sigma_ref, dtype=np.float64), 1e-300))
    th = r.max() - threshold_db
    s, r = np.maximum(s, th) - th, np.maximum(r, th) - th
    w = np.asarray(weights, dtype=np.float64)
    return float(np.sum(w * (s - r) ** 2) / np.sum(w * r ** 2))
