"""Mie series for plane-wave scattering by a PEC sphere (Sec. 5, reference [18]).

Textbook series (e.g. Bohren & Huffman, Ch. 4) in the perfect-conductor limit:
a_n = psi_n'(x)/xi_n'(x), b_n = psi_n(x)/xi_n(x), psi_n = x j_n(x),
xi_n = x h_n(x), x = k a.  Amplitudes
S1 = sum (2n+1)/(n(n+1)) (a_n pi_n + b_n tau_n), S2 = sum (2n+1)/(n(n+1)) (a_n tau_n + b_n pi_n),
pi_n = P_n^1(cos t)/sin t, tau_n = d P_n^1(cos t)/dt.  For an x-polarised wave along
+z, the co-polarised bistatic RCS in the E-plane (phi = 0) is 4 pi |S2|^2 / k^2 and in
the H-plane (phi = 90 deg) 4 pi |S1|^2 / k^2.
"""
from __future__ import annotations

import numpy as np
from scipy.special import spherical_jn, spherical_yn


def _pi_tau(nmax, theta):
    mu = np.cos(theta)
    pi = np.zeros((nmax + 1,) + np.shape(theta))
    tau = np.zeros_like(pi)
    pi[1] = 1.0
    for n in range(2, nmax + 1):
        pi[n] = (2 * n - 1) / (n - 1) * mu * pi[n - 1] - n / (n - 1) * pi[n - 2]
    for n in range(1, nmax + 1):
        tau[n] = n * mu * pi[n] - (n + 1) * pi[n - 1]
    return pi, tau


def rcs(ka: float, k: float, theta, plane: str = "E", nmax: int | None = None):
    """Bistatic RCS (m^2) at scattering angles ``theta`` (theta = pi: backscatter)."""
    theta = np.asarray(theta, dtype=np.float64)
    if nmax is None:
        nmax = int(ka + 4 * ka ** (1 / 3) + 10)
    n = np.arange(1, nmax + 1)
    jn, djn = spherical_jn(n, ka), spherical_jn(n, ka, derivative=True)
    yn, dyn = spherical_yn(n, ka), spherical_yn(n, ka, derivative=True)
    psi, dpsi = ka * jn, jn + ka * djn
    hn, dhn = jn + 1j * yn, djn + 1j * dyn
    xi, dxi = ka * hn, hn + ka * dhn
    a, b = dpsi / dxi, psi / xi
    pi, tau = _pi_tau(nmax, theta)
    c = ((2 * n + 1) / (n * (n + 1)))[:, None] if theta.ndim else (2 * n + 1) / (n * (n + 1))
    pi, tau = pi[1:], tau[1:]
    if theta.ndim:
        a, b = a[:, None], b[:, None]
    S1 = np.sum(c * (a * pi + b * tau), axis=0)
    S2 = np.sum(c * (a * tau + b * pi), axis=0)
    S = S2 if plane == "E" else S1
    return 4 * np.pi * np.abs(S) ** 2 / k ** 2


def db_error(sig, sig_ref, weights=None, below_peak_db: float = 80.0) -> float:
    """Thresholded dB-error norm of Eq. 2 (TH = peak - 80 dB), over sampled angles."""
    sig, sig_ref = np.asarray(sig), np.asarray(sig_ref)
    w = np.ones_like(sig) if weights is None else np.asarray(weights)
    TH = 10 * np.log10(sig_ref.max()) - below_peak_db
    a = np.maximum(10 * np.log10(np.maximum(sig, 1e-300)), TH) - TH
    r = np.maximum(10 * np.log10(np.maximum(sig_ref, 1e-300)), TH) - TH
    return float(np.sum(w * (a - r) ** 2) / np.sum(w * r ** 2))
