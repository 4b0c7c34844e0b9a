"""Radar cross section of a marched current envelope and the dB-error norm (Sec. 2.4).

Test infrastructure: only the tests, the smoke check and the benchmark's CPU baseline use it.

The paper measures accuracy by the co-polarised bistatic RCS at one frequency over all
scattering directions, compared in the thresholded dB norm of Eq. 2 (``mie.db_error``).
The RCS of a time-domain solution is its Fourier transform at that frequency divided by
that of the incident field.  Readings, each a plain restatement:

* envelope convention (Sec. 1): x(t) = Re{x~(t) e^{j w_c t}}, so for f > 0 near f_c the
  spectrum is X(f) = X~(Omega) / 2 with Omega = 2 pi (f - f_c) and
  X~(Omega) = int x~(t) e^{-j Omega t} dt; the factor 1/2 cancels in the ratio of
  scattered to incident spectra;
* the current envelope is the CPPIF interpolant of its samples (Eq. 3):
  x~(t) = sum_l I_l T(t/dt - l), so X~(Omega) = dt That(Omega dt) sum_l I_l e^{-j Omega l dt}
  with That(w) = int T(u) e^{-j w u} du;
* the incident envelope at the origin is that of Eq. 1, e(t) = g(t - t_d) e^{-j w_c t_d},
  g(tau) = exp(-tau^2 / (2 sigma^2)), with the closed-form transform
  E~(Omega) = sigma sqrt(2 pi) exp(-sigma^2 Omega^2 / 2) exp(-j (w_c + Omega) t_d);
* X~(Omega) / E~(Omega) is then the frequency-domain current for a unit plane wave
  p exp(-j k k.r) at f (the time-differentiated EFIE of Eq. 4 at f is the
  frequency-domain EFIE times j w), whose RCS ``efie.rcs_fd`` evaluates at k = 2 pi f / c.
"""
from __future__ import annotations

import math

import numpy as np

from scipy import integrate

from . import blif, efie, tbasis


def cppif_spectrum(w, Q: int = 2, npts: int = 24) -> np.ndarray:
    """That(w) = int T(u) e^{-j w u} du over the support (-1, Q] of the CPPIF of order Q
    (Eq. 3), by Gauss-Legendre quadrature with ``npts`` nodes on each unit piece."""
    w = np.atleast_1d(np.asarray(w, dtype=np.float64))
    x, wt = np.polynomial.legendre.leggauss(npts)
    out = np.zeros(w.shape, dtype=complex)
    for j in range(Q + 1):  # piece (j-1, j]
        u = j - 0.5 + 0.5 * x
        Tu = tbasis.T(u, Q)
        out += 0.5 * np.sum(wt * Tu * np.exp(-1j * np.outer(w, u)), axis=1)
    return out


def blif_spectrum(w: float, M: int, beta: float) -> complex:
    """That(w) = int T(u) e^{-j w u} du of the BLIF over (-M, M) (scipy's adaptive quadrature on
    each unit interval).  The extrapolation only changes how the samples are solved for: the
    envelope between them is still sum_l I_l T(t/dt - l)."""
    re = im = 0.0
    for j in range(-M, M):
        re += integrate.quad(lambda u: blif.T(np.array([u]), M, beta)[0] * math.cos(w * u), j, j + 1,
                             epsabs=1e-15, epsrel=1e-13)[0]
        im -= integrate.quad(lambda u: blif.T(np.array([u]), M, beta)[0] * math.sin(w * u), j, j + 1,
                             epsabs=1e-15, epsrel=1e-13)[0]
    return complex(re, im)


def basis_spectrum(w: float, p: efie.Params) -> complex:
    """That(w) of the temporal basis of ``p`` (CPPIF or BLIF)."""
    if p.basis == "blif":
        return blif_spectrum(w, p.M, p.beta)
    return complex(cppif_spectrum(w, p.Q)[0])


def envelope_spectrum_p(I: np.ndarray, p: efie.Params, Omega: float, l0: int = 1) -> np.ndarray:
    """``envelope_spectrum`` for the basis of ``p``."""
    l = np.arange(l0, l0 + len(I))
    s = np.tensordot(np.exp(-1j * Omega * l * p.dt), np.asarray(I), axes=(0, 0))
    return p.dt * basis_spectrum(Omega * p.dt, p) * s


def envelope_spectrum(I: np.ndarray, dt: float, Q: int, Omega: float, l0: int = 1) -> np.ndarray:
    """X~(Omega) of the interpolated envelope with samples I[l - l0] at t = l dt
    (``I``: [n_steps, ...])."""
    l = np.arange(l0, l0 + len(I))
    ph = np.exp(-1j * Omega * l * dt)
    s = np.tensordot(ph, np.asarray(I), axes=(0, 0))
    return dt * cppif_spectrum(Omega * dt, Q)[0] * s


def incident_spectrum(sigma: float, t_d: float, f_c: float, Omega: float) -> complex:
    """E~(Omega) of the Gaussian envelope of Eq. 1 at the origin."""
    wc = 2 * math.pi * f_c
    return sigma * math.sqrt(2 * math.pi) * math.exp(-0.5 * (sigma * Omega) ** 2) * np.exp(-1j * (wc + Omega) * t_d)


def rcs_td(rwg, p: efie.Params, I: np.ndarray, sigma: float, t_d: float, f: float, rhat, pol, l0: int = 1):
    """Bistatic RCS (m^2) at frequency f, directions rhat [nd, 3] and receive
    polarisations pol [nd, 3], of the marched envelope I [n_steps, ns] excited by the
    Gaussian plane wave of Eq. 1 (sigma, t_d; f_c = p.f_c)."""
    Omega = 2 * math.pi * (f - p.f_c)
    Ifd = envelope_spectrum_p(I, p, Omega, l0) / incident_spectrum(sigma, t_d, p.f_c, Omega)
    return efie.rcs_fd(rwg, efie.Params(dt=p.dt, f_c=f, Q=p.Q), Ifd, rhat, pol)


def sphere_directions(n_theta: int, n_phi: int):
    """Gauss-Legendre nodes in cos(theta) times n_phi equispaced phi: directions rhat,
    theta-polarisation unit vectors, and quadrature weights of the unit sphere
    (the integrals of Eq. 2 in sin(theta) dtheta dphi)."""
    x, wx = np.polynomial.legendre.leggauss(n_theta)
    th = np.arccos(x)
    ph = 2 * math.pi * np.arange(n_phi) / n_phi
    T, P = np.meshgrid(th, ph, indexing="ij")
    rhat = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], -1).reshape(-1, 3)
    eth = np.stack([np.cos(T) * np.cos(P), np.cos(T) * np.sin(P), -np.sin(T)], -1).reshape(-1, 3)
    w = np.repeat(wx, n_phi) * (2 * math.pi / n_phi)
    return rhat, eth, w, T.ravel(), P.ravel()
