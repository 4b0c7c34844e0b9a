"""Band-limited interpolatory temporal basis (BLIF) with causal extrapolation (Sec. 3,
the alternative to the CPPIF of Eq. 3; Sec. 3.1.2: half-width M = 3 and N_omega = 2 N_samp
for ET-MOT).

Test infrastructure: only the tests, the smoke check and the benchmark's CPU baseline use it.

The paper defines both parts only through its refs [10], [15]; the readings here:

* the BLIF is the approximate prolate spheroidal (APS) interpolant of Knab (1979): with
  u in units of the time step and the envelope's half band f_bw = beta / dt,
      T(u) = sinc(u) w(u) for |u| < M, 0 otherwise,  sinc(u) = sin(pi u)/(pi u),
      w(u) = G(M^2 - u^2) / G(M^2),  G(s) = sinh(b sqrt(s)) / sqrt(s),  b = pi (1 - 2 beta),
  b being the guard band between the sampled band (pi per step) and the signal band
  (2 pi beta per step); T(n) = delta_n0 for every integer n, and T(+-M) = 0;
* causal form: the samples l+1 .. l+M-1 that T reaches at the test time l dt are not yet
  known; each is extrapolated from the N_samp = M samples l, l-1, .., l-M+1,
      I_{l+p} ~ sum_q E[p, q] I_{l-q},
  E[p] the least-squares fit of exp(j w_n p) ~ sum_q E[p, q] exp(-j w_n q) over
  N_omega = 2 N_samp frequencies w_n spaced evenly over the band [-2 pi beta, 2 pi beta]
  (edges included);
* the effective time factor of delay m is then
      T_m(v) = T(v) + sum_{p=1..M-1} E[p, m] T(v - m - p),  v = m - R/(c dt),
  (the second sum only for m < N_samp), so that sum_m Z_m I_{l-m} keeps the causal form of
  Eq. 5 with Z_m built from T_m.
"""
from __future__ import annotations

import math

import numpy as np


def _sinc_derivs(u: np.ndarray, dmax: int) -> list[np.ndarray]:
    """d^k/du^k sin(pi u)/(pi u), k = 0..dmax: the Taylor series of sin(x)/x for |pi u| < 1,
    else the product rule on sin(x) * x^-1 (d^i sin x = sin(x + i pi/2))."""
    x = math.pi * u
    small = np.abs(x) < 1.0
    xs, xl = x[small], x[~small]
    sl, cl = np.sin(xl), np.cos(xl)
    dsin = [sl, cl, -sl, -cl]
    inv = 1.0 / xl
    ipow = [inv]                        # x^-(j+1), j = 0..dmax
    for _ in range(dmax):
        ipow.append(ipow[-1] * inv)
    x2 = xs * xs
    out = []
    for k in range(dmax + 1):
        val = np.zeros_like(x)
        # sum_n (-1)^n x^(2n) / (2n+1)! differentiated k times: terms c_n x^(2n-k), n >= k/2;
        # with j = n - ceil(k/2) they are c_n x^(2j) x^(k mod 2), summed by Horner in x^2
        n0 = (k + 1) // 2
        acc = np.zeros_like(xs)
        for n in range(n0 + 14, n0 - 1, -1):
            c = (-1) ** n * math.factorial(2 * n) / math.factorial(2 * n - k) / math.factorial(2 * n + 1)
            acc = acc * x2 + c
        val[small] = acc * xs if k % 2 else acc
        acc = np.zeros_like(xl)
        for i in range(k + 1):          # d^(k-i) x^-1 = (-1)^(k-i) (k-i)! x^-(k-i+1)
            acc = acc + math.comb(k, i) * dsin[i % 4] * (-1) ** (k - i) * math.factorial(k - i) * ipow[k - i]
        val[~small] = acc
        out.append(val * math.pi ** k)
    return out


def _G_derivs(s: np.ndarray, b: float, dmax: int) -> list[np.ndarray]:
    """d^k/ds^k of G(s) = sinh(b sqrt s)/sqrt s, k = 0..dmax (<= 3).  With x = b sqrt(s),
    G = b i_0(x) (i_n the modified spherical Bessel functions) and (1/x d/dx)^k i_0 =
    i_k(x)/x^k, so G^(k)(s) = b^(2k+1) r_k(x) / 2^k with r_k = i_k(x)/x^k:
        r_k = sum_j (x^2/2)^j / (j! (2k+2j+1)!!)                       (x < 4, positive terms)
        r_0 = sinh x / x,  r_1 = (x cosh x - sinh x) / x^3,
        r_2 = ((x^2 + 3) sinh x - 3 x cosh x) / x^5,
        r_3 = ((x^3 + 15 x) cosh x - (6 x^2 + 15) sinh x) / x^7          (x >= 4)."""
    x = b * np.sqrt(s)
    lo = x < 4.0
    xs, xl = x[lo], x[~lo]
    h = 0.5 * xs * xs
    sh, ch = np.sinh(xl), np.cosh(xl)
    closed = [sh / xl, (xl * ch - sh) / xl ** 3, ((xl ** 2 + 3) * sh - 3 * xl * ch) / xl ** 5,
              ((xl ** 3 + 15 * xl) * ch - (6 * xl ** 2 + 15) * sh) / xl ** 7]
    out = []
    for k in range(dmax + 1):
        r = np.empty_like(x)
        acc = np.zeros_like(xs)
        for j in range(22, -1, -1):
            acc = acc * h + 1.0 / (math.factorial(j) * float(np.prod(np.arange(2 * k + 2 * j + 1, 0, -2))))
        r[lo] = acc
        r[~lo] = closed[k]
        out.append(b ** (2 * k + 1) * r / 2.0 ** k)
    return out


def T(u, M: int = 3, beta: float = 0.25, deriv: int = 0) -> np.ndarray:
    """T^(deriv)(u) of the APS BLIF of half-width M for the band fraction beta = f_bw dt."""
    if not 0.0 < beta < 0.5:
        raise ValueError("beta = f_bw dt must lie in (0, 1/2)")
    if deriv > 3:
        raise ValueError("derivatives up to the third")
    u = np.asarray(u, dtype=np.float64)
    out = np.zeros_like(u)
    inside = np.abs(u) < M
    ui = u[inside]
    b = math.pi * (1.0 - 2.0 * beta)
    s = M * M - ui * ui
    G = _G_derivs(s, b, deriv) + [None] * (3 - deriv)
    G0 = _G_derivs(np.array([float(M * M)]), b, 0)[0][0]
    # w and its u-derivatives by the chain rule through s = M^2 - u^2 (s' = -2u, s'' = -2)
    w = [G[0]]
    if deriv >= 1:
        w.append(-2.0 * ui * G[1])
    if deriv >= 2:
        w.append(4.0 * ui ** 2 * G[2] - 2.0 * G[1])
    if deriv >= 3:
        w.append(-8.0 * ui ** 3 * G[3] + 12.0 * ui * G[2])
    w = [x / G0 for x in w]
    sn = _sinc_derivs(ui, deriv)
    acc = np.zeros_like(ui)
    for k in range(deriv + 1):
        acc = acc + math.comb(deriv, k) * sn[k] * w[deriv - k]
    out[inside] = acc
    return out


def band_frequencies(M: int, beta: float) -> np.ndarray:
    """The N_omega = 2 M fit frequencies (radians per step), edges of the band included."""
    return 2.0 * math.pi * beta * np.linspace(-1.0, 1.0, 2 * M)


def extrapolation(M: int = 3, beta: float = 0.25, n_samp: int | None = None,
                  omegas: np.ndarray | None = None) -> np.ndarray:
    """E [M, n_samp] (row p = 0 unused): I_{l+p} ~ sum_q E[p, q] I_{l-q}, p = 1..M-1, each
    row the least-squares solution over the fit frequencies (numpy's lstsq)."""
    n_samp = M if n_samp is None else n_samp
    w = band_frequencies(M, beta) if omegas is None else np.asarray(omegas, float)
    A = np.exp(-1j * np.outer(w, np.arange(n_samp)))
    E = np.zeros((M, n_samp), dtype=complex)
    for p in range(1, M):
        E[p] = np.linalg.lstsq(A, np.exp(1j * w * p), rcond=None)[0]
    return E


def T_eff(m, v, M: int, beta: float, E: np.ndarray, deriv: int = 0) -> np.ndarray:
    """The causal time factor T_m(v) of delay m (broadcast against v), see the module
    docstring; E from ``extrapolation`` (its real part: the fit frequencies are symmetric)."""
    v = np.asarray(v, dtype=np.float64)
    m = np.broadcast_to(np.asarray(m, dtype=np.float64), v.shape)
    out = T(v, M, beta, deriv)
    Er = E.real
    n_samp = E.shape[1]
    for q in range(n_samp):
        sel = m == q
        if not np.any(sel):
            continue
        for p in range(1, M):
            out[sel] += Er[p, q] * T(v[sel] - q - p, M, beta, deriv)
    return out
