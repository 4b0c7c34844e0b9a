"""Far-field objective of a march and its gradient with respect to the incident
envelope samples, by dense linear algebra (the reference for the adjoint march).

Not in the paper: the gradient is a library feature built on the march of Eq. 5.
Definitions (readings, each a plain restatement):

* incident envelope on the time grid: E~inc(r, t) = p e(t - r.k/c) e^{-j k_c r.k} with
  e(tau) = sum_i a_i T(tau/dt - i) (the CPPIF of Eq. 3 as the interpolant of the
  envelope samples a_i).  Tested as in Eq. 4, V_l[k] = <S_k, D E~inc(., l dt)> =
  sum_i a_i B_{l-i}[k] with the taps
      B_s[k] = <S_k, p ((T'(s - u)/dt + j w_c T(s - u)) e^{-j k_c r.k}>,  u = r.k/(c dt);
* far-field envelope in direction r (transverse unit vectors e_1, e_2, reading R24):
      F_q(n) = -mu/(4 pi) sum_l sum_k I_l[k] A_{n-l}[q][k],
      A_s[q][k] = int S_k(r).e_q (DT)(s + r.r'/(c dt)) e^{+j k_c r.r'} dS',
  (DT)(u) = T'(u)/dt + j w_c T(u);
* objective J = sum_n sum_dirs sum_q |F_q(n)|^2 over a given range of n;
* with the march I = M^{-1} V (M block lower-triangular Toeplitz in Z_0..Z_{N_g}),
  dJ/d(conj a) = B^H M^{-H} A^H F  (Wirtinger derivative of a real function).
"""
from __future__ import annotations

import numpy as np

from . import efie, tbasis
from .constants import MU0


def _half_bases(rwg):
    g = efie.Geometry(rwg)
    S = (g.P[:, None, :, :] - g.vfree[:, :, None, :]) * g.coef[:, :, None, None]   # [nt,3,7,3]
    return g, S


def incident_taps(rwg, p: efie.Params, khat, phat, s_range):
    """B_s[k] for s in s_range (list of ints): [len(s_range), ns]."""
    if p.basis != "cppif":
        raise NotImplementedError("the adjoint taps interpolate with the CPPIF")
    g, S = _half_bases(rwg)
    khat, phat = np.asarray(khat, float), np.asarray(phat, float)
    u = (g.P @ khat) / p.cdt                                           # [nt,7]
    ph = np.exp(-1j * p.kc * (g.P @ khat))
    sp = np.einsum("tpqx,x->tpq", S, phat)                            # [nt,3,7]
    out = np.zeros((len(s_range), rwg.ns), dtype=complex)
    for si, s in enumerate(s_range):
        v = s - u
        f = (tbasis.T(v, p.Q, 1) / p.dt + 1j * p.wc * tbasis.T(v, p.Q, 0)) * ph
        contrib = np.einsum("tq,tq,tpq->tp", f, g.W, sp)
        for pp in range(3):
            np.add.at(out[si], g.k[:, pp], contrib[:, pp])
    return out


def farfield_taps(rwg, p: efie.Params, rhat, e1, e2, s_range):
    """A_s[d][q][k] for directions d, transverse components q: [len(s_range), nd, 2, ns]."""
    if p.basis != "cppif":
        raise NotImplementedError("the adjoint taps interpolate with the CPPIF")
    g, S = _half_bases(rwg)
    rhat = np.atleast_2d(rhat)
    E = np.stack([np.atleast_2d(e1), np.atleast_2d(e2)], axis=1)     # [nd,2,3]
    out = np.zeros((len(s_range), len(rhat), 2, rwg.ns), dtype=complex)
    for d in range(len(rhat)):
        w = (g.P @ rhat[d]) / p.cdt
        ph = np.exp(1j * p.kc * (g.P @ rhat[d]))
        for q in range(2):
            sp = np.einsum("tpqx,x->tpq", S, E[d, q])
            for si, s in enumerate(s_range):
                v = s + w
                f = (tbasis.T(v, p.Q, 1) / p.dt + 1j * p.wc * tbasis.T(v, p.Q, 0)) * ph
                contrib = np.einsum("tq,tq,tpq->tp", f, g.W, sp)
                for pp in range(3):
                    np.add.at(out[si, d, q], g.k[:, pp], contrib[:, pp])
    return out


def excitation_from_samples(B, s_range, a, i0, n_steps):
    """V_l = sum_i a_i B_{l-i}, l = 1..n_steps, samples a_i for i = i0..i0+len(a)-1."""
    V = np.zeros((n_steps, B.shape[1]), dtype=complex)
    for l in range(1, n_steps + 1):
        for si, s in enumerate(s_range):
            i = l - s
            if i0 <= i < i0 + len(a):
                V[l - 1] += a[i - i0] * B[si]
    return V


def farfield(A, s_range, I, n_range, mu: float = MU0):
    """F(n)[d][q] = -mu/4pi sum_l sum_k A_{n-l}[d][q][k] I_l[k]; I is [n_steps, ns] (l from 1);
    mu the background permeability (vacuum by default)."""
    nd = A.shape[1]
    F = np.zeros((len(n_range), nd, 2), dtype=complex)
    for ni, n in enumerate(n_range):
        for si, s in enumerate(s_range):
            l = n - s
            if 1 <= l <= len(I):
                F[ni] += np.einsum("dqk,k->dq", A[si], I[l - 1])
    return -mu / (4 * np.pi) * F


def objective(F):
    return float(np.sum(np.abs(F) ** 2))


def gradient(Z, B, sB, A, sA, a, i0, n_steps, n_range, mu: float = MU0):
    """(J, dJ/d conj(a)) with the march solved densely: Z[N_g+1, ns, ns]."""
    ns = Z.shape[1]
    ng = Z.shape[0] - 1
    V = excitation_from_samples(B, sB, a, i0, n_steps)
    from .march import march_dense

    I = march_dense(Z, V[:, None, :])[:, 0, :]
    F = farfield(A, sA, I, n_range, mu)
    J = objective(F)
    # G_l = dJ/d conj(I_l) = sum_n (-mu/4pi)^* A_{n-l}^H F(n)
    G = np.zeros((n_steps, ns), dtype=complex)
    c = np.conj(-mu / (4 * np.pi))
    for ni, n in enumerate(n_range):
        for si, s in enumerate(sA):
            l = n - s
            if 1 <= l <= n_steps:
                G[l - 1] += c * np.einsum("dqk,dq->k", np.conj(A[si]), F[ni])
    # M^H lam = G: backward march with Z_m^H
    lam = np.zeros_like(G)
    ZH = np.conj(np.transpose(Z, (0, 2, 1)))
    for l in range(n_steps, 0, -1):
        r = G[l - 1].copy()
        for m in range(1, ng + 1):
            if l + m <= n_steps:
                r -= ZH[m] @ lam[l + m - 1]
        lam[l - 1] = np.linalg.solve(ZH[0], r)
    grad = np.zeros(len(a), dtype=complex)
    for ii in range(len(a)):
        i = i0 + ii
        for si, s in enumerate(sB):
            l = i + s
            if 1 <= l <= n_steps:
                grad[ii] += np.conj(B[si]) @ lam[l - 1]
    return J, grad
