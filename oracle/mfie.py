"""The magnetic-field integral equation and the combined-field equation of Sec. 2.1 (CFIE
with alpha = 0.5 for spheres, alpha = 1 for plates, Sec. 5.1) on the RWG basis, by plain
dense fills.

Test infrastructure: only the tests, the smoke check and the benchmark's CPU baseline use it.

The paper defers the operator to its refs [5], [7]; readings, each a plain restatement:

* MFIE for a closed PEC surface, exterior limit, Galerkin-tested with S_k:
      (1/2) <S_k, J> + <S_k, n x PV int R^ x [J(tau)/R^2 + dJ/dt(tau)/(c R)] dS' / (4 pi)>
          = <S_k, n x H_inc>,
  tau = t - R/c, R^ = (r - r')/R, n the outward unit normal of the test triangle (from the
  face's vertex order);
* envelopes (Sec. 1): d/dt -> D = d/dt + j w_c and the retardation phase e^{-j k_c R}; the
  equation is differentiated once in time, as the EFIE of Eq. 4 is, so with the CPPIF T
  (Eq. 3) and v = m - R/(c dt)
      K_m[k,k'] = (1/2) (DT)(m) <S_k, S_k'>
                + (1/4 pi) <S_k, n x int R^ x S_k' [(DT)(v)/R^2 + (D^2 T)(v)/(c R)] e^{-j k_c R} dS'>,
      W_l[k]   = <S_k, n x D H~inc(., l dt)>,  H~inc = (1/eta) (k x p) g(tau) e^{-j w_c (r.k/c + t_d)},
  (DT)(u) = T'(u)/dt + j w_c T(u) (D^2 T as in Eq. 4);
* the principal value over the test triangle itself vanishes (R^ and S' lie in its plane,
  so n x (R^ x S') is normal to it); pairs the EFIE treats as singular (a shared vertex,
  or centroids closer than twice the mean edge) integrate the source triangle with the
  7-point rule on each of 4^3 sub-triangles, the others with the 7-point rule;
* CFIE: alpha (Z_m I = V) + (1 - alpha) eta (K_m I = W), eta = sqrt(mu/eps);
* frequency domain at f_c: (DT) -> 1 and (D^2 T) -> j w, i.e. the kernel
  (1 + j k R)/R^2 e^{-j k R}/(4 pi) and the Gram factor 1/2.
"""
from __future__ import annotations

import math

import numpy as np

from . import efie, quad


def normals(rwg) -> np.ndarray:
    """Unit normals [nt, 3] of the faces, (b - a) x (c - a) of their vertex order."""
    a, b, c = (rwg.V[rwg.F[:, i]] for i in range(3))
    n = np.cross(b - a, c - a)
    return n / np.linalg.norm(n, axis=1)[:, None]


def subdivided_rule(levels: int):
    """The 7-point rule on each of the 4^levels congruent sub-triangles of the reference
    triangle: barycentric points [7 4^levels, 3] and weights summing to 1."""
    bary7, w7 = quad.cowper7()
    tris = [np.eye(3)]
    for _ in range(levels):
        nxt = []
        for T in tris:
            a, b, c = T
            ab, bc, ca = (a + b) / 2, (b + c) / 2, (c + a) / 2
            nxt += [np.array([a, ab, ca]), np.array([ab, b, bc]), np.array([ca, bc, c]), np.array([ab, bc, ca])]
        tris = nxt
    pts = np.concatenate([bary7 @ T for T in tris])
    w = np.tile(w7, len(tris)) / len(tris)
    return pts, w


def _dT(v, p: efie.Params, m=None):
    return p.T(v, 1, m) / p.dt + 1j * p.wc * p.T(v, 0, m)


def _kernel_td(m: np.ndarray, R: np.ndarray, p: efie.Params):
    """[nm, *R.shape]: [(DT)(v)/R^2 + (D^2 T)(v)/(c R)] e^{-j k_c R} / (4 pi)."""
    mb = m.reshape((-1,) + (1,) * R.ndim)
    v = mb - R[None] / p.cdt
    ph = np.exp(-1j * p.kc * R)[None] / (4 * math.pi)
    return (_dT(v, p, mb) / R[None] ** 2 + efie._d2T(v, p, 0, mb) / (p.c * R[None])) * ph


def _kernel_fd(m: np.ndarray, R: np.ndarray, p: efie.Params):
    return ((1 + 1j * p.kc * R) / R ** 2 * np.exp(-1j * p.kc * R) / (4 * math.pi))[None]


def _pair_blocks(g, nrm, t, tp, m, p, kern, src_rule):
    """K blocks [nm, n, 3, 3] of the curl term between the half-bases of test triangles t
    and source triangles tp (distinct), the source integrated with src_rule."""
    bary, ws = src_rule
    V, F = g.rwg.V, g.rwg.F
    A, B, C = (V[F[tp, i]] for i in range(3))
    Ps = bary[None, :, 0:1] * A[:, None] + bary[None, :, 1:2] * B[:, None] + bary[None, :, 2:3] * C[:, None]
    Ws = ws[None, :] * g.rwg.area[tp][:, None]                     # [n,ns]
    Pt, Wt = g.P[t], g.W[t]                                           # [n,7,3], [n,7]
    d = Pt[:, :, None, :] - Ps[:, None, :, :]                        # [n,7,ns,3]
    R = np.linalg.norm(d, axis=-1)
    Rh = d / R[..., None]
    f = kern(m, R, p)                                                 # [nm,n,7,ns]
    St = g.coef[t][:, :, None, None] * (Pt[:, None, :, :] - g.vfree[t][:, :, None, :])      # [n,3,7,3]
    Ss = g.coef[tp][:, :, None, None] * (Ps[:, None, :, :] - g.vfree[tp][:, :, None, :])    # [n,3,ns,3]
    nt = nrm[t]                                                       # [n,3]
    # S_p . (n x (R^ x S_q)) = (S_p . R^)(n . S_q) - (S_p . S_q)(n . R^)
    SpR = np.einsum("npax,nabx->npab", St, Rh)                        # [n,3,7,ns]
    nSq = np.einsum("nx,nqbx->nqb", nt, Ss)                           # [n,3,ns]
    SpSq = np.einsum("npax,nqbx->npqab", St, Ss)                      # [n,3,3,7,ns]
    nR = np.einsum("nx,nabx->nab", nt, Rh)                            # [n,7,ns]
    val = SpR[:, :, None] * nSq[:, None, :, None, :] - SpSq * nR[:, None, None]
    WW = Wt[:, :, None] * Ws[:, None, :]
    return np.einsum("mnab,nab,npqab->mnpq", f, WW, val)


def fill_dense(rwg, p: efie.Params, n_delays: int | None = None, freq: bool = False, chunk: int = 512):
    """Dense K_0..K_{N_g} (or the frequency-domain MFIE matrix at f_c if ``freq``)."""
    g = efie.Geometry(rwg)
    nrm = normals(rwg)
    ns, ntri = rwg.ns, len(rwg.F)
    if freq:
        m = np.zeros(1)
        kern = _kernel_fd
        gram = np.array([0.5 + 0j])
    else:
        if n_delays is None:
            n_delays = efie.n_delays_mot(g, p)
        m = np.arange(n_delays + 1, dtype=np.float64)
        kern = _kernel_td
        gram = 0.5 * _dT(m, p, m)
    out = np.zeros((len(m), ns, ns), dtype=complex)
    T_, TP_ = np.meshgrid(np.arange(ntri), np.arange(ntri), indexing="ij")
    T_, TP_ = T_.ravel(), TP_.ravel()
    diff = T_ != TP_
    near = g.singular_mask(T_, TP_) & diff
    far = ~g.singular_mask(T_, TP_) & diff
    rule7 = quad.cowper7()
    rule_near = subdivided_rule(3)
    for sel, rule in ((far, rule7), (near, rule_near)):
        idx = np.nonzero(sel)[0]
        step = chunk if rule is rule7 else max(1, chunk // 32)
        for s in range(0, len(idx), step):
            ii = idx[s:s + step]
            blk = _pair_blocks(g, nrm, T_[ii], TP_[ii], m, p, kern, rule)
            efie._assemble(g, T_[ii], TP_[ii], blk, out, ns)
    # Gram term on each face: (1/2) (DT)(m) int S_p . S_q
    tt = np.arange(ntri)
    S = g.coef[:, :, None, None] * (g.P[:, None, :, :] - g.vfree[:, :, None, :])            # [nt,3,7,3]
    G = np.einsum("na,npax,nqax->npq", g.W, S, S)
    efie._assemble(g, tt, tt, gram[:, None, None, None] * G[None], out, ns)
    return out[0] if freq else out


def _incident_h(rwg, p: efie.Params, khat, phat):
    """Tangential factor n x (k x p)/eta at every cubature point, [nt, 3]."""
    eta = math.sqrt(p.mu / p.eps)
    h = np.cross(np.asarray(khat, float), np.asarray(phat, float)) / eta
    return np.cross(normals(rwg), h[None, :])


def excitation(rwg, p: efie.Params, khat, phat, sigma: float, t_d: float, steps) -> np.ndarray:
    """W_l[k] = <S_k, n x D H~inc>: [len(steps), ns] for one plane wave."""
    g = efie.Geometry(rwg)
    nh = _incident_h(rwg, p, khat, phat)                              # [nt,3]
    steps = np.asarray(steps, dtype=np.float64)
    delay = g.P @ np.asarray(khat, float) / p.c                       # [nt,7]
    tau = steps[:, None, None] * p.dt - delay[None] - t_d
    gt = np.exp(-tau ** 2 / (2 * sigma ** 2))
    tf = (-tau / sigma ** 2 + 1j * p.wc) * gt * np.exp(-1j * p.wc * (delay + t_d))[None]        # [nl,nt,7]
    S = g.coef[:, :, None, None] * (g.P[:, None, :, :] - g.vfree[:, :, None, :])            # [nt,3,7,3]
    Sn = np.einsum("npax,nx->npa", S, nh)                              # [nt,3,7]
    contrib = np.einsum("lna,na,npa->lnp", tf, g.W, Sn)
    out = np.zeros((len(steps), rwg.ns), dtype=complex)
    for pp in range(3):
        np.add.at(out.T, g.k[:, pp], contrib[:, :, pp].T)
    return out


def excitation_fd(rwg, p: efie.Params, khat, phat) -> np.ndarray:
    """W[k] = <S_k, n x (k x p)/eta e^{-j k_c k.r}> at f_c: [ns]."""
    g = efie.Geometry(rwg)
    nh = _incident_h(rwg, p, khat, phat)
    ph = np.exp(-1j * p.kc * (g.P @ np.asarray(khat, float)))
    S = g.coef[:, :, None, None] * (g.P[:, None, :, :] - g.vfree[:, :, None, :])
    contrib = np.einsum("na,na,npax,nx->np", ph, g.W, S, nh)
    out = np.zeros(rwg.ns, dtype=complex)
    for pp in range(3):
        np.add.at(out, g.k[:, pp], contrib[:, pp])
    return out
