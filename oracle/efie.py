"""Envelope EFIE of ET-MOT: impedance matrices Z_m (Eq. 4) and excitation V_l (Eq. 1).

Readings (the paper defers the matrix entries to its references [5], [7]):

* envelope convention x(t) = Re{x~(t) e^{+j w_c t}} (Sec. 1, "baseband
  representation"); the envelope of d/dt is D = d/dt + j w_c;
* time-differentiated EFIE (alpha = 1 in Sec. 2.1's CFIE), Galerkin tested with
  the RWG functions at t = l dt (Sec. 3).  With the expansion of Eq. 3 this gives

    Z_m[k,k'] = int_Tk int_Tk' [ mu/(4 pi) S_k.S_k' (D^2 T)(m - R/(c dt))
                + 1/(4 pi eps) (div S_k)(div' S_k') T(m - R/(c dt)) ] e^{-j k_c R} / R

  with (D^2 T)(u) = T''(u)/dt^2 + 2 j w_c T'(u)/dt - w_c^2 T(u), and
  V_l[k] = <S_k, D E~inc(., l dt)>;
* cubature: Cowper's 7-point rule on test and source triangles.  Triangle pairs
  that share a vertex, or whose centroids are closer than twice the mean edge
  length, use singularity extraction: f(R)/R = f(0)/R + (f(R) - f(0))/R, the first
  part's inner integral in closed form (``singular``), the bounded remainder by
  cubature (its R = 0 value is the one-sided derivative f'(0+)).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import blif, quad, singular, tbasis
from .constants import C0, EPS0, MU0
from .rwg import RWG


@dataclasses.dataclass
class Params:
    """Time step, carrier, temporal basis and the homogeneous background medium (Sec. 2.1:
    relative permittivity and permeability; vacuum by default).  The basis is the CPPIF of
    order Q (Eq. 3), or with ``basis="blif"`` the BLIF of half-width M for the band fraction
    beta = f_bw dt with its causal extrapolation (``blif``)."""
    dt: float
    f_c: float
    Q: int = 2
    eps_r: float = 1.0
    mu_r: float = 1.0
    basis: str = "cppif"
    M: int = 3
    beta: float = 0.25

    def __post_init__(self):
        if self.basis not in ("cppif", "blif"):
            raise ValueError("basis is 'cppif' or 'blif'")
        self._E = blif.extrapolation(self.M, self.beta) if self.basis == "blif" else None

    @property
    def support(self) -> int:
        """Upper end of the basis' support in steps: Q (CPPIF, (-1, Q]) or M (BLIF, (-M, M))."""
        return self.Q if self.basis == "cppif" else self.M

    def T(self, v, deriv: int = 0, m=None) -> np.ndarray:
        """T^(deriv)(v); with the delay ``m`` (broadcast against v) the causal time factor
        of that delay, which for the BLIF adds the extrapolated samples."""
        if self.basis == "cppif":
            return tbasis.T(v, self.Q, deriv)
        if m is None:
            return blif.T(v, self.M, self.beta, deriv)
        return blif.T_eff(m, v, self.M, self.beta, self._E, deriv)

    @property
    def wc(self) -> float:
        return 2.0 * math.pi * self.f_c

    @property
    def c(self) -> float:
        return C0 / math.sqrt(self.eps_r * self.mu_r)

    @property
    def mu(self) -> float:
        return MU0 * self.mu_r

    @property
    def eps(self) -> float:
        return EPS0 * self.eps_r

    @property
    def kc(self) -> float:
        return self.wc / self.c

    @property
    def cdt(self) -> float:
        return self.c * self.dt


# ----------------------------------------------------------------------------
# time factors
# ----------------------------------------------------------------------------


def _d2T(v, p: Params, extra_deriv: int = 0, m=None):
    """(D^2 T)^(extra_deriv)(v) in physical units of the T argument (the time factor of
    delay ``m`` where given)."""
    T0 = p.T(v, 0 + extra_deriv, m)
    T1 = p.T(v, 1 + extra_deriv, m)
    T2 = p.T(v, 2 + extra_deriv, m)
    return T2 / p.dt ** 2 + 2j * p.wc * T1 / p.dt - p.wc ** 2 * T0


def time_kernels(m: np.ndarray, R: np.ndarray, p: Params):
    """f^A_m(R) = (D^2 T)(m - R/cdt) e^{-j k R},  f^phi_m(R) = T(m - R/cdt) e^{-j k R}.

    ``m`` has shape [nm]; the result has shape [nm, *R.shape].
    """
    mb = m.reshape((-1,) + (1,) * R.ndim)
    v = mb - R[None] / p.cdt
    ph = np.exp(-1j * p.kc * R)[None]
    return _d2T(v, p, 0, mb) * ph, p.T(v, 0, mb) * ph


def time_kernels_at0(m: np.ndarray, p: Params):
    """Values and one-sided R-derivatives at R = 0+ of both time kernels."""
    v = m.astype(np.float64)
    fA0, fP0 = _d2T(v, p, 0, v), p.T(v, 0, v).astype(complex)
    dA0 = -_d2T(v, p, 1, v) / p.cdt - 1j * p.kc * fA0
    dP0 = -p.T(v, 1, v) / p.cdt - 1j * p.kc * fP0
    return fA0, fP0, dA0, dP0


def freq_kernels(R: np.ndarray, p: Params):
    """Frequency-domain EFIE kernels at f_c, shaped like ``time_kernels`` with nm = 1."""
    g = np.exp(-1j * p.kc * R)[None]
    return 1j * p.wc * g, -1j / p.wc * g


def freq_kernels_at0(p: Params):
    return (np.array([1j * p.wc]), np.array([-1j / p.wc + 0j]),
            np.array([1j * p.wc * (-1j * p.kc)]), np.array([-1j / p.wc * (-1j * p.kc)]))


# ----------------------------------------------------------------------------
# triangle-pair blocks
# ----------------------------------------------------------------------------


class Geometry:
    """Per-triangle cubature points and half-basis data of a mesh."""

    def __init__(self, rwg: RWG):
        self.rwg = rwg
        bary, w = quad.cowper7()
        self.P = quad.points(rwg.V, rwg.F, bary)                     # [nt,7,3]
        self.W = w[None, :] * rwg.area[:, None]                      # [nt,7]
        self.k, self.s, fv = rwg.tri_bases()                         # [nt,3]
        self.vfree = rwg.V[fv]                                       # [nt,3,3]
        ell = rwg.length[self.k]                                     # [nt,3]
        self.coef = self.s * ell / (2.0 * rwg.area[:, None])         # S = coef (r - vfree)
        self.div = self.s * ell / rwg.area[:, None]                  # div S
        self.cent = rwg.V[rwg.F].mean(axis=1)
        self.mean_edge = float(np.mean(rwg.length))

    def singular_mask(self, t: np.ndarray, tp: np.ndarray) -> np.ndarray:
        F = self.rwg.F
        share = np.zeros(len(t), dtype=bool)
        for a in range(3):
            for b in range(3):
                share |= F[t, a] == F[tp, b]
        dist = np.linalg.norm(self.cent[t] - self.cent[tp], axis=1)
        return share | (dist < 2.0 * self.mean_edge)


def tri_pair_blocks(g: Geometry, t: np.ndarray, tp: np.ndarray, m: np.ndarray, p: Params,
                    kern=time_kernels, kern0=time_kernels_at0, scale=None):
    """Galerkin blocks between the three half-bases of test triangle ``t`` and
    source triangle ``tp``:  ``Z[nm, npair, 3, 3]``."""
    cA, cP = scale if scale is not None else (p.mu / (4 * np.pi), 1 / (4 * np.pi * p.eps))
    Pt, Ps = g.P[t], g.P[tp]                                         # [n,7,3]
    Wt, Ws = g.W[t], g.W[tp]
    dvec = Pt[:, :, None, :] - Ps[:, None, :, :]                     # [n,7,7,3]
    R = np.linalg.norm(dvec, axis=-1)                                # [n,7,7]
    sing = g.singular_mask(t, tp)
    fA, fP = kern(m, R, p)                                           # [nm,n,7,7]
    if np.any(sing):
        fA0, fP0, dA0, dP0 = kern0(m, p)
        fA0, fP0 = fA0[:, None, None, None], fP0[:, None, None, None]
        dA0, dP0 = dA0[:, None, None, None], dP0[:, None, None, None]
        zero = R == 0.0
        with np.errstate(divide="ignore", invalid="ignore"):
            gA = np.where(zero[None], dA0, (fA - fA0) / R[None])
            gP = np.where(zero[None], dP0, (fP - fP0) / R[None])
        s = sing[None, :, None, None]
        with np.errstate(divide="ignore", invalid="ignore"):
            hA = np.where(s, gA, fA / R[None])
            hP = np.where(s, gP, fP / R[None])
    else:
        hA, hP = fA / R[None], fP / R[None]
    WW = Wt[:, :, None] * Ws[:, None, :]                             # [n,7,7]
    # rho_a = r_a - v_p (test), rho'_b = r'_b - v_q (source)
    rt = Pt[:, None, :, :] - g.vfree[t][:, :, None, :]              # [n,3p,7,3]
    rs = Ps[:, None, :, :] - g.vfree[tp][:, :, None, :]             # [n,3q,7,3]
    dots = np.einsum("npax,nqbx->npqab", rt, rs)                     # [n,3,3,7,7]
    IA = np.einsum("mnab,nab,npqab->mnpq", hA, WW, dots)
    IP = np.einsum("mnab,nab->mn", hP, WW)
    if np.any(sing):
        idx = np.nonzero(sing)[0]
        # closed-form inner integrals at the test points of the singular pairs
        V = g.rwg.V
        F = g.rwg.F
        A, B, C = (V[F[tp[idx], i]][:, None, :] for i in range(3))
        I0, I1 = singular.potential_integrals(Pt[idx], A, B, C)     # [ns,7], [ns,7,3]
        Wi = Wt[idx]
        # int_T' (r' - v_q)/R = I1 + (r - v_q) I0
        vq = g.vfree[tp[idx]]                                        # [ns,3,3]
        inner = I1[:, None, :, :] + (Pt[idx][:, None, :, :] - vq[:, :, None, :]) * I0[:, None, :, None]
        sA = np.einsum("na,npax,nqax->npq", Wi, rt[idx], inner)      # [ns,3,3]
        sP = np.einsum("na,na->n", Wi, I0)
        IA[:, idx] += fA0.reshape(-1, 1, 1, 1) * sA[None]
        IP[:, idx] += fP0.reshape(-1, 1) * sP[None]
    ct, cs = g.coef[t], g.coef[tp]
    dt_, ds = g.div[t], g.div[tp]
    Z = cA * IA * (ct[:, :, None] * cs[:, None, :])[None] \
        + cP * IP[:, :, None, None] * (dt_[:, :, None] * ds[:, None, :])[None]
    return Z


def _assemble(g: Geometry, t, tp, blk, out, ns):
    """Scatter [nm, n, 3, 3] triangle blocks into dense [nm, ns, ns]."""
    kt, ks = g.k[t], g.k[tp]                                          # [n,3]
    rows = np.broadcast_to(kt[:, :, None], blk.shape[1:])
    cols = np.broadcast_to(ks[:, None, :], blk.shape[1:])
    flat = (rows * ns + cols).ravel()
    for mi in range(blk.shape[0]):
        np.add.at(out[mi].reshape(-1), flat, blk[mi].ravel())


def max_point_distance(g: Geometry) -> float:
    pts = g.P.reshape(-1, 3)
    best = 0.0
    for i in range(0, len(pts), 2048):
        d = np.linalg.norm(pts[i:i + 2048, None, :] - pts[None, :, :], axis=-1)
        best = max(best, float(d.max()))
    return best


def n_delays_mot(g: Geometry, p: Params) -> int:
    """N_g = floor(R_max / (c dt) + Q): last delay with a non-zero entry (Sec. 3,
    after Eq. 4, with l_max read as the upper end of the basis' support: the CPPIF order Q,
    or the BLIF half-width M), R_max over cubature points."""
    return int(math.floor(max_point_distance(g) / p.cdt + p.support))


def fill_dense(rwg: RWG, p: Params, n_delays: int | None = None, chunk: int = 4096,
               freq: bool = False):
    """Dense Z_0..Z_{N_g} (or the frequency-domain EFIE matrix if ``freq``)."""
    g = Geometry(rwg)
    ns, nt = rwg.ns, len(rwg.F)
    if freq:
        m = np.zeros(1)
        kw = dict(kern=lambda m_, R, p_: freq_kernels(R, p_),
                  kern0=lambda m_, p_: freq_kernels_at0(p_))
    else:
        if n_delays is None:
            n_delays = n_delays_mot(g, p)
        m = np.arange(n_delays + 1, dtype=np.float64)
        kw = {}
    out = np.zeros((len(m), ns, ns), dtype=complex)
    T_, TP_ = np.meshgrid(np.arange(nt), np.arange(nt), indexing="ij")
    T_, TP_ = T_.ravel(), TP_.ravel()
    for i in range(0, len(T_), chunk):
        t, tp = T_[i:i + chunk], TP_[i:i + chunk]
        _assemble(g, t, tp, tri_pair_blocks(g, t, tp, m, p, **kw), out, ns)
    return out[0] if freq else out


def fill_pairs(rwg: RWG, p: Params, pairs: np.ndarray, n_delays: int, chunk: int = 4096):
    """Entries Z_m[k, k'] for the listed RWG pairs: ``[nm, npairs]``."""
    g = Geometry(rwg)
    m = np.arange(n_delays + 1, dtype=np.float64)
    k, kp = pairs[:, 0], pairs[:, 1]
    out = np.zeros((len(m), len(pairs)), dtype=complex)
    for a in range(2):
        for b in range(2):
            t, tp = rwg.tri[k, a], rwg.tri[kp, b]
            for i in range(0, len(t), chunk):
                sl = slice(i, i + chunk)
                blk = tri_pair_blocks(g, t[sl], tp[sl], m, p)         # [nm,n,3,3]
                # locate the half-basis slots of k in t and of k' in tp
                pi = np.argmax(g.k[t[sl]] == k[sl, None], axis=1)
                qi = np.argmax(g.k[tp[sl]] == kp[sl, None], axis=1)
                n = np.arange(len(pi))
                out[:, sl] += blk[:, n, pi, qi]
    return out


# ----------------------------------------------------------------------------
# excitation (Eq. 1)
# ----------------------------------------------------------------------------


def excitation(rwg: RWG, p: Params, khat, phat, sigma: float, t_d: float, steps) -> np.ndarray:
    """V_l[k] = <S_k, p (g'(tau) + j w_c g(tau)) e^{-j w_c (r.k/c + t_d)}>,
    tau = l dt - r.k/c - t_d, g = exp(-tau^2 / (2 sigma^2)).

    Returns ``[len(steps), nb, ns]``.
    """
    g = Geometry(rwg)
    khat, phat = np.atleast_2d(khat), np.atleast_2d(phat)
    steps = np.asarray(steps, dtype=np.float64)
    out = np.zeros((len(steps), len(khat), rwg.ns), dtype=complex)
    for b in range(len(khat)):
        delay = g.P @ khat[b] / p.c                                    # [nt,7]
        tau = steps[:, None, None] * p.dt - delay[None] - t_d
        env = np.exp(-tau ** 2 / (2 * sigma ** 2))
        val = (-tau / sigma ** 2 + 1j * p.wc) * env * np.exp(-1j * p.wc * (delay + t_d))[None]
        # S_k(r).phat on each half-basis
        sp = np.einsum("tpqx,x->tpq", g.P[:, None, :, :] - g.vfree[:, :, None, :], phat[b])
        sp = sp * g.coef[:, :, None]                                   # [nt,3,7]
        contrib = np.einsum("ltq,tq,tpq->ltp", val, g.W, sp)           # [nl,nt,3]
        for pp in range(3):
            np.add.at(out[:, b, :].T, g.k[:, pp], contrib[:, :, pp].T)
    return out


def excitation_fd(rwg: RWG, p: Params, khat, phat) -> np.ndarray:
    """Frequency-domain EFIE excitation <S_k, p e^{-j k_c k.r}>: ``[nb, ns]``."""
    g = Geometry(rwg)
    khat, phat = np.atleast_2d(khat), np.atleast_2d(phat)
    out = np.zeros((len(khat), rwg.ns), dtype=complex)
    for b in range(len(khat)):
        ph = np.exp(-1j * p.kc * (g.P @ khat[b]))
        sp = np.einsum("tpqx,x->tpq", g.P[:, None, :, :] - g.vfree[:, :, None, :], phat[b]) \
            * g.coef[:, :, None]
        contrib = np.einsum("tq,tq,tpq->tp", ph, g.W, sp)
        for pp in range(3):
            np.add.at(out[b], g.k[:, pp], contrib[:, pp])
    return out


def far_field_fd(rwg: RWG, p: Params, I: np.ndarray, rhat: np.ndarray) -> np.ndarray:
    """Radiation vector of frequency-domain currents ``I[ns]`` at f_c:
    F(rhat) = (I - rhat rhat) . sum_k I_k int S_k(r') e^{+j k_c rhat.r'} dS'.
    The scattered far field is E = -j w mu/(4 pi) e^{-j k r}/r F.  Returns ``[ndir,3]``."""
    g = Geometry(rwg)
    rhat = np.atleast_2d(rhat)
    out = np.zeros((len(rhat), 3), dtype=complex)
    for d in range(len(rhat)):
        ph = np.exp(1j * p.kc * (g.P @ rhat[d]))                           # [nt,7]
        S = (g.P[:, None, :, :] - g.vfree[:, :, None, :]) * g.coef[:, :, None, None]
        Ik = I[g.k]                                                          # [nt,3]
        vec = np.einsum("tq,tq,tp,tpqx->x", ph, g.W, Ik, S)
        out[d] = vec - rhat[d] * (rhat[d] @ vec)
    return out


def rcs_fd(rwg: RWG, p: Params, I: np.ndarray, rhat: np.ndarray, pol: np.ndarray) -> np.ndarray:
    """RCS 4 pi (w mu / 4 pi)^2 |pol . F|^2 for a unit incident field."""
    F = far_field_fd(rwg, p, I, rhat)
    e = np.einsum("dx,dx->d", F, np.atleast_2d(pol))
    return 4 * np.pi * (p.wc * p.mu / (4 * np.pi)) ** 2 * np.abs(e) ** 2
