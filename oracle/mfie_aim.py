"""The AIM form of the envelope MFIE operator K_m (Sec. 4 applied to the MFIE term of the CFIE,
Sec. 2.1), evaluated plainly on the auxiliary grid of an ``aim.AimOracle``.

Test infrastructure: only the tests, the smoke check and the benchmark's CPU baseline use it.

The far part of K_m is the curl of a grid vector potential, tested with S_k:

* with g_m(R) = (DT)(m - R/(c dt)) e^{-j k_c R} / R one has
  grad g_m = -[(DT)(v)/R^2 + (D^2 T)(v)/(c R)] e^{-j k_c R} R^, so the curl term of ``mfie``
  equals -(1/4 pi) <S_k, n x curl A_m>, A_m(r) = int g_m(|r - r'|) S_k'(r') dS';
* sources: A_m is the grid convolution of g_m (G(0) = 0, as for the EFIE kernels) with the
  EFIE's anterpolated x, y, z components L_c x (stage i);
* testing: <S_k, n x curl A> = int (S_k x n) . curl A dS.  With A interpolated from the test
  RWG's 4x4x4 stencil, the weight of node n for the component A_e is
      C_x[n, k] = int (w_y d_z - w_z d_y) L_n,  C_y = int (w_z d_x - w_x d_z) L_n,
      C_z = int (w_x d_y - w_y d_x) L_n,      w = S_k x n,
  found, like L_c, by matching the moments of every monomial of degree <= 3 per axis;
* K^FFT_m = -(1/4 pi) sum_e C_e^T G^K_m L_e, and the pre-corrected near zone
  K^near_m = K_m - K^FFT_m on the near pairs (the Gram term (1/2)(DT)(m)<S_k, S_k'> lives
  there: it couples only RWGs that share a triangle).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from . import mfie, quad
from .aim import AimOracle


class MfieAim:
    def __init__(self, A: AimOracle):
        self.A = A
        self.p = A.p
        self._C = None
        self._near = None

    # ------------------------------------------------------------------ test weights
    @property
    def curl_weights(self) -> np.ndarray:
        """C [3, ns, 64]: the weights of the grid potential's x, y, z components."""
        if self._C is None:
            self._C = self._moment_matching()
        return self._C

    def _moment_matching(self, nq: int = 8) -> np.ndarray:
        A, rwg = self.A, self.A.rwg
        bary, w = quad.collapsed_gauss(nq)
        d = np.arange(4)
        lz, ly, lx = np.meshgrid(d, d, d, indexing="ij")
        alpha = np.stack([lx.ravel(), ly.ravel(), lz.ravel()], axis=1)       # [64,3]
        Vm = np.prod(alpha[None, :, :].astype(float) ** alpha[:, None, :], axis=2)
        nrm = mfie.normals(rwg)
        mom = np.zeros((3, rwg.ns, 64))
        for side, sign in ((0, 1.0), (1, -1.0)):
            t = rwg.tri[:, side]
            P = quad.points(rwg.V, rwg.F[t], bary)                           # [ns,nq,3]
            W = w[None, :] * rwg.area[t][:, None]
            vf = rwg.V[rwg.free[:, side]]
            S = sign * (rwg.length / (2 * rwg.area[t]))[:, None, None] * (P - vf[:, None, :])
            wv = np.cross(S, nrm[t][:, None, :])                              # S x n, [ns,nq,3]
            r_a = A.origin[None, :] + A.h * A.anchor
            xi = (P - r_a[:, None, :]) / A.h
            # d/dr_e of xi^alpha = (alpha_e / h) xi^(alpha - e_e)
            dmono = []
            for e in range(3):
                a2 = alpha.copy()
                a2[:, e] = np.maximum(a2[:, e] - 1, 0)
                dmono.append(alpha[None, None, :, e] / A.h * np.prod(xi[:, :, None, :] ** a2[None, None], axis=3))
            dx, dy, dz = dmono
            for c, (f1, g1, f2, g2) in enumerate(((1, dz, 2, dy), (2, dx, 0, dz), (0, dy, 1, dx))):
                integrand = wv[:, :, f1, None] * g1 - wv[:, :, f2, None] * g2     # [ns,nq,64]
                mom[c] += np.einsum("kq,kqa->ka", W, integrand)
        sol = np.linalg.solve(Vm, mom.reshape(-1, 64).T).T
        return sol.reshape(3, rwg.ns, 64)

    def curl_sparse(self, e: int) -> sp.csr_matrix:
        ns = self.A.rwg.ns
        return sp.csr_matrix((self.curl_weights[e].ravel(), (self.A.nodes.ravel(), np.repeat(np.arange(ns), 64))),
                             shape=(self.A.n ** 3, ns))

    # ------------------------------------------------------------------ kernel and far part
    def kernel_values(self, m: int, dijk: np.ndarray) -> np.ndarray:
        """G^K_m at integer offsets: (DT)(m - R/(c dt)) e^{-j k R} / R, G(0) = 0."""
        p, h = self.p, self.A.h
        d = dijk.astype(np.float64)
        R = h * np.sqrt(d[..., 0] ** 2 + d[..., 1] ** 2 + d[..., 2] ** 2)
        v = m - R / p.cdt
        f = p.T(v, 1, m) / p.dt + 1j * p.wc * p.T(v, 0, m)
        with np.errstate(divide="ignore", invalid="ignore"):
            return np.where(R > 0, f * np.exp(-1j * p.kc * R) / R, 0.0)

    def fft_dense(self, m: int) -> np.ndarray:
        """Dense K^FFT_m = -(1/4 pi) sum_e C_e^T G^K_m L_e on the active nodes."""
        A = self.A
        act = A.active
        ijk = A.node_ijk(act)
        G = self.kernel_values(m, ijk[:, None, :] - ijk[None, :, :])
        out = 0
        for e in range(3):
            C = self.curl_sparse(e)[act].toarray()
            L = A.lam_sparse(e)[act].toarray()
            out = out + C.T @ G @ L
        return -out / (4 * math.pi)

    # ------------------------------------------------------------------ near zone and operator
    def exact(self, n_delays: int | None = None) -> np.ndarray:
        """The direct K_0..K_{N_g} of ``mfie.fill_dense`` (N_g of the grid by default)."""
        nd = self.A.n_delays if n_delays is None else n_delays
        return mfie.fill_dense(self.A.rwg, self.p, n_delays=nd)

    def dense(self, m: int, K_exact: np.ndarray) -> np.ndarray:
        """K^AIM_m = K^FFT_m + (K_m - K^FFT_m) on the near pairs (``K_exact`` from ``exact``)."""
        F = self.fft_dense(m)
        pr = self.A.pairs
        out = F.copy()
        out[pr[:, 0], pr[:, 1]] = K_exact[m][pr[:, 0], pr[:, 1]]
        return out
