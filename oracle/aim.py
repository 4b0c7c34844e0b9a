"""The ET-AIM operator of Eq. 5 (Sec. 4, stages i-iv), evaluated plainly.

Z^AIM_m = Z^FFT_m + Z^near_m with

  Z^FFT_m = mu/(4 pi) sum_{c in x,y,z} L_c^T G^A_m L_c + 1/(4 pi eps) L_div^T G^phi_m L_div

* anterpolation L_c (stage i): one 4x4x4 stencil per RWG anchored at
  floor((x_e - x0)/h) - 1 per axis, clamped to [0, N-4], x_e the midpoint of the
  RWG's edge; coefficients from moment matching up to order 3 per axis (Sec. 5.1:
  "moments up to order 3"), i.e. the 64 x 64 Vandermonde system
  sum_n L_c[n,k] xi_n^a = int S_k^c xi^a dS, 0 <= a_x, a_y, a_z <= 3, xi = (r - r_anchor)/h;
  c = div uses the scalar div S_k;
* propagation (stage ii): G^A_m(D) = (D^2 T)(m - R/(c dt)) e^{-j k R}/R and
  G^phi_m(D) = T(m - R/(c dt)) e^{-j k R}/R for the integer node offset D,
  R = h |D|, and G(0) = 0; a non-periodic (linear) convolution over the grid;
* interpolation (stage iii) is the transpose L_c^T;
* near-zone pre-correction (stage iv): for RWG pairs whose edge midpoints are at
  most ``near_radius`` apart, Z^near_m = Z_m - Z^FFT_m; zero otherwise.

The convolution is given twice: by its definition (a direct sum over node pairs)
and through a zero-padded numpy FFT, which the tests pin to the direct sum.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from . import efie, quad
from .constants import EPS0, MU0
from .rwg import RWG

CA = MU0 / (4 * math.pi)          # vacuum values of the two kernel constants
CP = 1.0 / (4 * math.pi * EPS0)


class AimOracle:
    def __init__(self, rwg: RWG, n: int, h: float, origin, near_radius: float, p: efie.Params):
        self.rwg, self.n, self.h, self.p = rwg, int(n), float(h), p
        self.ca, self.cp = p.mu / (4 * math.pi), 1.0 / (4 * math.pi * p.eps)  # mu/4pi, 1/(4 pi eps)
        self.origin = np.asarray(origin, dtype=np.float64)
        self.near_radius = float(near_radius)
        self.anchor = self._anchors()
        self.nodes = self._stencil_nodes()                    # [ns,64] linear node index
        act = np.unique(self.nodes)
        self.active = act
        self._lam = None                                       # computed on first use
        self._n_delays = None
        self._pairs = None
        self._near_vals = None

    @property
    def lam(self) -> np.ndarray:
        """Anterpolation coefficients [4, ns, 64]."""
        if self._lam is None:
            self._lam = self._moment_matching()
        return self._lam

    @property
    def n_delays(self) -> int:
        if self._n_delays is None:
            self._n_delays = self._n_delays_grid()
        return self._n_delays

    @property
    def pairs(self) -> np.ndarray:
        if self._pairs is None:
            self._pairs = self._near_pairs()
        return self._pairs

    # ------------------------------------------------------------------ stencils
    def _anchors(self):
        xe = self.rwg.midpoint()
        a = np.floor((xe - self.origin[None, :]) / self.h).astype(np.int64) - 1
        return np.clip(a, 0, self.n - 4)

    def node_ijk(self, lin):
        n = self.n
        return np.stack([lin % n, (lin // n) % n, lin // (n * n)], axis=-1)

    def _stencil_nodes(self):
        n = self.n
        d = np.arange(4)
        lz, ly, lx = np.meshgrid(d, d, d, indexing="ij")        # node order: x fastest
        off = np.stack([lx.ravel(), ly.ravel(), lz.ravel()], axis=1)   # [64,3]
        ijk = self.anchor[:, None, :] + off[None]
        return (ijk[..., 2] * n + ijk[..., 1]) * n + ijk[..., 0]

    def _moment_matching(self, nq: int = 8, chunk: int = 8192):
        rwg = self.rwg
        bary, w = quad.collapsed_gauss(nq)
        d = np.arange(4)
        lz, ly, lx = np.meshgrid(d, d, d, indexing="ij")
        alpha = np.stack([lx.ravel(), ly.ravel(), lz.ravel()], axis=1)  # [64,3] exponents
        # Vandermonde V[a, n] = prod xi_n^a with xi_n in {0..3}^3 (same ordering)
        Vm = np.prod(alpha[None, :, :].astype(float) ** alpha[:, None, :], axis=2)  # [a, n]
        lam = np.zeros((4, rwg.ns, 64))
        for k0 in range(0, rwg.ns, chunk):
            ks = slice(k0, min(rwg.ns, k0 + chunk))
            for side, sign in ((0, 1.0), (1, -1.0)):
                t = rwg.tri[ks, side]
                P = quad.points(rwg.V, rwg.F[t], bary)                  # [nk,nq,3]
                W = w[None, :] * rwg.area[t][:, None]
                vf = rwg.V[rwg.free[ks, side]]
                S = sign * (rwg.length[ks] / (2 * rwg.area[t]))[:, None, None] * (P - vf[:, None, :])
                div = sign * rwg.length[ks] / rwg.area[t]
                r_a = self.origin[None, :] + self.h * self.anchor[ks]     # [nk,3]
                xi = (P - r_a[:, None, :]) / self.h                       # [nk,nq,3]
                mono = np.prod(xi[:, :, None, :] ** alpha[None, None], axis=3)  # [nk,nq,64]
                for c in range(3):
                    lam[c, ks] += np.einsum("kq,kq,kqa->ka", W, S[..., c], mono)
                lam[3, ks] += np.einsum("kq,k,kqa->ka", W, div, mono)
        # solve V lam = moments per RWG and component
        sol = np.linalg.solve(Vm, lam.reshape(-1, 64).T).T
        return sol.reshape(4, rwg.ns, 64)

    def lam_sparse(self, c: int) -> sp.csr_matrix:
        """L_c as an [N^3, ns] sparse matrix."""
        ns = self.rwg.ns
        rows = self.nodes.ravel()
        cols = np.repeat(np.arange(ns), 64)
        return sp.csr_matrix((self.lam[c].ravel(), (rows, cols)), shape=(self.n ** 3, ns))

    # ------------------------------------------------------------------ kernels
    def _n_delays_grid(self, hull_above: int = 20000):
        """N_g = floor(R_max/(c dt) + Q), R_max the largest distance between two
        stencil nodes (a reading of the N_g formula after Eq. 4).  The farthest pair
        of a point set lies on its convex hull, so large sets are first reduced to the
        hull's vertices (scipy); squared integer distances are exact in FP64."""
        ijk = self.node_ijk(self.active).astype(np.float64)
        if len(ijk) > hull_above:
            from scipy.spatial import ConvexHull

            try:
                ijk = ijk[ConvexHull(ijk).vertices]
            except Exception:
                pass
        sq = (ijk * ijk).sum(1)
        best = 0.0
        for i in range(0, len(ijk), 4096):
            d2 = sq[i:i + 4096, None] + sq[None, :] - 2.0 * (ijk[i:i + 4096] @ ijk.T)
            best = max(best, float(d2.max()))
        rmax = self.h * math.sqrt(int(round(best)))
        return int(math.floor(rmax / self.p.cdt + self.p.support))

    def kernel_values(self, m: int, dijk: np.ndarray):
        """(G^A_m, G^phi_m) at integer offsets ``dijk[...,3]`` (G(0) = 0)."""
        d = dijk.astype(np.float64)
        R = self.h * np.sqrt(d[..., 0] ** 2 + d[..., 1] ** 2 + d[..., 2] ** 2)
        v = m - R / self.p.cdt
        ph = np.exp(-1j * self.p.kc * R)
        p = self.p
        D2T = p.T(v, 2, m) / p.dt ** 2 + 2j * p.wc * p.T(v, 1, m) / p.dt - p.wc ** 2 * p.T(v, 0, m)
        with np.errstate(divide="ignore", invalid="ignore"):
            GA = np.where(R > 0, D2T * ph / R, 0.0)
            GP = np.where(R > 0, p.T(v, 0, m) * ph / R, 0.0)
        return GA, GP

    # ------------------------------------------------------------------ grid sums
    def conv_direct(self, m: int, src: np.ndarray, kind: int, targets=None, chunk: int = 2048):
        """P[n] = sum_{n'} G_m(n - n') src[n'] over source nodes where src != 0.
        ``src`` is [N^3]; ``kind`` 0 = G^A, 1 = G^phi.  Returns P at ``targets``
        (default: every node).  G depends on |D_x|, |D_y|, |D_z| only; large grids
        look it up in a table of those offsets."""
        srcn = np.nonzero(src)[0]
        sv = src[srcn]
        sijk = self.node_ijk(srcn)
        tgt = np.arange(self.n ** 3) if targets is None else np.asarray(targets)
        tijk = self.node_ijk(tgt)
        out = np.zeros(len(tgt), dtype=complex)
        tab = self._kernel_table(m, kind) if self.n > 64 else None
        schunk = max(1, (1 << 24) // max(1, min(chunk, len(tgt))))
        for i in range(0, len(tgt), chunk):
            for j in range(0, len(srcn), schunk):
                d = tijk[i:i + chunk, None, :] - sijk[None, j:j + schunk, :]
                if tab is None:
                    G = self.kernel_values(m, d)[kind]
                else:
                    d = np.abs(d)
                    G = tab[d[..., 2], d[..., 1], d[..., 0]]
                out[i:i + chunk] += G @ sv[j:j + schunk]
        return out

    def _kernel_table(self, m: int, kind: int) -> np.ndarray:
        key = (m, kind)
        if not hasattr(self, "_tabs"):
            self._tabs = {}
        if key not in self._tabs:
            r = np.arange(self.n)
            tab = np.empty((self.n, self.n, self.n), dtype=complex)
            for z in range(self.n):
                ty, tx = np.meshgrid(r, r, indexing="ij")
                off = np.stack([tx, ty, np.full_like(tx, z)], axis=-1)
                tab[z] = self.kernel_values(m, off)[kind]
            self._tabs[key] = tab
        return self._tabs[key]

    def kernel_grid(self, m: int, kind: int) -> np.ndarray:
        """G_m embedded even-symmetrically in the (2N)^3 padded grid (index N unused)."""
        n2 = 2 * self.n
        i = np.arange(n2)
        off = np.where(i < self.n, i, i - n2)
        off[self.n] = 0
        dz, dy, dx = np.meshgrid(off, off, off, indexing="ij")
        G = self.kernel_values(m, np.stack([dx, dy, dz], axis=-1))[kind]
        G[self.n, :, :] = 0
        G[:, self.n, :] = 0
        G[:, :, self.n] = 0
        return G

    def kernel_fft(self, m: int, kind: int) -> np.ndarray:
        """numpy FFT of ``kernel_grid(m, kind)``, kept after the first request."""
        if not hasattr(self, "_kfft"):
            self._kfft = {}
        if (m, kind) not in self._kfft:
            self._kfft[(m, kind)] = np.fft.fftn(self.kernel_grid(m, kind))
        return self._kfft[(m, kind)]

    def conv_fft(self, m: int, src: np.ndarray, kind: int) -> np.ndarray:
        """The same linear convolution through a zero-padded FFT of size (2N)^3."""
        n, n2 = self.n, 2 * self.n
        a = np.zeros((n2, n2, n2), dtype=complex)
        a[:n, :n, :n] = src.reshape(n, n, n)
        out = np.fft.ifftn(np.fft.fftn(a) * self.kernel_fft(m, kind))
        return out[:n, :n, :n].ravel()

    # ------------------------------------------------------------------ operators
    def anterpolate(self, x: np.ndarray) -> np.ndarray:
        """Source grids [4, N^3] for one current vector x[ns]."""
        return np.stack([self.lam_sparse(c) @ x for c in range(4)])

    def interpolate(self, P: np.ndarray) -> np.ndarray:
        """y[k] = mu/4pi sum_{c=x,y,z} L_c^T P_c + 1/(4 pi eps) L_div^T P_div."""
        y = self.ca * sum(self.lam_sparse(c).T @ P[c] for c in range(3))
        return y + self.cp * (self.lam_sparse(3).T @ P[3])

    def fft_part(self, m: int, x: np.ndarray, method: str = "fft") -> np.ndarray:
        S = self.anterpolate(x)
        if method == "fft":
            P = np.stack([self.conv_fft(m, S[c], 0 if c < 3 else 1) for c in range(4)])
        else:
            P = np.stack([self.conv_direct(m, S[c], 0 if c < 3 else 1) for c in range(4)])
        return self.interpolate(P)

    def fft_part_rows(self, m: int, x: np.ndarray, rows) -> np.ndarray:
        """Selected output rows of Z^FFT_m x by direct sums (for large grids)."""
        rows = np.asarray(rows)
        S = self.anterpolate(x)
        y = np.zeros(len(rows), dtype=complex)
        for i, k in enumerate(rows):
            tg = self.nodes[k]
            for c in range(4):
                P = self.conv_direct(m, S[c], 0 if c < 3 else 1, targets=tg)
                y[i] += (self.ca if c < 3 else self.cp) * (self.lam[c, k] @ P)
        return y

    def fft_dense(self, m: int) -> np.ndarray:
        """Dense Z^FFT_m (small problems): L^T G L restricted to active nodes."""
        act = self.active
        ijk = self.node_ijk(act)
        GA, GP = self.kernel_values(m, ijk[:, None, :] - ijk[None, :, :])
        out = 0
        for c in range(4):
            L = self.lam_sparse(c)[act].toarray()                 # [nact, ns]
            out = out + (self.ca * (L.T @ GA @ L) if c < 3 else self.cp * (L.T @ GP @ L))
        return out

    def fft_pairs(self, m: int, pairs: np.ndarray) -> np.ndarray:
        """Z^FFT_m[k,k'] for listed pairs (64 x 64 node sums per component).

        G_m depends on |D_x|, |D_y|, |D_z| only, so it is tabulated once over the
        offsets that occur and looked up."""
        k, kp = pairs[:, 0], pairs[:, 1]
        ia, ib = self.node_ijk(self.nodes[k]), self.node_ijk(self.nodes[kp])
        dmax = int(np.abs(self.anchor[k] - self.anchor[kp]).max()) + 4 if len(pairs) else 4
        r = np.arange(dmax + 1)
        tz, ty, tx = np.meshgrid(r, r, r, indexing="ij")
        TA, TP = self.kernel_values(m, np.stack([tx, ty, tz], axis=-1))
        out = np.zeros(len(pairs), dtype=complex)
        for i in range(0, len(pairs), 512):
            sl = slice(i, i + 512)
            d = np.abs(ia[sl, :, None, :] - ib[sl, None, :, :])
            GA, GP = TA[d[..., 2], d[..., 1], d[..., 0]], TP[d[..., 2], d[..., 1], d[..., 0]]
            for c in range(4):
                G = GA if c < 3 else GP
                val = np.einsum("pa,pab,pb->p", self.lam[c, k[sl]], G, self.lam[c, kp[sl]])
                out[sl] += (self.ca if c < 3 else self.cp) * val
        return out

    # ------------------------------------------------------------------ near zone
    def _near_pairs(self, tree_above: int = 20000):
        """Pairs with |x_e(k) - x_e(k')|^2 <= r^2 (inclusive), sorted by (k, k').
        Large meshes take candidates from a k-d tree with a slightly larger radius; the
        decision is always the same squared-distance comparison."""
        xe = self.rwg.midpoint()
        if self.near_radius < 0:
            return np.zeros((0, 2), dtype=np.int64)
        r2 = self.near_radius * self.near_radius
        if len(xe) > tree_above:
            from scipy.spatial import cKDTree

            cand = cKDTree(xe).query_pairs(self.near_radius * (1 + 1e-6) + 1e-12, output_type="ndarray")
            cand = np.concatenate([cand, cand[:, ::-1], np.stack([np.arange(len(xe))] * 2, axis=1)])
            d = xe[cand[:, 0]] - xe[cand[:, 1]]
            d2 = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2]
            pr = cand[d2 <= r2].astype(np.int64)
        else:
            out = []
            for i in range(0, len(xe), 1024):
                d = xe[i:i + 1024, None, :] - xe[None, :, :]
                d2 = d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1] + d[..., 2] * d[..., 2]
                a, b = np.nonzero(d2 <= r2)
                out.append(np.stack([a + i, b], axis=1))
            pr = np.concatenate(out) if out else np.zeros((0, 2), dtype=np.int64)
        order = np.lexsort((pr[:, 1], pr[:, 0]))
        return pr[order]

    def near_values(self, n_delays: int | None = None) -> np.ndarray:
        """Z^near_m on the near pairs, ``[N_g + 1, npairs]``."""
        nd = self.n_delays if n_delays is None else n_delays
        if self._near_vals is None or self._near_vals.shape[0] != nd + 1:
            Z = efie.fill_pairs(self.rwg, self.p, self.pairs, nd)
            F = np.stack([self.fft_pairs(m, self.pairs) for m in range(nd + 1)])
            self._near_vals = Z - F
        return self._near_vals

    def near_matrix(self, m: int) -> sp.csr_matrix:
        ns = self.rwg.ns
        v = self.near_values()[m]
        return sp.csr_matrix((v, (self.pairs[:, 0], self.pairs[:, 1])), shape=(ns, ns))

    def matvec(self, m: int, x: np.ndarray, method: str = "fft") -> np.ndarray:
        """Z^AIM_m x (Eq. 5)."""
        return self.fft_part(m, x, method) + self.near_matrix(m) @ x

    def dense(self, m: int) -> np.ndarray:
        return self.fft_dense(m) + self.near_matrix(m).toarray()
