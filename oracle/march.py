"""Time marching of the envelope systems: Eq. 4 (ET-MOT) and Eq. 5 (ET-AIM).

For l = 1..N_t:  Z_0 I_l = V_l - sum_{m=1..min(N_g, l-1)} Z_m I_{l-m},  with I_l = 0 for
l <= 0 (the march starts from rest).  The immediate system is solved exactly by an
LU factorisation (scipy) or, for operators given only as products, by GMRES.
Arrays are indexed by step l - 1.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla


def march_dense(Z: np.ndarray, V: np.ndarray) -> np.ndarray:
    """Z[N_g+1, ns, ns], V[N_t, nb, ns] -> I[N_t, nb, ns]."""
    nt, nb, ns = V.shape
    ng = Z.shape[0] - 1
    lu = sla.lu_factor(Z[0])
    I = np.zeros_like(V)
    for l in range(1, nt + 1):
        rhs = V[l - 1].T.copy()                                   # [ns, nb]
        for m in range(1, min(ng, l - 1) + 1):
            rhs -= Z[m] @ I[l - 1 - m].T
        I[l - 1] = sla.lu_solve(lu, rhs).T
    return I


def rhs_operator(matvec, ng: int, hist: np.ndarray, l: int) -> np.ndarray:
    """sum_{m=1..min(N_g, l-1)} Z_m I_{l-m} for one RHS: hist[N_t, ns] (step-indexed)."""
    out = 0
    for m in range(1, min(ng, l - 1) + 1):
        out = out + matvec(m, hist[l - 1 - m])
    return out


def march_operator(matvec, ng: int, V: np.ndarray, tol: float = 1e-10, maxiter: int = 2000, precond=None):
    """The same march with Z_m given as ``matvec(m, x)`` and GMRES for Z_0 (warm start:
    the previous step's currents).  ``precond`` (optional) is a linear operator
    approximating Z_0^{-1}, passed to scipy's GMRES; whatever it is, each step repeats
    GMRES from its last iterate until the true relative residual ||b - Z_0 x|| / ||b||
    is at most ``tol``.

    Returns ``(I, iterations[N_t, nb])``."""
    nt, nb, ns = V.shape
    I = np.zeros_like(V)
    its = np.zeros((nt, nb), dtype=np.int64)
    A = spla.LinearOperator((ns, ns), matvec=lambda x: matvec(0, x), dtype=complex)
    for b in range(nb):
        for l in range(1, nt + 1):
            rhs = V[l - 1, b] - rhs_operator(matvec, ng, I[:, b], l)
            cnt = [0]

            def cb(_):
                cnt[0] += 1
            x = I[l - 2, b].copy() if l > 1 else np.zeros(ns, dtype=complex)
            for _ in range(20):
                x, info = spla.gmres(A, rhs, x0=x, rtol=tol, atol=0.0, restart=50, maxiter=maxiter,
                                     callback=cb, callback_type="pr_norm", M=precond)
                if np.linalg.norm(rhs - A.matvec(x)) <= tol * np.linalg.norm(rhs):
                    break
            I[l - 1, b] = x
            its[l - 1, b] = cnt[0]
    return I, its
