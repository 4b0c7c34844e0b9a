"""Near-zone sparse approximate inverse (SAI) of the immediate matrix -- test
infrastructure (the oracle for the library's optional right preconditioner).

Not in the paper: Sec. 5.1 preconditions the immediate system with its diagonal.  The
library can instead use a right preconditioner M with the sparsity of the near zone
(Sec. 4, stage iv: the pairs whose edge midpoints are within the near radius).  Its
definition, restated plainly:

* S_k = the near set of RWG k (ascending indices; k is in it);
* Zn[i, j] = Z_0[i, j] (the Galerkin entry of the immediate matrix, Eq. 4 with m = 0)
  when (i, j) is a near pair, 0 otherwise;
* column k of M is supported on S_k and solves  Zn[S_k, S_k] m_k = e_k  (e_k the unit
  vector of k within S_k), i.e. m_k is column k of the inverse of the near block
  around k;
* M[s, k] = m_k[s]; the near pattern is symmetric, so M lives on the near CSR pattern
  (row s, column k).

Special cases that pin it: a near zone of self pairs only gives M = diag(1 / Z_0[k, k])
(the paper's diagonal preconditioner); a near zone covering every pair gives M = Z_0^{-1}.
"""
from __future__ import annotations

import numpy as np


def near_sai(ns: int, pairs: np.ndarray, z0: np.ndarray) -> np.ndarray:
    """M on the near pairs.

    pairs: [npairs, 2] (row, col) sorted by (row, col), symmetric, including (k, k);
    z0: Z_0 on those pairs.  Returns values v with v[e] = M[pairs[e, 0], pairs[e, 1]].
    One dense solve per column (numpy.linalg.solve)."""
    pairs = np.asarray(pairs, dtype=np.int64)
    z0 = np.asarray(z0, dtype=np.complex128)
    where = {(int(r), int(c)): e for e, (r, c) in enumerate(pairs)}
    start = np.searchsorted(pairs[:, 0], np.arange(ns + 1))
    out = np.zeros(len(pairs), dtype=np.complex128)
    for k in range(ns):
        S = pairs[start[k]:start[k + 1], 1]
        n = len(S)
        A = np.zeros((n, n), dtype=np.complex128)
        for i, si in enumerate(S):
            for j, sj in enumerate(S):
                e = where.get((int(si), int(sj)))
                if e is not None:
                    A[i, j] = z0[e]
        rhs = (S == k).astype(np.complex128)
        m = np.linalg.solve(A, rhs)
        for i, si in enumerate(S):
            out[where[(int(si), k)]] = m[i]
    return out
