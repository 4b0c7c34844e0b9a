"""Near-zone sparse approximate inverse (SAI) of the immediate matrix -- test
infrastructure (the oracle for the library's optional right preconditioner).

Not in the paper: Sec. 5.1 preconditions the immediate system with its diagonal.  The
library can instead use a right preconditioner M with the sparsity of the near zone
(Sec. 4, stage iv: the pairs whose edge midpoints are within the near radius).  Its
definition (a Frobenius-norm minimising approximate inverse on a fixed pattern),
restated plainly:

* S_k = the pattern set of RWG k: the RWGs whose edge midpoints are within the pattern
  radius of k's (by default the near radius; ascending indices; k is in it);
* Zn[i, j] = Z_0[i, j] (the Galerkin entry of the immediate matrix, Eq. 4 with m = 0)
  when (i, j) is a pattern pair, 0 otherwise;
* column k of M is supported on S_k and minimises || Zn[:, S_k] m_k - e_k ||_2 over all
  rows (only the rows R_k that meet a near set of S_k are non-zero);
* M[s, k] = m_k[s]; the pattern is symmetric, so M lives on its CSR form (row s,
  column k).

Special cases that pin it: a near zone of self pairs only gives M = diag(1 / Z_0[k, k])
(the paper's diagonal preconditioner); a near zone covering every pair gives M = Z_0^{-1};
every column satisfies the normal equations Zn[:, S_k]^H (Zn[:, S_k] m_k - e_k) = 0.
"""
from __future__ import annotations

import numpy as np


def near_sai(ns: int, pairs: np.ndarray, z0: np.ndarray) -> np.ndarray:
    """M on the near pairs.

    pairs: [npairs, 2] (row, col) sorted by (row, col), symmetric, including (k, k);
    z0: Z_0 on those pairs.  Returns values v with v[e] = M[pairs[e, 0], pairs[e, 1]].
    One dense least-squares problem per column (numpy.linalg.lstsq)."""
    pairs = np.asarray(pairs, dtype=np.int64)
    z0 = np.asarray(z0, dtype=np.complex128)
    where = {(int(r), int(c)): e for e, (r, c) in enumerate(pairs)}
    start = np.searchsorted(pairs[:, 0], np.arange(ns + 1))
    out = np.zeros(len(pairs), dtype=np.complex128)
    for k in range(ns):
        S = pairs[start[k]:start[k + 1], 1]
        R = np.unique(np.concatenate([pairs[start[s]:start[s + 1], 1] for s in S]))  # near sets of S
        A = np.zeros((len(R), len(S)), dtype=np.complex128)
        for i, r in enumerate(R):
            for j, s in enumerate(S):
                e = where.get((int(r), int(s)))
                if e is not None:
                    A[i, j] = z0[e]
        rhs = (R == k).astype(np.complex128)
        m = np.linalg.lstsq(A, rhs, rcond=None)[0]
        for i, si in enumerate(S):
            out[where[(int(si), k)]] = m[i]
    return out
