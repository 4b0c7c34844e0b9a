"""Write the oracle's marched currents of the 7680-RWG sphere workloads on sampled rows.

Fixture for tests/test_gpu_march_oracle.py.  Calls only ``oracle/`` (and the seeded
input generators); nothing comes from the CUDA library.  The march is Eq. 5 solved step
by step with the oracle's ET-AIM operator (FFT grid convolution, pinned to direct grid
sums) and GMRES to a true relative residual of 1e-10 (preconditioned by the oracle's
near-zone sparse approximate inverse, which changes only the path of the solve).

Workloads (seeded, synthetic):
* sphere7680: icosphere subdivision 4 (7680 RWG), 600 MHz +-30 %, 64^3 grid, one
  +z-incident x-polarised wave; steps 1..24 (the pulse peaks near step 15);
* sphere7680_b64: the same mesh, 600 MHz +-10 %, the first two of the 64 seeded waves;
  steps 1..24.

Output: ``sphere7680_march_rows.txt`` with one line per (workload, wave, step, row):
``workload wave step row re im``.  48 rows per workload, drawn with PCG64(7).

    python tests/golden/make_sphere7680_marches.py      # about an hour on 8 cores
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import aim as oaim  # noqa: E402
from oracle import efie, march, precond  # noqa: E402
from oracle.rwg import build_rwg  # noqa: E402
from paper_1408_7060_gb300.inputs import make_workload, seeded_rows  # noqa: E402

OUT = os.path.join(HERE, "sphere7680_march_rows.txt")
N_STEPS = 24
N_ROWS = 48
CASES = (("sphere7680", (0,)), ("sphere7680_b64", (0, 1)))


def march_rows(name: str, waves) -> tuple[np.ndarray, np.ndarray]:
    w = make_workload(name)
    rwg = build_rwg(*w.mesh)
    p = efie.Params(dt=w.dt, f_c=w.f_c, Q=w.order)
    t0 = time.time()
    A = oaim.AimOracle(rwg, w.grid_n, w.h, w.origin, w.near_radius, p)
    A.near_values()
    z0 = efie.fill_pairs(rwg, p, A.pairs, 0)[0]
    M = precond.near_sai(rwg.ns, A.pairs, z0)
    Msp = sp.csr_matrix((M, (A.pairs[:, 0], A.pairs[:, 1])), shape=(rwg.ns, rwg.ns))
    P = spla.LinearOperator((rwg.ns, rwg.ns), matvec=lambda x: Msp @ x, dtype=complex)
    print(f"{name}: setup {time.time() - t0:.0f} s, N_g = {A.n_delays}", flush=True)
    k, ph = w.khat[list(waves)], w.phat[list(waves)]
    V = efie.excitation(rwg, p, k, ph, w.sigma, w.t_d, np.arange(1, N_STEPS + 1))
    t0 = time.time()
    I, its = march.march_operator(A.matvec, A.n_delays, V, tol=1e-10, precond=P)
    print(f"{name}: march {time.time() - t0:.0f} s, GMRES iterations per step {its.mean():.1f}", flush=True)
    rows = seeded_rows(rwg.ns, N_ROWS, 7)
    return rows, I[:, :, rows]


def main():
    lines = ["# workload wave step row re im  (oracle ET-AIM march, GMRES true residual <= 1e-10)"]
    for name, waves in CASES:
        rows, I = march_rows(name, waves)
        for bi, wv in enumerate(waves):
            for l in range(N_STEPS):
                for r, v in zip(rows, I[l, bi]):
                    lines.append(f"{name} {wv} {l + 1} {r} {v.real:.17e} {v.imag:.17e}")
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main()
