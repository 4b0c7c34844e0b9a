"""Write the oracle's ET-AIM products on sampled rows for the 491 520-RWG sphere array.

Fixture for the GPU test of the largest workload and for the benchmark's stated error.
Calls only ``oracle/`` (and the seeded input generators); nothing comes from the CUDA
library.  For a seeded current vector x (PCG64(11), standard normal real and imaginary
parts) and seeded rows (PCG64(12)), the rows of Z~AIM_m x (Eq. 5) for m = 0 and 1:
the grid part by direct sums over the grid (no FFT), the near part from the oracle's
Galerkin entries minus their grid approximation for the pairs of those rows.

Workload array491k: 4 x 4 icosphere-5 spheres (r = 0.5 m, 1.5 m pitch), 1 GHz +-5 %,
384^3 grid, near radius 3 grid steps.

Output: ``array491k_matvec_rows.txt``, one line per (delay, row): ``m row re im``.

    python tests/golden/make_array491k_rows.py      # tens of minutes on one core
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import aim as oaim  # noqa: E402
from oracle import efie  # noqa: E402
from oracle.rwg import build_rwg  # noqa: E402
from paper_1408_7060_gb300.inputs import make_workload, seeded_rows, seeded_vector  # noqa: E402

OUT = os.path.join(HERE, "array491k_matvec_rows.txt")
N_ROWS = 4
DELAYS = (0, 1)


def main():
    w = make_workload("array491k")
    rwg = build_rwg(*w.mesh)
    p = efie.Params(dt=w.dt, f_c=w.f_c, Q=w.order)
    t0 = time.time()
    A = oaim.AimOracle(rwg, w.grid_n, w.h, w.origin, w.near_radius, p)
    print(f"setup {time.time() - t0:.0f} s, N_g = {A.n_delays}, {len(A.pairs)} near pairs", flush=True)
    x = seeded_vector(rwg.ns, 11)
    rows = seeded_rows(rwg.ns, N_ROWS, 12)
    pr = A.pairs[np.isin(A.pairs[:, 0], rows)]
    Zd = efie.fill_pairs(rwg, p, pr, max(DELAYS))
    lines = [f"# m row re im  (oracle rows of Z~AIM_m x, direct grid sums; N_g = {A.n_delays})"]
    for m in DELAYS:
        t0 = time.time()
        y = A.fft_part_rows(m, x, rows)
        Zn = Zd[m] - A.fft_pairs(m, pr)
        for (k, kp), z in zip(pr, Zn):
            y[np.searchsorted(rows, k)] += z * x[kp]
        print(f"m = {m}: {time.time() - t0:.0f} s", flush=True)
        for r, v in zip(rows, y):
            lines.append(f"{m} {r} {v.real:.17e} {v.imag:.17e}")
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main()
