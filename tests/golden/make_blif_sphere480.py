"""Write the oracle's ET-AIM products and march of the 480-RWG sphere with the BLIF basis.

Fixture for tests/test_gpu_blif.py.  Calls only ``oracle/`` (and the seeded input
generators); nothing comes from the CUDA library.

Workload (seeded, synthetic): the 480-RWG sphere of radius 1 m, 150 MHz +-20 % (chi = 6),
16^3 grid, 0.3 m near zone, one +z-incident x-polarised wave; BLIF half-width M = 3 with
the band fraction beta = f_bw dt = 1/4 (Sec. 3.1.2) and its causal extrapolation.

Output: ``blif_sphere480.txt``:
* ``ng N_g``;
* ``prod m row re im``: (Z~_m x)[row] for every delay m, x the complex vector drawn with
  numpy's default_rng(41) (standard normal real and imaginary parts, in that order), on 96
  rows drawn with PCG64(8);
* ``march step row re im``: the currents of Eq. 5 solved by dense LU on the oracle's AIM
  matrices, steps 1..50, on 32 rows drawn with PCG64(9);
* ``mot step row re im``: the direct ET-MOT currents of Eq. 4 (the oracle's Galerkin fill of
  the same envelope EFIE with the same time factors, dense LU), same steps and rows.

    python tests/golden/make_blif_sphere480.py      # a few minutes on one core
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import aim as oaim  # noqa: E402
from oracle import efie, march  # noqa: E402
from oracle.rwg import build_rwg  # noqa: E402
from paper_1408_7060_gb300.inputs import make_workload, seeded_rows  # noqa: E402

OUT = os.path.join(HERE, "blif_sphere480.txt")


def workload():
    return make_workload("sphere480", band_frac=0.2, n_t=50, basis="blif", order=3)


def main():
    w = workload()
    rwg = build_rwg(*w.mesh)
    p = efie.Params(dt=w.dt, f_c=w.f_c, basis="blif", M=w.order, beta=w.beta)
    A = oaim.AimOracle(rwg, w.grid_n, w.h, w.origin, w.near_radius, p)
    ZA = np.stack([A.dense(m) for m in range(A.n_delays + 1)])
    rng = np.random.default_rng(41)
    x = rng.standard_normal(rwg.ns) + 1j * rng.standard_normal(rwg.ns)
    V = efie.excitation(rwg, p, w.khat, w.phat, w.sigma, w.t_d, np.arange(1, w.n_t + 1))
    I = march.march_dense(ZA, V)[:, 0]
    J = march.march_dense(efie.fill_dense(rwg, p), V)[:, 0]
    prow, mrow = seeded_rows(rwg.ns, 96, 8), seeded_rows(rwg.ns, 32, 9)
    lines = ["# blif sphere480: ng N_g | prod m row re im | march / mot step row re im (oracle ET-AIM / "
             "direct ET-MOT, dense LU)",
             f"ng {A.n_delays}"]
    for m in range(A.n_delays + 1):
        y = ZA[m] @ x
        lines += [f"prod {m} {r} {y[r].real:.17e} {y[r].imag:.17e}" for r in prow]
    for l in range(w.n_t):
        lines += [f"march {l + 1} {r} {I[l, r].real:.17e} {I[l, r].imag:.17e}" for r in mrow]
    for l in range(w.n_t):
        lines += [f"mot {l + 1} {r} {J[l, r].real:.17e} {J[l, r].imag:.17e}" for r in mrow]
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main()
