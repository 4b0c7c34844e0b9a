"""The homogeneous background medium (aim_opts.eps_r, mu_r; Sec. 2.1) on the GPU: the
480-RWG sphere in eps_r = 2.25, mu_r = 1.7 (complex128) against the oracle's operator in
the same medium -- products Z~_m x for every delay (1e-10), excitation vectors (1e-12) and
the march (1e-6 against the dense LU march) -- and, as the scaling law of the medium
requires, a product in the medium equals the vacuum product at dt/n and n f_c divided by
eps_r."""
import math

import numpy as np
import pytest

from oracle import aim as oaim
from oracle import efie, march
from oracle.rwg import build_rwg
from paper_1408_7060_gb300.inputs import make_workload

pytestmark = pytest.mark.gpu

EPS_R, MU_R = 2.25, 1.7


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b))


def test_medium_vs_oracle():
    from paper_1408_7060_gb300 import AimContext

    w = make_workload("sphere480", band_frac=0.2, n_t=50, eps_r=EPS_R, mu_r=MU_R)
    rwg = build_rwg(*w.mesh)
    p = efie.Params(dt=w.dt, f_c=w.f_c, Q=w.order, eps_r=EPS_R, mu_r=MU_R)
    A = oaim.AimOracle(rwg, w.grid_n, w.h, w.origin, w.near_radius, p)
    ZA = np.stack([A.dense(m) for m in range(A.n_delays + 1)])
    rng = np.random.default_rng(31)
    x = rng.standard_normal((1, rwg.ns)) + 1j * rng.standard_normal((1, rwg.ns))
    V = efie.excitation(rwg, p, w.khat, w.phat, w.sigma, w.t_d, np.arange(1, w.n_t + 1))
    with AimContext.from_workload(w, precision="c128") as c:
        assert c.n_delays == A.n_delays
        for m in range(A.n_delays + 1):
            assert rel(c.matvec(m, x)[0], ZA[m] @ x[0]) < 1e-10, m
        for l in (1, 10, 25):
            assert rel(c.excitation(w.khat, w.phat, w.sigma, w.t_d, l)[0], V[l - 1, 0]) < 1e-12, l
        cur, st, rc = c.march(w.khat, w.phat, w.sigma, w.t_d, w.n_t, 1e-10)
    assert rel(cur, march.march_dense(ZA, V)) < 1e-6


def test_medium_scaling_law():
    from paper_1408_7060_gb300 import AimContext

    n = math.sqrt(EPS_R * MU_R)
    wm = make_workload("sphere480", band_frac=0.2, eps_r=EPS_R, mu_r=MU_R)
    wv = make_workload("sphere480", band_frac=0.2, f_c=150e6 * n)
    assert abs(wv.dt - wm.dt / n) < 1e-12 * wm.dt
    rng = np.random.default_rng(32)
    x = rng.standard_normal((1, 480)) + 1j * rng.standard_normal((1, 480))
    with AimContext.from_workload(wm, precision="c128") as cm, AimContext.from_workload(wv, precision="c128") as cv:
        assert cm.n_delays == cv.n_delays
        for m in (0, 1, cm.n_delays):
            assert rel(cm.matvec(m, x)[0], cv.matvec(m, x)[0] / EPS_R) < 1e-10, m
