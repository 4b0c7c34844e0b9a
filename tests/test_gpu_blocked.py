"""The multilevel blocked delayed sums of the right-hand side (aim_opts.rhs_blocked,
Sec. 4 stage ii) on the GPU.

* 480-RWG sphere at 150 MHz +-20 % (N_g <= 4, squares of 1, 2 and 4 steps): the
  blocked complex128 march agrees with the oracle's LU march of the AIM operator (1e-6)
  and with the direct-sum march within the solves' tolerance (both solved to 1e-10: the
  sums differ in rounding order only, measured 3.7e-11 over 60 steps; bound 1e-9);
* the same sphere at 1.2 GHz +-50 % (N_g = 24 > 16: 32-step top squares, launched as
  16-step sub-squares, the one whose delays all exceed N_g skipped): blocked and direct
  marches agree within 1e-9 in complex128 and 1e-5 in complex64;
* 7680-RWG sphere (complex64, N_g = 7): blocked and direct marches agree within 1e-5 and
  the blocked march keeps matching across aim_march_continue calls (its pending sums
  carry over).
"""
import numpy as np
import pytest

from oracle import aim as oaim
from oracle import efie, march
from oracle.rwg import build_rwg
from paper_1408_7060_gb300.inputs import make_workload

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b))


def test_blocked_march_vs_oracle_and_direct():
    from paper_1408_7060_gb300 import AimContext

    w = make_workload("sphere480", band_frac=0.2, n_t=60)
    rwg = build_rwg(*w.mesh)
    p = efie.Params(dt=w.dt, f_c=w.f_c, Q=w.order)
    A = oaim.AimOracle(rwg, w.grid_n, w.h, w.origin, w.near_radius, p)
    ZA = np.stack([A.dense(m) for m in range(A.n_delays + 1)])
    V = efie.excitation(rwg, p, w.khat, w.phat, w.sigma, w.t_d, np.arange(1, w.n_t + 1))
    ref = march.march_dense(ZA, V)
    with AimContext.from_workload(w, precision="c128", rhs_blocked=1) as c:
        assert c.info["rhs_blocked"] == 1 and c.n_delays == A.n_delays
        blk, st, _ = c.march(w.khat, w.phat, w.sigma, w.t_d, w.n_t, 1e-10)
    with AimContext.from_workload(w, precision="c128") as c:
        dirc, _, _ = c.march(w.khat, w.phat, w.sigma, w.t_d, w.n_t, 1e-10)
    assert st["last_step"] == w.n_t
    assert rel(blk, ref) < 1e-6
    assert rel(blk, dirc) < 1e-9


def test_blocked_sub_squares_large_ng():
    from paper_1408_7060_gb300 import AimContext

    w = make_workload("sphere480", f_c=1.2e9, band_frac=0.5, n_t=80)
    got = {}
    for prec in ("c128", "c64"):
        for blocked in (0, 1):
            with AimContext.from_workload(w, precision=prec, rhs_blocked=blocked) as c:
                assert c.n_delays > 16
                got[prec, blocked] = c.march(w.khat, w.phat, w.sigma, w.t_d, w.n_t, 1e-10 if prec == "c128" else 1e-6)[0]
    assert rel(got["c128", 1], got["c128", 0]) < 1e-9
    assert rel(got["c64", 1], got["c64", 0]) < 1e-5


def test_blocked_sphere7680_with_continue():
    import torch

    from paper_1408_7060_gb300 import AimContext

    w = make_workload("sphere7680")
    n1, n2 = 23, 17
    out = {}
    for blocked in (0, 1):
        with AimContext.from_workload(w, rhs_blocked=blocked) as c:
            a = torch.empty((n1, 1, c.ns), dtype=torch.complex128, device="cuda")
            b = torch.empty((n2, 1, c.ns), dtype=torch.complex128, device="cuda")
            c.march(w.khat, w.phat, w.sigma, w.t_d, n1, w.tol, out=a)
            c.march_continue(w.khat, w.phat, w.sigma, w.t_d, n2, w.tol, out=b)
            out[blocked] = torch.cat([a, b]).cpu().numpy()
    assert rel(out[1], out[0]) < 1e-5
