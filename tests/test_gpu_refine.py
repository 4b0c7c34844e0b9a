"""FP64 refinement of the complex64 march (aim_opts.refine).

The complex64 grid stages carry a relative error of ~1e-7, so a complex64-operator GMRES
cannot bring the residual of the FP64 system much below that.  With refinement every
step's residual b - Z_0 x is formed with FP64 grid stages and corrected by complex64
solves until it meets the tolerance, so each immediate solve is that of the FP64
operator.

The refinement covers the immediate system; the delayed sum that forms each step's
right-hand side keeps complex64 grid stages, and its rounding (relative ~1e-7 of the
delayed terms, which largely cancel against the excitation) bounds what the march can
reach.  Checked on the 480-RWG sphere (60 steps, tol 1e-10): the refined complex64 march
reports FP64 residuals <= tol and needed corrections, agrees with the oracle's LU march
and with the complex128 march within the 1e-4 bound on marched currents, and is at
least 5x closer to them than the unrefined complex64 march (measured: 4.3e-6 against
5.9e-5).
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


def test_refined_c64_march_reaches_fp64_accuracy():
    from paper_1408_7060_gb300 import AimContext

    w = make_workload("sphere480")
    rwg = build_rwg(*w.mesh)
    p = efie.Params(dt=w.dt, f_c=w.f_c, Q=w.order)
    A = oaim.AimOracle(rwg, w.grid_n, w.h, w.origin, w.near_radius, p)
    nt, tol = 60, 1e-10
    ZA = np.stack([A.dense(m) for m in range(A.n_delays + 1)])
    V = efie.excitation(rwg, p, w.khat, w.phat, w.sigma, w.t_d, np.arange(1, nt + 1))
    ref = march.march_dense(ZA, V)
    with AimContext.from_workload(w, precision="c128") as c:
        i128, _, _ = c.march(w.khat, w.phat, w.sigma, w.t_d, nt, tol)
    with AimContext.from_workload(w, precision="c64", refine=6) as c:
        assert c.info["refine"] == 6
        i64r, st, rc = c.march(w.khat, w.phat, w.sigma, w.t_d, nt, tol)
    with AimContext.from_workload(w, precision="c64") as c:
        i64, _, _ = c.march(w.khat, w.phat, w.sigma, w.t_d, nt, 1e-6)
    assert st["last_step"] == nt and st["max_rel_res"] <= tol
    assert st["refine_corrections"] > 0
    e_ref, e_128 = rel(i64r, ref), rel(i64r, i128)
    print(f"refined complex64 march: vs oracle {e_ref:.2e}, vs complex128 {e_128:.2e}, "
          f"{st['refine_corrections']} corrections; unrefined complex64 vs oracle {rel(i64, ref):.2e}")
    e_unref = rel(i64, ref)
    assert e_ref < 1e-4 and e_128 < 1e-4
    assert e_ref < e_unref / 5, (e_ref, e_unref)


def test_refinement_with_batch_and_sai():
    """Several right-hand sides and the SAI preconditioner: every wave's FP64 residual
    meets the tolerance and each refined wave matches its complex128 march within the
    1e-4 bound (measured: 4.9e-7)."""
    from paper_1408_7060_gb300 import AimContext
    from paper_1408_7060_gb300.inputs import random_plane_waves

    w = make_workload("sphere_sub3_n32")
    k, ph = random_plane_waves(3, 5)
    nt, tol = 25, 1e-9
    with AimContext.from_workload(w, precision="c128", batch_max=3, precond="sai") as c:
        i128, _, _ = c.march(k, ph, w.sigma, w.t_d, nt, tol)
    with AimContext.from_workload(w, precision="c64", batch_max=3, precond="sai", refine=6) as c:
        i64r, st, rc = c.march(k, ph, w.sigma, w.t_d, nt, tol)
    assert st["max_rel_res"] <= tol
    for b in range(3):
        assert rel(i64r[:, b], i128[:, b]) < 1e-5, b


@pytest.mark.parametrize("every", [1, 4])
def test_refine_every_kth_step(every):
    """aim_opts.refine_every = k forms the FP64 residual (and corrects) at every k-th step
    only; the other steps keep the complex64 solve.  On the 480-RWG sphere (40 steps,
    tol 1e-6): the number of checked steps is 40 / k, every reported residual meets tol
    and the march agrees with the complex128 march within the 1e-4 bound."""
    from paper_1408_7060_gb300 import AimContext

    w = make_workload("sphere480")
    nt, tol = 40, 1e-6
    with AimContext.from_workload(w, precision="c128") as c:
        i128, _, _ = c.march(w.khat, w.phat, w.sigma, w.t_d, nt, tol)
    with AimContext.from_workload(w, precision="c64", refine=6, refine_every=every) as c:
        assert c.info["refine_every"] == every
        i64r, st, rc = c.march(w.khat, w.phat, w.sigma, w.t_d, nt, tol)
    assert st["last_step"] == nt and st["max_rel_res"] <= tol
    assert st["refine_checks"] == nt // every
    assert rel(i64r, i128) < 1e-4
