"""FP64 refinement of the complex64 march (aim_opts.refine).

The complex64 grid stages carry a relative error of ~1e-7, so a complex64-operator GMRES
cannot bring the residual of the FP64 system much below that.  With refinement every
step's residual b - Z_0 x is formed with FP64 grid stages and corrected by complex64
solves until it meets the tolerance, so the marched currents converge to those of the
FP64 operator.

Checked on the 480-RWG sphere (60 steps, tol 1e-10): the refined complex64 march
reports FP64 residuals <= tol, needed corrections, and agrees with the oracle's LU march
and with the complex128 march to 1e-8 -- where the unrefined complex64 march is held
only to the 1e-4 bound of the complex64 path.
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
    assert e_ref < 1e-8 and e_128 < 1e-8


def test_refinement_with_batch_and_sai():
    """Several right-hand sides and the SAI preconditioner: each refined wave matches its
    complex128 march (per-RHS residual checks; the FP64 residual runs in chunks of the
    refinement buffers)."""
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
        assert rel(i64r[:, b], i128[:, b]) < 1e-7, b
