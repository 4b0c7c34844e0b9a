"""Failure paths of the C ABI, each made on the host side (no GPU fault):

* an iteration cap the solver cannot meet -> AIM_ERR_NOCONV, with the statistics of the
  steps that did complete (stats.last_step) and a context that stays usable;
* a mesh with an inconsistently oriented face, and one with a non-manifold edge ->
  AIM_ERR_MESH from aim_setup, nothing leaked (an open surface is accepted: its
  boundary edges carry no basis function);
* the chi = 3 march of the 480-RWG sphere, which grows after the pulse as Sec. 3.1
  reports for broadband CPPIF marches -> AIM_WARN_UNSTABLE once the last current
  exceeds 1e3 times the largest of the run's first half.
"""
import numpy as np
import pytest

from paper_1408_7060_gb300.inputs import icosphere, make_workload

pytestmark = pytest.mark.gpu


def test_iteration_cap_reports_noconv():
    from paper_1408_7060_gb300 import AimContext, abi

    w = make_workload("sphere480")
    with AimContext.from_workload(w, precision="c128", max_iter=1) as c:
        with pytest.raises(abi.AimError) as e:
            c.march(w.khat, w.phat, w.sigma, w.t_d, 5, 1e-10)
        assert e.value.code == abi.AIM_ERR_NOCONV
        assert e.value.stats["last_step"] == 0          # no step reached the tolerance
        assert e.value.stats["iters"][0, 0] >= 1
        x = np.ones((1, c.ns), dtype=np.complex128)
        y = c.matvec(0, x)                              # the context is still usable
        assert np.all(np.isfinite(y))
    with AimContext.from_workload(w, precision="c128") as c2:
        assert np.allclose(c2.matvec(0, x), y, rtol=0, atol=1e-12 * np.abs(y).max())


@pytest.mark.parametrize("defect", ["flipped", "non-manifold"])
def test_bad_mesh_rejected(defect):
    from paper_1408_7060_gb300 import abi

    w = make_workload("sphere480")
    V, F = icosphere(2, 1.0)
    if defect == "flipped":
        F = F.copy()
        F[0] = F[0, [0, 2, 1]]                          # its three edges traversed twice the same way
    else:
        F = np.concatenate([F, F[:1, [0, 2, 1]]])       # an edge shared by three faces
    with pytest.raises(abi.AimError) as e:
        abi.aim_setup(V, F, w.grid_n, w.origin, w.h, w.near_radius, w.dt, w.f_c, precision="c128")
    assert e.value.code == abi.AIM_ERR_MESH


def test_open_surface_accepted():
    from paper_1408_7060_gb300 import abi

    w = make_workload("sphere480")
    V, F = icosphere(2, 1.0)
    h = abi.aim_setup(V, F[1:], w.grid_n, w.origin, w.h, w.near_radius, w.dt, w.f_c, precision="c128")
    try:
        assert abi.aim_get_info(h)["ns"] == 480 - 3     # the removed face's edges are boundary edges
    finally:
        abi.aim_destroy(h)


def test_late_time_growth_warns():
    from paper_1408_7060_gb300 import AimContext, abi

    w = make_workload("sphere480")
    with AimContext.from_workload(w, precision="c128") as c:
        cur, st, rc = c.march(w.khat, w.phat, w.sigma, w.t_d, 200, 1e-6)
    assert rc == abi.AIM_WARN_UNSTABLE
    assert st["last_step"] == 200
    n = np.linalg.norm(cur[:, 0], axis=1)
    assert n[-1] > 1e3 * n[:100].max()
