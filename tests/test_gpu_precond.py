"""The near-zone SAI right preconditioner on the GPU: its values against the oracle's
per-column solves, the diagonal special case, marches that reach the oracle's solution,
fewer GMRES iterations, and the captured solve against the host-driven one."""
import numpy as np
import pytest

from oracle import aim as oaim
from oracle import efie, march
from oracle.precond import near_sai
from oracle.rwg import build_rwg
from paper_1408_7060_gb300.inputs import make_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def s480():
    w = make_workload("sphere480")
    rwg = build_rwg(*w.mesh)
    p = efie.Params(dt=w.dt, f_c=w.f_c, Q=w.order)
    A = oaim.AimOracle(rwg, w.grid_n, w.h, w.origin, w.near_radius, p)
    z0 = efie.fill_pairs(rwg, p, A.pairs, 0)[0]
    return w, rwg, p, A, z0


def ctx(w, **kw):
    from paper_1408_7060_gb300 import AimContext

    return AimContext.from_workload(w, **kw)


def pairs_within(rwg, r):
    """All RWG pairs with edge midpoints within r (inclusive), sorted (brute force)."""
    xe = rwg.midpoint()
    d = xe[:, None, :] - xe[None, :, :]
    a, b = np.nonzero(d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1] + d[..., 2] * d[..., 2] <= r * r)
    return np.stack([a, b], axis=1)


def csr_pairs(rowptr, col):
    return np.stack([np.repeat(np.arange(len(rowptr) - 1), np.diff(rowptr)), col], axis=1)


def test_sai_values_vs_oracle(s480):
    """Near-zone pattern (rows of at most 15): FP64 elimination, agreement to 1e-9."""
    w, rwg, p, A, z0 = s480
    ref = near_sai(rwg.ns, A.pairs, z0)
    for prec in ("c128", "c64"):
        with ctx(w, precision=prec, precond="sai") as c:
            assert c.info["preconditioner"] == 1
            rowptr, col, got = c.preconditioner()
            assert np.array_equal(csr_pairs(rowptr, col), A.pairs)
            assert np.abs(got - ref).max() < 1e-9 * np.abs(ref).max(), prec


def test_sai_wide_pattern_vs_oracle(s480):
    """Pattern of twice the near radius (rows of up to 45: FP32 elimination of the
    normal equations, which are summed in FP64): its pattern is exactly the pairs within
    the radius and its values agree with the oracle's least-squares columns to 1e-3."""
    w, rwg, p, A, z0 = s480
    r = 2 * w.near_radius
    pr = pairs_within(rwg, r)
    zr = efie.fill_pairs(rwg, p, pr, 0)[0]
    ref = near_sai(rwg.ns, pr, zr)
    with ctx(w, precision="c64", precond="sai", precond_radius=r) as c:
        rowptr, col, got = c.preconditioner()
    assert np.array_equal(csr_pairs(rowptr, col), pr)
    assert np.abs(got - ref).max() < 1e-3 * np.abs(ref).max()


def test_diag_getter(s480):
    w, rwg, p, A, z0 = s480
    with ctx(w, precision="c128") as c:
        rowptr, col, got = c.preconditioner()
    assert np.array_equal(rowptr, np.arange(rwg.ns + 1)) and np.array_equal(col, np.arange(rwg.ns))
    diag = A.pairs[:, 0] == A.pairs[:, 1]
    assert np.abs(got * z0[diag] - 1).max() < 1e-10


def test_sai_march_vs_oracle(s480):
    """Same converged march as the oracle's LU march (the preconditioner changes only
    the path of the solve)."""
    w, rwg, p, A, z0 = s480
    nt = 60
    ZA = np.stack([A.dense(m) for m in range(A.n_delays + 1)])
    V = efie.excitation(rwg, p, w.khat, w.phat, w.sigma, w.t_d, np.arange(1, nt + 1))
    ref = march.march_dense(ZA, V)
    with ctx(w, precision="c128", precond="sai") as c:
        cur, stats, rc = c.march(w.khat, w.phat, w.sigma, w.t_d, nt, 1e-10)
    assert stats["last_step"] == nt
    err = np.linalg.norm(cur - ref, axis=2) / np.linalg.norm(ref, axis=2).max(axis=0, keepdims=True)
    assert err.max() < 1e-6, err.max()


def test_sai_fewer_iterations(s480):
    w = s480[0]
    its = {}
    for key, kw in (("diag", {}), ("sai", {"precond": "sai"}),
                    ("sai2", {"precond": "sai", "precond_radius": 2 * w.near_radius})):
        with ctx(w, precision="c64", **kw) as c:
            _, stats, _ = c.march(w.khat, w.phat, w.sigma, w.t_d, 40, 1e-6)
            its[key] = stats["total_iters"]
    assert its["sai"] <= 0.75 * its["diag"], its
    assert its["sai2"] < its["sai"], its


def test_sai_graph_matches_host_loop(s480):
    import os

    w = s480[0]
    os.environ["AIM_GB300_GRAPHS"] = "0"
    try:
        with ctx(w, precision="c64", precond="sai") as c0:
            a, sa, _ = c0.march(w.khat, w.phat, w.sigma, w.t_d, 25, 1e-6)
    finally:
        del os.environ["AIM_GB300_GRAPHS"]
    with ctx(w, precision="c64", precond="sai") as c1:
        b, sb, _ = c1.march(w.khat, w.phat, w.sigma, w.t_d, 25, 1e-6)
    assert sa["total_iters"] == sb["total_iters"]
    assert np.array_equal(a, b)


def test_sai_full_size_iterations():
    """The 7680-RWG sphere (64^3 grid): short marches with the diagonal, the near-zone
    SAI and the SAI on twice the near radius reach the same currents (to the solver
    tolerance) with fewer iterations each."""
    w = make_workload("sphere7680")
    out = {}
    for key, kw in (("diag", {}), ("sai", {"precond": "sai"}),
                    ("sai2", {"precond": "sai", "precond_radius": 2 * w.near_radius})):
        with ctx(w, **kw) as c:
            cur, stats, rc = c.march(w.khat, w.phat, w.sigma, w.t_d, 30, 1e-6)
            out[key] = (cur, stats["total_iters"])
    a = out["diag"][0]
    for key in ("sai", "sai2"):
        assert np.linalg.norm(out[key][0] - a) <= 1e-4 * np.linalg.norm(a), key
    assert out["sai2"][1] < out["sai"][1] < out["diag"][1], {k: v[1] for k, v in out.items()}
    print(f"\nsphere7680, 30 steps: GMRES iterations diag {out['diag'][1]}, near SAI {out['sai'][1]}, "
          f"SAI on 2 x the near radius {out['sai2'][1]}")


def test_zero_start_march_vs_oracle(s480):
    """GMRES started from zero (the first residual is b, no operator product) reaches the
    oracle's LU march like the warm start does, with either preconditioner."""
    w, rwg, p, A, z0 = s480
    nt = 60
    ZA = np.stack([A.dense(m) for m in range(A.n_delays + 1)])
    V = efie.excitation(rwg, p, w.khat, w.phat, w.sigma, w.t_d, np.arange(1, nt + 1))
    ref = march.march_dense(ZA, V)
    for kw in ({}, {"precond": "sai"}):
        with ctx(w, precision="c128", zero_start=True, **kw) as c:
            cur, stats, rc = c.march(w.khat, w.phat, w.sigma, w.t_d, nt, 1e-10)
        assert stats["last_step"] == nt
        err = np.linalg.norm(cur - ref, axis=2) / np.linalg.norm(ref, axis=2).max(axis=0, keepdims=True)
        assert err.max() < 1e-6, (kw, err.max())


def test_zero_start_graph_matches_host_loop(s480):
    import os

    w = s480[0]
    os.environ["AIM_GB300_GRAPHS"] = "0"
    try:
        with ctx(w, precision="c64", precond="sai", zero_start=True) as c0:
            a, sa, _ = c0.march(w.khat, w.phat, w.sigma, w.t_d, 25, 1e-6)
    finally:
        del os.environ["AIM_GB300_GRAPHS"]
    with ctx(w, precision="c64", precond="sai", zero_start=True) as c1:
        b, sb, _ = c1.march(w.khat, w.phat, w.sigma, w.t_d, 25, 1e-6)
    assert sa["total_iters"] == sb["total_iters"]
    assert np.array_equal(a, b)
