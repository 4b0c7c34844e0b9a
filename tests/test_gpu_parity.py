"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Small cases (a 480-RWG sphere on a 16^3 grid, a 1920-RWG sphere on a 32^3 grid)
span several FFT tiles and ragged stencil/near-zone rows; the 7680-RWG sphere on
the 64^3 grid is the benchmark workload, compared on sampled outputs.

Tolerances: complex128 path 1e-10 relative (FP64 rounding through the FFTs);
complex64 grid path 1e-5 relative L2 per matvec and 1e-4 for marched currents;
integer/index tables bit-exact.
"""
import numpy as np
import pytest

from oracle import aim as oaim
from oracle import efie, march
from oracle.rwg import build_rwg
from paper_1408_7060_gb300.inputs import make_workload

pytestmark = pytest.mark.gpu

CASES = {}


def case(name, **over):
    key = (name, tuple(sorted(over.items())))
    if key not in CASES:
        w = make_workload(name, **over)
        rwg = build_rwg(*w.mesh)
        p = efie.Params(dt=w.dt, f_c=w.f_c, Q=w.order)
        A = oaim.AimOracle(rwg, w.grid_n, w.h, w.origin, w.near_radius, p)
        CASES[key] = (w, rwg, p, A)
    return CASES[key]


def ctx_for(w, **over):
    from paper_1408_7060_gb300 import AimContext

    return AimContext.from_workload(w, **over)


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b))


@pytest.fixture(scope="module")
def s480():
    return case("sphere480")


@pytest.fixture(scope="module")
def s480_ctx(s480):
    w = s480[0]
    c = ctx_for(w, precision="c128")
    yield c
    c.close()


@pytest.fixture(scope="module")
def s480_ctx64(s480):
    w = s480[0]
    c = ctx_for(w, precision="c64")
    yield c
    c.close()


# ------------------------------------------------------------------ setup tables

def test_rwg_table_bit_exact(s480, s480_ctx):
    w, rwg, p, A = s480
    e, t, f = s480_ctx.rwg_table()
    assert np.array_equal(e, rwg.edge) and np.array_equal(t, rwg.tri) and np.array_equal(f, rwg.free)


def test_anterp_tables(s480, s480_ctx):
    w, rwg, p, A = s480
    anchor, lam = s480_ctx.anterp()
    assert np.array_equal(anchor, A.anchor)
    ref = np.transpose(A.lam, (1, 0, 2))               # [ns][4][64]
    assert np.abs(lam - ref).max() < 1e-11 * np.abs(ref).max()


def test_n_delays_and_active(s480, s480_ctx):
    w, rwg, p, A = s480
    assert s480_ctx.n_delays == A.n_delays
    assert s480_ctx.info["n_active"] == len(A.active)


def test_near_zone(s480, s480_ctx):
    w, rwg, p, A = s480
    rowptr, col, val = s480_ctx.near()
    assert np.array_equal(col, A.pairs[:, 1]) and np.array_equal(np.diff(rowptr), np.bincount(A.pairs[:, 0], minlength=rwg.ns))
    ref = A.near_values()
    for m in range(A.n_delays + 1):
        sc = np.abs(ref[0]).max()
        assert np.abs(val[m] - ref[m]).max() < 1e-9 * sc, m


def z_embedded(G2, lz):
    """The (2N)^3 kernel grid [z][y][x] re-embedded with z period lz: offsets |dz| < lz/2
    taken from the 2N grid, plane lz/2 zero (the layout the context's z transform uses)."""
    n2 = G2.shape[0]
    iz = np.arange(lz)
    dz = np.where(iz < lz // 2, iz, iz - lz)
    out = G2[dz % n2].copy()
    out[lz // 2] = 0
    return out


def test_kernel_spectra(s480, s480_ctx):
    w, rwg, p, A = s480
    n = A.n
    lz = s480_ctx.info["z_len"]
    assert lz % 16 == 0 and 2 * (s480_ctx.info["box_hi"][2] - s480_ctx.info["box_lo"][2] + 1) <= lz <= 2 * n
    M = (2 * n) ** 2 * lz
    for m in range(A.n_delays + 1):
        for kind in (0, 1):
            G = np.fft.fftn(z_embedded(A.kernel_grid(m, kind), lz))[: lz // 2 + 1, : n + 1, : n + 1]
            G *= (oaim.CA if kind == 0 else oaim.CP) / M
            got = s480_ctx.kernel_spectrum(m, kind)
            assert np.abs(got - G).max() < 1e-12 * np.abs(G).max(), (m, kind)


# ------------------------------------------------------------------ operator

def test_matvec_c128(s480, s480_ctx):
    w, rwg, p, A = s480
    rng = np.random.default_rng(7)
    x = rng.standard_normal((2, rwg.ns)) + 1j * rng.standard_normal((2, rwg.ns))
    for m in range(A.n_delays + 1):
        y = s480_ctx.matvec(m, x[:1])
        assert rel(y[0], A.matvec(m, x[0])) < 1e-10, m


def test_matvec_c128_device_pointers(s480, s480_ctx):
    import torch

    w, rwg, p, A = s480
    rng = np.random.default_rng(8)
    x = rng.standard_normal((1, rwg.ns)) + 1j * rng.standard_normal((1, rwg.ns))
    y = s480_ctx.matvec(1, torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(y[0], A.matvec(1, x[0])) < 1e-10


def test_matvec_c64(s480, s480_ctx64):
    w, rwg, p, A = s480
    rng = np.random.default_rng(9)
    x = rng.standard_normal((1, rwg.ns)) + 1j * rng.standard_normal((1, rwg.ns))
    for m in range(A.n_delays + 1):
        assert rel(s480_ctx64.matvec(m, x)[0], A.matvec(m, x[0])) < 1e-5, m


def test_excitation(s480, s480_ctx):
    w, rwg, p, A = s480
    for l in (1, 10, 17, 30):
        V = s480_ctx.excitation(w.khat, w.phat, w.sigma, w.t_d, l)
        ref = efie.excitation(rwg, p, w.khat, w.phat, w.sigma, w.t_d, [l])[0]
        assert rel(V, ref) < 1e-12


def test_rhs(s480, s480_ctx, s480_ctx64):
    w, rwg, p, A = s480
    ng = A.n_delays
    rng = np.random.default_rng(11)
    hist = rng.standard_normal((ng, 1, rwg.ns)) + 1j * rng.standard_normal((ng, 1, rwg.ns))
    for l in (1, 2, ng, ng + 5):
        ref = sum(A.matvec(m, hist[m - 1, 0]) for m in range(1, ng + 1) if l - m >= 1) if l > 1 else np.zeros(rwg.ns)
        got = s480_ctx.rhs(l, hist)[0]
        got64 = s480_ctx64.rhs(l, hist)[0]
        if l == 1:
            assert np.abs(got).max() == 0.0 and np.abs(got64).max() == 0.0
        else:
            assert rel(got, ref) < 1e-10
            assert rel(got64, ref) < 1e-5


# ------------------------------------------------------------------ march

def test_march_c128_vs_oracle(s480, s480_ctx):
    """The GPU march solves Eq. 5 with the oracle's operator: compare with the
    oracle's LU march over the first 60 steps (the chi = 3 march grows later, as
    Sec. 3.1.1 predicts for CPPIF; both grow identically)."""
    w, rwg, p, A = s480
    nt = 60
    ZA = np.stack([A.dense(m) for m in range(A.n_delays + 1)])
    V = efie.excitation(rwg, p, w.khat, w.phat, w.sigma, w.t_d, np.arange(1, nt + 1))
    ref = march.march_dense(ZA, V)
    cur, stats, rc = s480_ctx.march(w.khat, w.phat, w.sigma, w.t_d, nt, 1e-10)
    assert stats["last_step"] == nt
    err = np.linalg.norm(cur - ref, axis=2) / np.linalg.norm(ref, axis=2).max(axis=0, keepdims=True)
    assert err.max() < 1e-6, err.max()


def test_march_c64_vs_oracle(s480, s480_ctx64):
    w, rwg, p, A = s480
    nt = 60
    ZA = np.stack([A.dense(m) for m in range(A.n_delays + 1)])
    V = efie.excitation(rwg, p, w.khat, w.phat, w.sigma, w.t_d, np.arange(1, nt + 1))
    ref = march.march_dense(ZA, V)
    cur, stats, rc = s480_ctx64.march(w.khat, w.phat, w.sigma, w.t_d, nt, 1e-6)
    err = np.linalg.norm(cur - ref) / np.linalg.norm(ref)
    assert err < 1e-4, err


# ------------------------------------------------------------------ a second size (32^3 grid, 1920 RWG)

@pytest.fixture(scope="module")
def s1920():
    return case("sphere_sub3_n32")


def test_matvec_sub3(s1920):
    w, rwg, p, A = s1920
    rng = np.random.default_rng(3)
    x = rng.standard_normal((1, rwg.ns)) + 1j * rng.standard_normal((1, rwg.ns))
    with ctx_for(w, precision="c128") as c128, ctx_for(w, precision="c64") as c64:
        assert c128.n_delays == A.n_delays
        for m in (0, 1, A.n_delays):
            ref = A.matvec(m, x[0])
            assert rel(c128.matvec(m, x)[0], ref) < 1e-10
            assert rel(c64.matvec(m, x)[0], ref) < 1e-5


# ------------------------------------------------------------------ benchmark workload, sampled rows

def test_matvec_full_size_sampled():
    """7680-RWG sphere on the 64^3 grid (complex64): sampled output rows against
    direct grid sums and the oracle's near-zone entries for those rows."""
    w = make_workload("sphere7680")
    rwg = build_rwg(*w.mesh)
    p = efie.Params(dt=w.dt, f_c=w.f_c, Q=w.order)
    A = oaim.AimOracle(rwg, w.grid_n, w.h, w.origin, w.near_radius, p)
    rng = np.random.default_rng(5)
    x = rng.standard_normal((1, rwg.ns)) + 1j * rng.standard_normal((1, rwg.ns))
    rows = np.sort(rng.choice(rwg.ns, 12, replace=False))
    with ctx_for(w) as c:
        assert c.n_delays == A.n_delays
        for m in (0, 1):
            y = c.matvec(m, x)[0]
            ref = A.fft_part_rows(m, x[0], rows)
            sel = np.isin(A.pairs[:, 0], rows)
            pr = A.pairs[sel]
            Zn = efie.fill_pairs(rwg, p, pr, m)[m] - A.fft_pairs(m, pr)
            near = np.zeros(len(rows), dtype=complex)
            for (k, kp), z in zip(pr, Zn):
                near[np.searchsorted(rows, k)] += z * x[0, kp]
            ref = ref + near
            assert rel(y[rows], ref) < 1e-5, m


# ------------------------------------------------------------------ solver modes, resume

def test_graph_solver_matches_host_loop(s480):
    """The captured solve (conditional WHILE graph) runs the same kernels in the same
    order as the host-driven loop: identical currents."""
    import os

    w = s480[0]
    os.environ["AIM_GB300_GRAPHS"] = "0"
    try:
        with ctx_for(w, precision="c64") as c0:
            a, sa, _ = c0.march(w.khat, w.phat, w.sigma, w.t_d, 25, 1e-6)
    finally:
        del os.environ["AIM_GB300_GRAPHS"]
    with ctx_for(w, precision="c64") as c1:
        b, sb, _ = c1.march(w.khat, w.phat, w.sigma, w.t_d, 25, 1e-6)
    assert sa["total_iters"] == sb["total_iters"]
    assert np.array_equal(a, b)


def test_march_continue_resumes_exactly(s480):
    """march(n1) + march_continue(n2) == march(n1 + n2): the context holds the whole
    state of the march (the last N_g currents and their spectra)."""
    w = s480[0]
    with ctx_for(w, precision="c64") as c:
        full, _, _ = c.march(w.khat, w.phat, w.sigma, w.t_d, 30, 1e-6)
        a, _, _ = c.march(w.khat, w.phat, w.sigma, w.t_d, 12, 1e-6)
        b, _, _ = c.march_continue(w.khat, w.phat, w.sigma, w.t_d, 18, 1e-6)
    assert np.array_equal(np.concatenate([a, b]), full)


def test_matvec_n96_sampled():
    """96^3 grid (padded length 192 = 8*8*3: the radix-3 passes) on the 1920-RWG
    sphere, both precisions, sampled rows against direct grid sums."""
    w = make_workload("sphere_sub3_n96")
    rwg = build_rwg(*w.mesh)
    p = efie.Params(dt=w.dt, f_c=w.f_c, Q=w.order)
    A = oaim.AimOracle(rwg, w.grid_n, w.h, w.origin, w.near_radius, p)
    rng = np.random.default_rng(6)
    x = rng.standard_normal((1, rwg.ns)) + 1j * rng.standard_normal((1, rwg.ns))
    rows = np.sort(rng.choice(rwg.ns, 10, replace=False))
    for m in (0, 1):
        ref = A.fft_part_rows(m, x[0], rows)
        sel = np.isin(A.pairs[:, 0], rows)
        pr = A.pairs[sel]
        Zn = efie.fill_pairs(rwg, p, pr, m)[m] - A.fft_pairs(m, pr)
        for (k, kp), z in zip(pr, Zn):
            ref[np.searchsorted(rows, k)] += z * x[0, kp]
        for prec, tol in (("c128", 1e-10), ("c64", 1e-5)):
            with ctx_for(w, precision=prec) as c:
                assert c.n_delays == A.n_delays
                assert rel(c.matvec(m, x)[0][rows], ref) < tol, (m, prec)


def test_batched_march_vs_oracle(s480):
    """Several plane waves marched together (per-RHS GMRES masks inside one graph)
    give each wave's own march."""
    from paper_1408_7060_gb300.inputs import random_plane_waves

    w, rwg, p, A = s480
    k, pp = random_plane_waves(3, 0)
    nt = 30
    ZA = np.stack([A.dense(m) for m in range(A.n_delays + 1)])
    V = efie.excitation(rwg, p, k, pp, w.sigma, w.t_d, np.arange(1, nt + 1))
    ref = march.march_dense(ZA, V)
    with ctx_for(w, precision="c128", batch_max=3) as c:
        cur, stats, _ = c.march(k, pp, w.sigma, w.t_d, nt, 1e-10)
    assert stats["iters"].shape == (nt, 3)
    for b in range(3):
        err = np.linalg.norm(cur[:, b] - ref[:, b]) / np.linalg.norm(ref[:, b])
        assert err < 1e-6, (b, err)


# ------------------------------------------------------------------ smallest and largest power-of-two z pass

def _oracle_rows(A, rwg, p, m, x, rows):
    """Rows of Z~AIM_m x from direct grid sums plus the oracle's near-zone entries."""
    ref = A.fft_part_rows(m, x, rows)
    pr = A.pairs[np.isin(A.pairs[:, 0], rows)]
    Zn = efie.fill_pairs(rwg, p, pr, m)[m] - A.fft_pairs(m, pr)
    for (k, kp), z in zip(pr, Zn):
        ref[np.searchsorted(rows, k)] += z * x[kp]
    return ref


@pytest.mark.parametrize("name", ["sphere_sub2_n8", "array_sub2_n128"])
def test_pow2_lengths_matvec_and_rhs(name):
    """Padded lengths 16 and 256 (8^3 grid, 480-RWG sphere; 128^3 grid, 4x4 array of
    480-RWG spheres): sampled rows of the operator product and of the spectral-domain
    delay sum, both precisions.  The near zone is one grid step wide so that the grid
    part carries most interactions.  (An RWG many grid steps long makes the order-3
    moment matching ill-conditioned -- large grid sources of alternating sign whose
    sum cancels -- so both meshes keep edges within a few grid steps.)"""
    w = make_workload(name)
    w = make_workload(name, near_radius=1.0 * w.h)
    rwg = build_rwg(*w.mesh)
    p = efie.Params(dt=w.dt, f_c=w.f_c, Q=w.order)
    A = oaim.AimOracle(rwg, w.grid_n, w.h, w.origin, w.near_radius, p)
    ng = A.n_delays
    rng = np.random.default_rng(12)
    x = rng.standard_normal(rwg.ns) + 1j * rng.standard_normal(rwg.ns)
    rows = np.sort(rng.choice(rwg.ns, 6, replace=False))
    used = sorted({1, ng})
    hist = np.zeros((ng, 1, rwg.ns), dtype=complex)
    for m in used:
        hist[m - 1, 0] = rng.standard_normal(rwg.ns) + 1j * rng.standard_normal(rwg.ns)
    ref_mv = {m: _oracle_rows(A, rwg, p, m, x, rows) for m in (0, 1)}
    ref_rhs = sum(_oracle_rows(A, rwg, p, m, hist[m - 1, 0], rows) for m in used)
    for prec, tol in (("c128", 1e-10), ("c64", 1e-5)):
        with ctx_for(w, precision=prec) as c:
            assert c.n_delays == ng
            for m in (0, 1):
                assert rel(c.matvec(m, x[None])[0][rows], ref_mv[m]) < tol, (m, prec)
            assert rel(c.rhs(ng + 2, hist)[0][rows], ref_rhs) < tol, prec


def test_rhs_factor3_sampled():
    """The delayed sum of Eq. 5 on the 96^3 grid (padded length 192 = 64 x 3: the staged
    radix-3 delay-sum kernel, which recomputes each history slab's z-transform), every
    delay m = 1..N_g active, both precisions, sampled rows against the oracle's direct
    grid sums and near-zone entries."""
    w = make_workload("sphere_sub3_n96")
    rwg = build_rwg(*w.mesh)
    p = efie.Params(dt=w.dt, f_c=w.f_c, Q=w.order)
    A = oaim.AimOracle(rwg, w.grid_n, w.h, w.origin, w.near_radius, p)
    ng = A.n_delays
    rng = np.random.default_rng(31)
    hist = rng.standard_normal((ng, 1, rwg.ns)) + 1j * rng.standard_normal((ng, 1, rwg.ns))
    rows = np.sort(rng.choice(rwg.ns, 6, replace=False))
    ref = sum(_oracle_rows(A, rwg, p, m, hist[m - 1, 0], rows) for m in range(1, ng + 1))
    for prec, tol in (("c128", 1e-10), ("c64", 1e-5)):
        with ctx_for(w, precision=prec) as c:
            assert c.n_delays == ng
            got = c.rhs(ng + 1, hist)[0]
            assert rel(got[rows], ref) < tol, prec
