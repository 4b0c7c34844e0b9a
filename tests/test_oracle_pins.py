"""Pins of the CPU oracle to facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a closed form,
an independent quadrature, a library routine used for a special case, the Mie
series, brute force on a tiny input, or values printed in the paper.
"""
import math
import os

import numpy as np
import pytest

from oracle import aim, efie, march, mie, quad, singular, tbasis
from oracle.constants import C0
from oracle.rwg import build_rwg
from paper_1408_7060_gb300.inputs import icosphere, make_workload

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------- fixtures

@pytest.fixture(scope="module")
def s480():
    w = make_workload("sphere480")
    rwg = build_rwg(*w.mesh)
    p = efie.Params(dt=w.dt, f_c=w.f_c, Q=2)
    return w, rwg, p


@pytest.fixture(scope="module")
def s480_Z(s480):
    w, rwg, p = s480
    return efie.fill_dense(rwg, p)


@pytest.fixture(scope="module")
def s480_aim(s480):
    w, rwg, p = s480
    return aim.AimOracle(rwg, w.grid_n, w.h, w.origin, w.near_radius, p)


# --------------------------------------------------------------------------- paper values

def test_table1_band_convention():
    """Table I: f_c + 3/(2 pi sigma) = 300 MHz, chi = f_max/f_bw matches the labels."""
    rows = [l.split() for l in open(os.path.join(GOLD, "table1_pulses.txt")) if l[0] != "#"]
    for lab, fc, sig, td in rows:
        sigma = eval(sig, {"pi": math.pi}) * 1e-6
        fbw = 3.0 / (2 * math.pi * sigma)
        fmax = float(fc) * 1e6 + fbw
        assert abs(fmax - 300e6) < 1e-3 * 300e6
        chi = fmax / fbw
        assert abs(chi - float(lab)) / float(lab) < 0.03
        w = make_workload("sphere480", f_c=float(fc) * 1e6, band_frac=fbw / (float(fc) * 1e6))
        assert abs(w.sigma - sigma) < 1e-12 * sigma and abs(w.t_d - 8 * sigma) < 1e-20


def test_sec23_chi():
    rows = [l.split() for l in open(os.path.join(GOLD, "sec23_chi.txt")) if l[0] != "#"]
    for _, lo, hi, chi in rows:
        fbw = (float(hi) - float(lo)) / 2
        assert abs(float(hi) / fbw - float(chi)) < 1e-9 * float(chi)


# --------------------------------------------------------------------------- P1 basis

@pytest.mark.parametrize("Q", [1, 2, 3, 4])
def test_cppif_interpolation_and_reproduction(Q):
    j = np.arange(-3, 8)
    v = tbasis.T(j.astype(float), Q)
    assert np.allclose(v, (j == 0).astype(float), rtol=0, atol=1e-14)
    u = np.linspace(-0.999, 3.7, 211)
    for q in range(Q + 1):
        for d in range(3):
            s = sum((jj ** q) * tbasis.T(u - jj, Q, d) for jj in range(-8, 12))
            ref = np.polynomial.polynomial.polyval(u, np.polynomial.polynomial.polyder(
                np.eye(q + 1)[q], d) if d else np.eye(q + 1)[q])
            assert np.allclose(s, ref, atol=1e-11 * max(1.0, np.abs(ref).max())), (q, d)


def test_cppif_quadratic_closed_form():
    u = np.array([-0.5, 0.0, 0.5, 1.0, 1.5, 2.0, 2.5, -1.0])
    ref = np.array([0.375, 1.0, 0.75, 0.0, -0.125, 0.0, 0.0, 0.0])
    assert np.allclose(tbasis.T(u, 2), ref, atol=1e-15)


# --------------------------------------------------------------------------- quadrature

def test_cowper7_degree5():
    bary, w = quad.cowper7()
    assert abs(w.sum() - 1) < 1e-15
    # int over the unit triangle of x^a y^b = a! b! / (a+b+2)!, area 1/2
    for a in range(6):
        for b in range(6 - a):
            val = 0.5 * np.sum(w * bary[:, 0] ** a * bary[:, 1] ** b)
            ref = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            assert abs(val - ref) < 1e-15


def test_collapsed_gauss_exact():
    bary, w = quad.collapsed_gauss(6)
    for a in range(11):
        for b in range(11 - a):
            val = 0.5 * np.sum(w * bary[:, 0] ** a * bary[:, 1] ** b)
            ref = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            assert abs(val - ref) < 1e-14 * max(ref, 1e-3)


# --------------------------------------------------------------------------- P8 singular

def test_potential_integrals_vs_quadrature():
    rng = np.random.default_rng(5)
    bary, w = quad.collapsed_gauss(300)
    for _ in range(6):
        A, B, C = rng.standard_normal((3, 3))
        area = 0.5 * np.linalg.norm(np.cross(B - A, C - A))
        n = np.cross(B - A, C - A)
        n /= np.linalg.norm(n)
        # off-plane point and an in-plane interior point (split at the singular point)
        for r in (A / 3 + B / 3 + C / 3 + 0.7 * n + 0.1 * (B - A), 0.2 * A + 0.5 * B + 0.3 * C):
            I0, I1 = singular.potential_integrals(r, A, B, C)
            q0, q1 = 0.0, np.zeros(3)
            for a, b in ((A, B), (B, C), (C, A)):
                p = bary[:, 0:1] * a + bary[:, 1:2] * b + bary[:, 2:3] * r
                ar = 0.5 * np.linalg.norm(np.cross(b - a, r - a))
                if ar == 0:
                    continue
                # sub-triangle (a, b, r) with r at the collapsed vertex; sign by orientation
                sgn = np.sign(np.dot(np.cross(b - a, r - a), n)) if abs(np.dot(r - A, n)) < 1e-12 else None
                if sgn is None:
                    continue
                R = np.linalg.norm(p - r, axis=1)
                q0 += sgn * ar * np.sum(w / R)
                q1 += sgn * ar * np.sum(w[:, None] * (p - r) / R[:, None], axis=0)
            if abs(np.dot(r - A, n)) < 1e-12:
                assert abs(I0 - q0) < 1e-10 * abs(q0)
                assert np.linalg.norm(I1 - q1) < 1e-10 * np.linalg.norm(q1)
            else:
                pts = bary[:, 0:1] * A + bary[:, 1:2] * B + bary[:, 2:3] * C
                R = np.linalg.norm(pts - r, axis=1)
                assert abs(I0 - area * np.sum(w / R)) < 1e-10 * abs(I0)
                ref1 = area * np.sum(w[:, None] * (pts - r) / R[:, None], axis=0)
                assert np.linalg.norm(I1 - ref1) < 1e-10 * np.linalg.norm(ref1)


# --------------------------------------------------------------------------- RWG

def test_rwg_table(s480):
    w, rwg, p = s480
    nt = len(rwg.F)
    assert rwg.ns == 3 * nt // 2 == 480
    k, s, fv = rwg.tri_bases()
    assert (k >= 0).all() and sorted(np.bincount(k.ravel())) == [2] * rwg.ns
    for e in range(rwg.ns):
        lo, hi = rwg.edge[e]
        assert lo < hi
        f = list(rwg.F[rwg.tri[e, 0]])
        i = f.index(lo)
        assert f[(i + 1) % 3] == hi            # T+ runs lo -> hi counter-clockwise
        a, b = rwg.V[lo], rwg.V[hi]
        mid = 0.5 * (a + b)
        tang = (b - a) / np.linalg.norm(b - a)
        for side, sign, want in ((0, 1.0, 1.0), (1, -1.0, -1.0)):
            vf = rwg.V[rwg.free[e, side]]
            t = rwg.tri[e, side]
            S = sign * rwg.length[e] / (2 * rwg.area[t]) * (mid - vf)
            ax = (mid - vf) - np.dot(mid - vf, tang) * tang
            ax /= np.linalg.norm(ax)           # in-plane edge normal pointing away from the apex
            # unit normal flux leaves T+ and enters T- (current continuity)
            assert abs(np.dot(S, ax) - want) < 1e-12


# --------------------------------------------------------------------------- P5, P6

def test_reciprocity(s480_Z, s480):
    w, rwg, p = s480
    g = efie.Geometry(rwg)
    Z = s480_Z
    # far pairs: exactly symmetric (same rule on both triangles)
    t = np.arange(len(rwg.F))
    T_, TP_ = np.meshgrid(t, t, indexing="ij")
    sing = g.singular_mask(T_.ravel(), TP_.ravel()).reshape(T_.shape)
    far = np.ones((rwg.ns, rwg.ns), dtype=bool)
    for a in range(2):
        for b in range(2):
            far &= ~sing[rwg.tri[:, a][:, None], rwg.tri[:, b][None, :]]
    for m in range(Z.shape[0]):
        sc = np.abs(Z[m]).max()
        assert np.abs((Z[m] - Z[m].T)[far]).max() < 1e-13 * sc
        assert np.abs(Z[m] - Z[m].T).max() < 2e-3 * sc


def test_dc_identity_operator(s480_Z, s480):
    """sum_m Z_m = j w_c Z^FD(f_c) (Sec. 3.1 compares ET-MOT with FD-MoM)."""
    w, rwg, p = s480
    ZF = efie.fill_dense(rwg, p, freq=True)
    S = s480_Z.sum(0)
    assert np.abs(S - 1j * p.wc * ZF).max() < 1e-13 * np.abs(S).max()


def test_dc_identity_operator_open_plate():
    """The same identity on an open surface (the 1 m plate of Table II, its boundary edges
    carrying no basis), with the plates' CPPIF of order 3."""
    w = make_workload("plate280")
    rwg = build_rwg(*w.mesh)
    p = efie.Params(dt=w.dt, f_c=w.f_c, Q=w.order)
    S = efie.fill_dense(rwg, p).sum(0)
    ZF = efie.fill_dense(rwg, p, freq=True)
    assert rwg.ns == 280
    assert np.abs(S - 1j * p.wc * ZF).max() < 1e-13 * np.abs(S).max()


def test_dc_identity_excitation(s480):
    """dt sum_l V_l = j w sigma sqrt(2 pi) e^{-j w t_d} V^FD (Gaussian sample sum)."""
    w, rwg, p = s480
    V = efie.excitation(rwg, p, w.khat, w.phat, w.sigma, w.t_d, np.arange(-40, 80))
    VF = efie.excitation_fd(rwg, p, w.khat, w.phat)[0]
    lhs = w.dt * V[:, 0].sum(0)
    rhs = 1j * p.wc * w.sigma * math.sqrt(2 * math.pi) * np.exp(-1j * p.wc * w.t_d) * VF
    assert np.linalg.norm(lhs - rhs) < 1e-12 * np.linalg.norm(rhs)


def test_dc_identity_march_narrowband():
    """A stable narrow-band march sums to the FD-MoM solution (whole ET-MOT march)."""
    w = make_workload("sphere480", f_c=150e6, band_frac=0.02, n_t=100)
    rwg = build_rwg(*w.mesh)
    p = efie.Params(dt=w.dt, f_c=w.f_c, Q=2)
    Z = efie.fill_dense(rwg, p)
    V = efie.excitation(rwg, p, w.khat, w.phat, w.sigma, w.t_d, np.arange(1, w.n_t + 1))
    I = march.march_dense(Z, V)
    ZF = efie.fill_dense(rwg, p, freq=True)
    VF = efie.excitation_fd(rwg, p, w.khat, w.phat)[0]
    ref = np.linalg.solve(ZF, VF) * w.sigma * math.sqrt(2 * math.pi) * np.exp(-1j * p.wc * w.t_d)
    S = w.dt * I[:, 0].sum(0)
    assert np.linalg.norm(S - ref) < 1e-9 * np.linalg.norm(ref)
    assert np.linalg.norm(I[-1, 0]) < 1e-12 * np.linalg.norm(I, axis=2).max()


def test_march_gmres_matches_lu(s480_Z, s480):
    w, rwg, p = s480
    Z = s480_Z
    V = efie.excitation(rwg, p, w.khat, w.phat, w.sigma, w.t_d, np.arange(1, 21))
    I1 = march.march_dense(Z, V)
    I2, its = march.march_operator(lambda m, x: Z[m] @ x, Z.shape[0] - 1, V, tol=1e-12)
    assert np.abs(I1 - I2).max() < 1e-9 * np.abs(I1).max()


# --------------------------------------------------------------------------- P7 Mie

def test_mie_limits():
    a = 1.0
    # Rayleigh: backscatter of a small PEC sphere = 9 pi a^2 (ka)^4
    ka = 0.01
    s = mie.rcs(ka, ka / a, np.pi)
    assert abs(s / (9 * np.pi * a * a * ka ** 4) - 1) < 1e-3
    # optical limit: backscatter -> pi a^2
    s = mie.rcs(60.0, 60.0, np.pi)
    assert abs(s / (np.pi * a * a) - 1) < 0.05
    # backscatter is polarisation independent
    assert abs(mie.rcs(3.0, 3.0, np.pi, "E") - mie.rcs(3.0, 3.0, np.pi, "H")) < 1e-12


def test_fdmom_vs_mie():
    """FD-MoM EFIE with the oracle's rules converges to the Mie series."""
    errs = []
    for sub in (2, 3):
        V, F = icosphere(sub, 1.0)
        rwg = build_rwg(V, F)
        p = efie.Params(dt=1e-9, f_c=150e6)
        ZF = efie.fill_dense(rwg, p, freq=True)
        VF = efie.excitation_fd(rwg, p, [0, 0, 1], [1, 0, 0])[0]
        I = np.linalg.solve(ZF, VF)
        th = np.linspace(0.01, np.pi - 0.01, 37)
        rh = np.stack([np.sin(th), 0 * th, np.cos(th)], 1)
        pol = np.stack([np.cos(th), 0 * th, -np.sin(th)], 1)
        s = efie.rcs_fd(rwg, p, I, rh, pol)
        sm = mie.rcs(p.kc, p.kc, th, "E")
        errs.append(np.abs(10 * np.log10(s / sm)).max())
        assert mie.db_error(s, sm, np.sin(th)) < 1e-3
    assert errs[0] < 1.0 and errs[1] < 0.3 and errs[1] < errs[0]


def test_db_error_norm():
    s = np.array([1.0, 0.1, 1e-12])
    assert mie.db_error(s, s) == 0.0
    # values below TH = peak - 80 dB are clipped to 0 dB
    assert mie.db_error(np.array([1.0, 1e-9]), np.array([1.0, 1e-10])) == 0.0


# --------------------------------------------------------------------------- AIM (P2, P3, P4)

def test_moment_matching_reproduces_cubics(s480_aim, s480):
    """sum_n L_c[n,k] p(r_n) = int S_k^c p dS for per-axis-cubic p (independent rule)."""
    w, rwg, p = s480
    A = s480_aim
    rng = np.random.default_rng(3)
    coef = rng.standard_normal((4, 4, 4))
    bary, wq = quad.collapsed_gauss(14)

    def poly(r):
        x = (r[..., 0] - 0.1) / 0.7
        y = (r[..., 1] + 0.2) / 0.7
        z = (r[..., 2] - 0.05) / 0.7
        return np.einsum("ijk,...i,...j,...k->...", coef, np.stack([x ** i for i in range(4)], -1),
                         np.stack([y ** i for i in range(4)], -1), np.stack([z ** i for i in range(4)], -1))

    ijk = A.node_ijk(A.nodes)                                     # [ns,64,3]
    rn = A.origin + A.h * ijk
    pn = poly(rn)
    for k in range(0, rwg.ns, 23):
        ref = np.zeros(4)
        for side, sign in ((0, 1.0), (1, -1.0)):
            t = rwg.tri[k, side]
            P = quad.points(rwg.V, rwg.F[t:t + 1], bary)[0]
            Wt = wq * rwg.area[t]
            S = sign * rwg.length[k] / (2 * rwg.area[t]) * (P - rwg.V[rwg.free[k, side]])
            pv = poly(P)
            ref[:3] += np.einsum("q,qc,q->c", Wt, S, pv)
            ref[3] += sign * rwg.length[k] / rwg.area[t] * np.sum(Wt * pv)
        got = A.lam[:, k, :] @ pn[k]
        assert np.allclose(got, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


def test_grid_convolution_fft_equals_direct(s480_aim):
    A = s480_aim
    rng = np.random.default_rng(1)
    src = np.zeros(A.n ** 3, dtype=complex)
    idx = rng.choice(A.n ** 3, 300, replace=False)
    src[idx] = rng.standard_normal(300) + 1j * rng.standard_normal(300)
    for m in range(A.n_delays + 1):
        for kind in (0, 1):
            a = A.conv_direct(m, src, kind)
            b = A.conv_fft(m, src, kind)
            assert np.linalg.norm(a - b) < 1e-12 * np.linalg.norm(a)


def test_box_deep_z_period_gives_the_linear_convolution(s480_aim):
    """Sources confined to n_z consecutive z-planes: a circular convolution of z period
    L_z >= 2 n_z (kernel offsets |dz| < L_z/2 taken from the 2N embedding, the plane L_z/2
    zero) gives on those planes the values of the 2N-padded linear convolution -- the
    reading behind the library's box-deep z transforms."""
    A = s480_aim
    n = A.n
    z0, nz = 5, 6
    rng = np.random.default_rng(41)
    src = np.zeros((n, n, n), dtype=complex)  # [z][y][x]
    src[z0:z0 + nz] = rng.standard_normal((nz, n, n)) + 1j * rng.standard_normal((nz, n, n))
    for m, kind in ((0, 0), (1, 1)):
        ref = A.conv_fft(m, src.ravel(), kind).reshape(n, n, n)[z0:z0 + nz]
        G2 = A.kernel_grid(m, kind)  # [z][y][x], period 2N
        for lz in (2 * nz, 16):
            iz = np.arange(lz)
            dz = np.where(iz < lz // 2, iz, iz - lz)
            G = G2[dz % (2 * n)].copy()
            G[lz // 2] = 0
            a = np.zeros((lz, 2 * n, 2 * n), dtype=complex)
            a[:nz, :n, :n] = src[z0:z0 + nz]
            out = np.fft.ifftn(np.fft.fftn(a) * np.fft.fftn(G))[:nz, :n, :n]
            assert np.abs(out - ref).max() < 1e-12 * np.abs(ref).max(), (m, kind, lz)


def test_grid_convolution_point_source(s480_aim):
    """A unit source at one node radiates the kernel itself: P[n] = G_m(n - n0)."""
    A = s480_aim
    n = A.n
    n0 = (3 * n + 5) * n + 7
    src = np.zeros(n ** 3, dtype=complex)
    src[n0] = 1.0
    P = A.conv_fft(1, src, 0)
    ijk = A.node_ijk(np.arange(n ** 3))
    d = ijk - A.node_ijk(np.array([n0]))
    R = A.h * np.sqrt((d.astype(float) ** 2).sum(1))
    v = 1 - R / A.p.cdt
    pp = A.p
    D2T = tbasis.T(v, 2, 2) / pp.dt ** 2 + 2j * pp.wc * tbasis.T(v, 2, 1) / pp.dt - pp.wc ** 2 * tbasis.T(v, 2)
    with np.errstate(divide="ignore", invalid="ignore"):
        ref = np.where(R > 0, D2T * np.exp(-1j * pp.kc * R) / R, 0)
    assert np.abs(P - ref).max() < 1e-12 * np.abs(ref).max()


def test_aim_with_everything_near_is_mot():
    """r_near >= diameter: pre-correction restores the direct matrices exactly."""
    w = make_workload("sphere_sub1_n10", f_c=150e6)
    rwg = build_rwg(*w.mesh)
    p = efie.Params(dt=w.dt, f_c=w.f_c, Q=2)
    A = aim.AimOracle(rwg, w.grid_n, w.h, w.origin, 10.0, p)
    Z = efie.fill_dense(rwg, p, n_delays=A.n_delays)
    for m in range(A.n_delays + 1):
        assert np.abs(A.dense(m) - Z[m]).max() < 1e-12 * np.abs(Z[0]).max()


def test_aim_no_near_is_grid_operator(s480):
    w, rwg, p = s480
    A = aim.AimOracle(rwg, w.grid_n, w.h, w.origin, -1.0, p)
    assert len(A.pairs) == 0
    rng = np.random.default_rng(2)
    x = rng.standard_normal(rwg.ns) + 1j * rng.standard_normal(rwg.ns)
    y = A.matvec(0, x, "direct")
    assert np.linalg.norm(y - A.fft_dense(0) @ x) < 1e-12 * np.linalg.norm(y)


def test_aim_fft_part_symmetric(s480_aim):
    A = s480_aim
    for m in (0, 2):
        Zf = A.fft_dense(m)
        assert np.abs(Zf - Zf.T).max() < 1e-13 * np.abs(Zf).max()


def test_n_delays(s480_aim, s480):
    """N_g from the largest stencil-node distance: floor(R_max/(c dt) + Q)."""
    w, rwg, p = s480
    A = s480_aim
    ijk = A.node_ijk(A.active).astype(float)
    lo, hi = ijk.min(0), ijk.max(0)
    # the active set of a sphere spans its bounding box diagonal or less
    assert A.n_delays <= math.floor(A.h * np.linalg.norm(hi - lo) / (C0 * w.dt) + 2)
    assert A.n_delays >= math.floor(A.h * (hi - lo).max() / (C0 * w.dt) + 2)


def test_direct_sum_offset_table_large_grid():
    """On grids above 64^3 the direct sum looks G up by |offset|; it must equal the
    kernel evaluated at the signed offsets."""
    w = make_workload("sphere_sub1_n96", f_c=150e6)
    rwg = build_rwg(*w.mesh)
    p = efie.Params(dt=w.dt, f_c=w.f_c, Q=2)
    A = aim.AimOracle(rwg, w.grid_n, w.h, w.origin, w.near_radius, p)
    rng = np.random.default_rng(4)
    src = np.zeros(A.n ** 3, dtype=complex)
    idx = rng.choice(A.n ** 3, 200, replace=False)
    src[idx] = rng.standard_normal(200) + 1j * rng.standard_normal(200)
    tg = rng.choice(A.n ** 3, 50, replace=False)
    for kind in (0, 1):
        got = A.conv_direct(1, src, kind, targets=tg)
        d = A.node_ijk(tg)[:, None, :] - A.node_ijk(idx)[None, :, :]
        ref = A.kernel_values(1, d)[kind] @ src[idx]
        assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()


def test_setup_shortcuts_match_plain(s480_aim):
    """The convex-hull reduction for N_g and the k-d tree prefilter of the near pairs
    (taken on large meshes) give what the plain all-pairs scans give."""
    A = s480_aim
    assert A._n_delays_grid(hull_above=0) == A._n_delays_grid(hull_above=10 ** 9)
    assert np.array_equal(A._near_pairs(tree_above=0), A._near_pairs(tree_above=10 ** 9))


def test_singular_threshold_has_margin_on_test_meshes():
    """Singular pairs are those sharing a vertex or with centroids closer than twice the
    mean edge length (R15).  On every mesh the parity tests use, no centroid distance lies
    within 1e-9 (relative) of that threshold, so the decision cannot depend on the order
    in which either side sums the edge lengths (a difference of ~1e-16 relative)."""
    from scipy.spatial import cKDTree

    from paper_1408_7060_gb300.inputs import ellipsoid_mesh, sphere_array

    meshes = [icosphere(s, 1.0) for s in range(1, 6)] + [sphere_array(s, 0.5, 1.5) for s in (2, 3, 5)]
    meshes.append(ellipsoid_mesh())
    for V, F in meshes:
        rwg = build_rwg(V, F) if len(F) < 30000 else None
        if rwg is not None:
            me = efie.Geometry(rwg).mean_edge
        else:  # the same mean over the unique edges, without the RWG table
            e = np.unique(np.sort(np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]]), 1), axis=0)
            me = float(np.mean(np.linalg.norm(V[e[:, 1]] - V[e[:, 0]], axis=1)))
        c = V[F].mean(axis=1)
        pr = cKDTree(c).query_pairs(2 * me * (1 + 1e-6), output_type="ndarray")
        d = np.linalg.norm(c[pr[:, 0]] - c[pr[:, 1]], axis=1)
        assert np.abs(d - 2 * me).min() > 1e-9 * 2 * me, len(F)
