"""Pins of the oracle's envelope-derivative terms by time moments.

The sums over delays, steps or taps that the DC identities use (zeroth moments) cancel
every T' and T'' term: the CPPIF partition of unity gives sum_j T^(d)(u - j) = 0 for
d = 1, 2.  The first and second moments do not.  With the CPPIF reproduction property
(Sec. 3, Eq. 3; exact for monomials of degree q <= Q),

    sum_m m^q T^(d)(m - tau) = (-1)^q [d^d/du^d u^q]_{u = -tau},

so  sum_m m T(m - tau) = tau,  sum_m m T'(m - tau) = -1,  sum_m m T''(m - tau) = 0,
    sum_m m^2 T(m - tau) = tau^2,  sum_m m^2 T' = -2 tau,  sum_m m^2 T'' = 2.

Each moment of the envelope operators (Eq. 4 with D = d/dt + j w_c, Sec. 1) is then a
Galerkin integral with a kernel that is a polynomial in R/(c dt) times e^{-j k_c R}/R,
filled here through the oracle's triangle-pair cubature with those kernels written out
in closed form.  A changed coefficient of T' in D^2 T (the 2 j w_c T'/dt term), of T''
or of the Gaussian's derivative in the excitation (Eq. 1) fails one of these pins; the
zeroth-moment pins cannot see them.

The excitation's first moment follows from the Gaussian's sample sums (Poisson summation
error below e^{-70} for these pulses):
    sum_l l g(l dt - d) = d sigma sqrt(2 pi) / dt^2,   sum_l l g'(l dt - d) = -sigma sqrt(2 pi) / dt^2.
"""
import math

import numpy as np
import pytest

from oracle import adjoint, efie, quad, tbasis
from oracle.constants import C0, EPS0, MU0
from oracle.rwg import build_rwg
from paper_1408_7060_gb300.inputs import icosphere, make_workload

CA = MU0 / (4 * math.pi)
CP = 1.0 / (4 * math.pi * EPS0)


@pytest.fixture(scope="module", params=[2, 3], ids=["Q2", "Q3"])
def small(request):
    """80-triangle sphere (120 RWG), the 150 MHz +-50 % pulse of the 480-RWG workload, CPPIF
    of order Q = 2 (the sphere workloads) and Q = 3 (the plates)."""
    w = make_workload("sphere480")
    V, F = icosphere(1, 1.0)
    rwg = build_rwg(V, F)
    p = efie.Params(dt=w.dt, f_c=w.f_c, Q=request.param)
    return w, rwg, p


def galerkin_fill(rwg, p, gA, gA0, dgA0, gP, gP0, dgP0):
    """Dense Galerkin matrix  int int [mu/4pi S.S' gA(R) + 1/(4 pi eps) div S div' S' gP(R)] / R
    through the oracle's cubature and singularity extraction, for kernels given as
    callables of R with their values and one-sided derivatives at R = 0+."""
    g = efie.Geometry(rwg)
    nt = len(rwg.F)

    def kern(m, R, p_):
        return gA(R)[None], gP(R)[None]

    def kern0(m, p_):
        return (np.array([gA0], dtype=complex), np.array([gP0], dtype=complex),
                np.array([dgA0], dtype=complex), np.array([dgP0], dtype=complex))

    out = np.zeros((1, rwg.ns, rwg.ns), dtype=complex)
    T_, TP_ = np.meshgrid(np.arange(nt), np.arange(nt), indexing="ij")
    T_, TP_ = T_.ravel(), TP_.ravel()
    blk = efie.tri_pair_blocks(g, T_, TP_, np.zeros(1), p, kern=kern, kern0=kern0, scale=(CA, CP))
    efie._assemble(g, T_, TP_, blk, out, rwg.ns)
    return out[0]


def test_cppif_moment_sums():
    """The moment sums used below, checked on the basis itself over a range of tau."""
    tau = np.linspace(0.0, 3.7, 97)
    m = np.arange(0, 12)[:, None]
    for Q in (2, 3):
        T = [tbasis.T(m - tau[None], Q, d) for d in range(3)]
        assert np.allclose((m * T[0]).sum(0), tau, atol=1e-13)
        assert np.allclose((m * T[1]).sum(0), -1.0, atol=1e-12)
        assert np.allclose((m * T[2]).sum(0), 0.0, atol=1e-11)
        assert np.allclose((m ** 2 * T[0]).sum(0), tau ** 2, atol=1e-12)
        assert np.allclose((m ** 2 * T[1]).sum(0), -2 * tau, atol=1e-11)
        assert np.allclose((m ** 2 * T[2]).sum(0), 2.0, atol=1e-10)


@pytest.fixture(scope="module")
def small_Z(small):
    w, rwg, p = small
    return efie.fill_dense(rwg, p)


def test_first_moment_of_the_delay_matrices(small, small_Z):
    """sum_m m Z_m: kernels A: (-2 j w/dt - w^2 R/(c dt)) e^{-jkR}, phi: R/(c dt) e^{-jkR}."""
    w, rwg, p = small
    wc, k, cdt, dt = p.wc, p.kc, p.cdt, p.dt
    ph = lambda R: np.exp(-1j * k * R)
    ref = galerkin_fill(rwg, p,
                        lambda R: (-2j * wc / dt - wc ** 2 * R / cdt) * ph(R), -2j * wc / dt,
                        -wc ** 2 / cdt - 1j * k * (-2j * wc / dt),
                        lambda R: R / cdt * ph(R), 0.0, 1.0 / cdt)
    m = np.arange(small_Z.shape[0])
    got = np.tensordot(m, small_Z, axes=(0, 0))
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


def test_second_moment_of_the_delay_matrices(small, small_Z):
    """sum_m m^2 Z_m: kernels A: (2/dt^2 - 4 j w R/(c dt^2) - w^2 R^2/(c dt)^2) e^{-jkR},
    phi: (R/(c dt))^2 e^{-jkR}."""
    w, rwg, p = small
    wc, k, cdt, dt = p.wc, p.kc, p.cdt, p.dt
    ph = lambda R: np.exp(-1j * k * R)
    a0 = 2.0 / dt ** 2
    ref = galerkin_fill(rwg, p,
                        lambda R: (a0 - 4j * wc * R / (cdt * dt) - wc ** 2 * (R / cdt) ** 2) * ph(R), a0,
                        -4j * wc / (cdt * dt) - 1j * k * a0,
                        lambda R: (R / cdt) ** 2 * ph(R), 0.0, 0.0)
    m = np.arange(small_Z.shape[0])
    got = np.tensordot(m.astype(float) ** 2, small_Z, axes=(0, 0))
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


def _test_integral(rwg, f):
    """<S_k, F(r)> for a vector field F(points[nt,7,3]) -> [nt,7,3], by the 7-point rule
    written out from the RWG definition (Sec. 3): [ns] complex."""
    bary, wq = quad.cowper7()
    P = quad.points(rwg.V, rwg.F, bary)
    Fv = f(P)
    out = np.zeros(rwg.ns, dtype=complex)
    for side, sign in ((0, 1.0), (1, -1.0)):
        t = rwg.tri[:, side]
        S = sign * (rwg.length / (2 * rwg.area[t]))[:, None, None] * (P[t] - rwg.V[rwg.free[:, side]][:, None, :])
        out += np.einsum("q,k,kqx,kqx->k", wq, rwg.area[t], S, Fv[t])
    return out


def test_excitation_first_moment(small):
    """sum_l l V_l = sigma sqrt(2 pi)/dt^2 <S_k, p (-1 + j w d(r)) e^{-j w d(r)}>,
    d(r) = r.k/c + t_d (Eq. 1 with the Gaussian's derivative g' = -tau/sigma^2 g)."""
    w, rwg, p = small
    l = np.arange(-40, 90)
    V = efie.excitation(rwg, p, w.khat, w.phat, w.sigma, w.t_d, l)[:, 0]
    got = np.tensordot(l.astype(float), V, axes=(0, 0))
    kh, ph_ = w.khat[0], w.phat[0]

    def field(P):
        d = P @ kh / C0 + w.t_d
        s = (-1.0 + 1j * p.wc * d) * np.exp(-1j * p.wc * d)
        return s[..., None] * ph_
    ref = w.sigma * math.sqrt(2 * math.pi) / w.dt ** 2 * _test_integral(rwg, field)
    assert np.linalg.norm(got - ref) < 1e-11 * np.linalg.norm(ref)


def test_incident_taps_moments(small):
    """Taps B_s of the sampled-envelope excitation: sum_s B_s = <S_k, p j w e^{-jk r.k}> and
    sum_s s B_s = <S_k, p (-1/dt + j w u) e^{-jk r.k}>, u = r.k/(c dt)."""
    w, rwg, p = small
    s = np.arange(-6, 9)
    kh, ph_ = w.khat[0], w.phat[0]
    B = adjoint.incident_taps(rwg, p, kh, ph_, list(s))
    for q, coef in ((0, lambda u: 1j * p.wc + 0 * u), (1, lambda u: -1.0 / p.dt + 1j * p.wc * u)):
        got = np.tensordot(s.astype(float) ** q, B, axes=(0, 0))

        def field(P):
            u = P @ kh / p.cdt
            return (coef(u) * np.exp(-1j * p.kc * (P @ kh)))[..., None] * ph_
        ref = _test_integral(rwg, field)
        assert np.linalg.norm(got - ref) < 1e-12 * np.linalg.norm(ref), q


def test_farfield_taps_moments(small):
    """Taps A_s of the far-field envelope: sum_s A_s = int S.e j w e^{+jk r.r'} and
    sum_s s A_s = int S.e (-1/dt - j w w_r) e^{+jk r.r'}, w_r = r.r'/(c dt)."""
    w, rwg, p = small
    s = np.arange(-6, 9)
    rhat = np.array([[0.3, -0.4, math.sqrt(1 - 0.25)]])
    e1 = np.cross(rhat[0], [1.0, 0, 0])
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(rhat[0], e1)
    A = adjoint.farfield_taps(rwg, p, rhat, e1[None], e2[None], list(s))     # [ns_, 1, 2, ns]
    for q, coef in ((0, lambda u: 1j * p.wc + 0 * u), (1, lambda u: -1.0 / p.dt - 1j * p.wc * u)):
        got = np.tensordot(s.astype(float) ** q, A[:, 0], axes=(0, 0))       # [2, ns]
        for qq, e in enumerate((e1, e2)):
            def field(P):
                u = P @ rhat[0] / p.cdt
                return (coef(u) * np.exp(1j * p.kc * (P @ rhat[0])))[..., None] * e
            ref = _test_integral(rwg, field)
            assert np.linalg.norm(got[qq] - ref) < 1e-12 * np.linalg.norm(ref), (q, qq)
