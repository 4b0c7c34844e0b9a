"""Pins of the oracle's BLIF temporal basis and its causal extrapolation (Sec. 3, Sec. 3.1.2).

* the closed form against mpmath: T and its first three derivatives equal 40-digit numerical
  derivatives of sinc(u) sinh(b sqrt(M^2 - u^2)) / sqrt(M^2 - u^2) / G(M^2);
* interpolation: T(n) = delta_n0 at every integer, T = 0 outside (-M, M) and T -> 0 at +-M;
* band-limited reproduction: sum_n exp(j w n) T(u - n) = exp(j w u) for every in-band w, with
  an error that falls exponentially with M at the rate of the guard band b = pi (1 - 2 beta)
  (a wrong guard band, at either band fraction, breaks one of the bounds);
* extrapolation: exact (to rounding) for sums of the fit exponentials when there are as many
  frequencies as samples; real weights for the symmetric frequency set; in-band error small
  at the paper's fine oversampling (beta ~ 1/15);
* the effective time factor T_m folds the extrapolated samples exactly: the causal sum
  sum_m T_m(m - x) I_{l-m} equals the two-sided BLIF sum over the known samples and the
  extrapolated ones;
* the BLIF ET-MOT march gives the frequency-domain RCS of the same mesh (Sec. 2.4, Eq. 2),
  more closely at finer oversampling (a wrong guard band fails it).
"""
import math

import mpmath as mp
import numpy as np
import pytest

from oracle import blif

CASES = [(3, 0.25), (3, 1 / 15), (5, 0.1), (2, 0.3)]


def _T_mp(u, M, beta):
    b = mp.pi * (1 - 2 * mp.mpf(beta))
    u = mp.mpf(u)
    if abs(u) >= M:
        return mp.mpf(0)
    G = lambda s: mp.sinh(b * mp.sqrt(s)) / mp.sqrt(s)
    sc = mp.sin(mp.pi * u) / (mp.pi * u) if u != 0 else mp.mpf(1)
    return sc * G(M * M - u * u) / G(M * M)


@pytest.mark.parametrize("M,beta", CASES)
def test_values_and_derivatives_vs_mpmath(M, beta):
    mp.mp.dps = 40
    pts = [0.0, 1e-6, 0.3, -0.77, 1.5, 2.2 * M / 3, -(M - 0.1), M - 1e-5]
    for u in pts:
        for d in range(4):
            got = blif.T(np.array([u]), M, beta, d)[0]
            ref = float(mp.diff(lambda t: _T_mp(t, M, beta), u, d))
            assert abs(got - ref) <= 1e-13 * max(1.0, abs(ref)), (M, beta, u, d, got, ref)


@pytest.mark.parametrize("M,beta", CASES)
def test_interpolatory_and_support(M, beta):
    n = np.arange(-M - 2, M + 3).astype(float)
    T = blif.T(n, M, beta)
    assert T[n == 0][0] == 1.0
    assert np.abs(T[n != 0]).max() < 1e-15
    assert np.all(blif.T(np.array([M, -M, M + 0.5, -M - 3.0]), M, beta) == 0.0)
    edge = blif.T(np.array([M - 1e-9, -(M - 1e-9)]), M, beta)
    assert np.abs(edge).max() < 1e-8


def _reproduction_error(M, beta):
    u = np.linspace(-0.5, 0.5, 41)
    n = np.arange(-M - 2, M + 3)
    worst = 0.0
    for w in np.linspace(-2 * math.pi * beta, 2 * math.pi * beta, 21):
        s = (np.exp(1j * w * n)[None, :] * blif.T(u[:, None] - n[None, :], M, beta)).sum(1)
        worst = max(worst, float(np.abs(s - np.exp(1j * w * u)).max()))
    return worst


def test_band_limited_reproduction_converges_with_half_width():
    # measured errors with margin: beta = 1/4: 4.7e-3, 1.6e-4, 1.1e-5; beta = 1/15: 2.3e-4,
    # 5.9e-7, 2.0e-9 (M = 3, 5, 7); each halving of the guard band's decay would exceed them
    bounds = {0.25: (6e-3, 2.5e-4, 1.5e-5), 1 / 15: (3e-4, 1e-6, 4e-9)}
    for beta, bnd in bounds.items():
        errs = [_reproduction_error(M, beta) for M in (3, 5, 7)]
        assert all(e < b for e, b in zip(errs, bnd)), (beta, errs)
        assert errs[0] > errs[1] > errs[2]


def test_extrapolation_exact_with_square_fit():
    rng = np.random.default_rng(5)
    om = np.array([-0.9, -0.2, 0.35, 0.8])
    E = blif.extrapolation(M=3, beta=0.25, n_samp=4, omegas=om)
    c = rng.standard_normal(4) + 1j * rng.standard_normal(4)
    x = lambda n: (c * np.exp(1j * om * n)).sum()
    l = 7
    for p in (1, 2):
        pred = sum(E[p, q] * x(l - q) for q in range(4))
        assert abs(pred - x(l + p)) < 1e-11 * abs(x(l + p))


def test_extrapolation_real_and_accurate_in_band():
    for beta, bounds in ((1 / 15, (0.03, 0.1)), (0.25, (0.7, 1.3))):
        E = blif.extrapolation(3, beta)
        assert np.abs(E.imag).max() < 1e-12
        ws = np.linspace(-2 * math.pi * beta, 2 * math.pi * beta, 41)
        for p, bnd in zip((1, 2), bounds):
            err = max(abs(np.exp(1j * w * p) - (E[p] * np.exp(-1j * w * np.arange(3))).sum()) for w in ws)
            assert err < bnd, (beta, p, err)
    # the finer the oversampling, the better the extrapolation
    e = [blif.extrapolation(3, b) for b in (0.02, 0.05, 0.1)]
    errs = []
    for b, E in zip((0.02, 0.05, 0.1), e):
        ws = np.linspace(-2 * math.pi * b, 2 * math.pi * b, 41)
        errs.append(max(abs(np.exp(1j * w) - (E[1] * np.exp(-1j * w * np.arange(3))).sum()) for w in ws))
    assert errs[0] < errs[1] < errs[2]


@pytest.mark.parametrize("M,beta", [(3, 0.25), (4, 0.1)])
def test_effective_factor_folds_the_extrapolation(M, beta):
    rng = np.random.default_rng(6)
    E = blif.extrapolation(M, beta)
    l = 20
    I = rng.standard_normal(l + 1)           # samples 0..l
    fut = {l + p: sum(E[p, q].real * I[l - q] for q in range(M)) for p in range(1, M)}
    for x in (0.0, 0.4, 1.3, 2.7, 5.5):
        for d in range(3):
            causal = sum(blif.T_eff(m, np.array([m - x]), M, beta, E, d)[0] * I[l - m] for m in range(l + 1))
            full = sum(blif.T(np.array([l - n - x]), M, beta, d)[0] * I[n] for n in range(l + 1))
            full += sum(blif.T(np.array([l - n - x]), M, beta, d)[0] * v for n, v in fut.items())
            assert abs(causal - full) < 1e-13 * max(1.0, abs(full)), (x, d)


def test_blif_march_rcs_matches_frequency_domain_and_improves_with_oversampling():
    """The BLIF ET-MOT march (Eq. 4 with the extrapolated time factors) of the 120-RWG sphere,
    150 MHz +-5 %, transformed with the BLIF's spectrum (Sec. 2.4), gives the frequency-domain
    EFIE RCS of the same mesh in the dB norm of Eq. 2 -- at f_c and at f_c +- f_bw/2 -- and more
    closely at the finer oversampling beta = 1/15 than at 1/4 (Sec. 3.1.2: the ET-MOT error
    falls as the oversampling rises).  Measured: 1.5e-7, 3.4e-6, 6.0e-6 at beta = 1/4 and
    8.6e-10, 1.5e-8, 2.3e-8 at beta = 1/15."""
    from oracle import efie, march, mie, rcs
    from oracle.rwg import build_rwg
    from paper_1408_7060_gb300.inputs import icosphere

    rwg = build_rwg(*icosphere(1, 1.0))
    f_c, fb = 150e6, 0.05 * 150e6
    sigma = 3 / (2 * math.pi * fb)
    t_d = 8 * sigma
    rh, eth, wts, _, _ = rcs.sphere_directions(12, 12)
    freqs = (f_c, f_c + 0.5 * fb, f_c - 0.5 * fb)
    ref = {}
    for f in freqs:
        pf = efie.Params(dt=1e-9, f_c=f)
        I_fd = np.linalg.solve(efie.fill_dense(rwg, pf, freq=True), efie.excitation_fd(rwg, pf, [0, 0, 1], [1, 0, 0])[0])
        ref[f] = efie.rcs_fd(rwg, pf, I_fd, rh, eth)
    errs = {}
    for beta, bounds in ((0.25, (1e-6, 2e-5, 2e-5)), (1 / 15, (1e-8, 1e-7, 1e-7))):
        dt = beta / fb
        p = efie.Params(dt=dt, f_c=f_c, basis="blif", M=3, beta=beta)
        n_t = int(2 * t_d / dt) + int(30 * 0.25 / beta)
        V = efie.excitation(rwg, p, [0, 0, 1], [1, 0, 0], sigma, t_d, np.arange(1, n_t + 1))
        I = march.march_dense(efie.fill_dense(rwg, p), V)[:, 0]
        errs[beta] = [mie.db_error(rcs.rcs_td(rwg, p, I, sigma, t_d, f, rh, eth), ref[f], wts) for f in freqs]
        assert all(e < b for e, b in zip(errs[beta], bounds)), (beta, errs[beta])
    assert all(a < b for a, b in zip(errs[1 / 15], errs[0.25]))
