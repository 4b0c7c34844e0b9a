"""Pins of the oracle's MFIE and CFIE (Sec. 2.1, CFIE alpha = 0.5 for spheres).

* the frequency-domain MFIE and CFIE currents of a PEC sphere give the Mie RCS, closer on
  the finer mesh (a wrong sign, normal or Gram factor does not converge);
* sum_m K_m = j w_c K_FD(f_c) (the CPPIF partition of unity, as for the EFIE);
* sum_m m K_m = -(1/dt) K'  with K' the same fill for the kernel (1 + j k R + k^2 R^2)/R^2
  e^{-jkR}/(4 pi) and the Gram factor 1/2: the first time moment, which pins the T'/dt terms
  of (DT) and (D^2 T) that the partition of unity cancels;
* dt sum_l W_l = j w_c sigma sqrt(2 pi) e^{-j w_c t_d} W_FD (the Gaussian sample sum);
* at chi = 3 the CFIE march decays where the EFIE march grows (the EFIE's interior-resonance
  growth on a closed surface; the CFIE is the paper's choice for spheres, Sec. 5.1).
"""
import math

import numpy as np
import pytest

from oracle import efie, mfie, mie
from oracle.rwg import build_rwg
from paper_1408_7060_gb300.inputs import icosphere, make_workload

TH = np.linspace(0.01, np.pi - 0.01, 37)
RH = np.stack([np.sin(TH), 0 * TH, np.cos(TH)], 1)
POL = np.stack([np.cos(TH), 0 * TH, -np.sin(TH)], 1)


def _rcs_errors(sub):
    rwg = build_rwg(*icosphere(sub, 1.0))
    p = efie.Params(dt=1e-9, f_c=150e6)
    KF = mfie.fill_dense(rwg, p, freq=True)
    W = mfie.excitation_fd(rwg, p, [0, 0, 1], [1, 0, 0])
    ZF = efie.fill_dense(rwg, p, freq=True)
    VF = efie.excitation_fd(rwg, p, [0, 0, 1], [1, 0, 0])[0]
    eta = math.sqrt(p.mu / p.eps)
    sm = mie.rcs(p.kc, p.kc, TH, "E")
    out = []
    for I in (np.linalg.solve(KF, W), np.linalg.solve(0.5 * ZF + 0.5 * eta * KF, 0.5 * VF + 0.5 * eta * W)):
        out.append(mie.db_error(efie.rcs_fd(rwg, p, I, RH, POL), sm, np.sin(TH)))
    return out


def test_fd_mfie_and_cfie_converge_to_mie():
    e1, e2 = _rcs_errors(1), _rcs_errors(2)
    for a, b in zip(e1, e2):
        assert b < a and b < 1e-4, (a, b)


@pytest.fixture(scope="module")
def s120():
    w = make_workload("sphere480", band_frac=0.3)
    rwg = build_rwg(*icosphere(1, 1.0))
    p = efie.Params(dt=w.dt, f_c=w.f_c, Q=2)
    return w, rwg, p, mfie.fill_dense(rwg, p)


def test_dc_identity(s120):
    w, rwg, p, K = s120
    KF = mfie.fill_dense(rwg, p, freq=True)
    S = K.sum(0)
    assert np.abs(S - 1j * p.wc * KF).max() < 1e-12 * np.abs(S).max()


def test_first_time_moment(s120):
    w, rwg, p, K = s120
    saved = mfie._kernel_fd
    try:
        mfie._kernel_fd = lambda m, R, p_: ((1 + 1j * p_.kc * R + (p_.kc * R) ** 2) / R ** 2
                                             * np.exp(-1j * p_.kc * R) / (4 * math.pi))[None]
        Kp = mfie.fill_dense(rwg, p, freq=True)
    finally:
        mfie._kernel_fd = saved
    got = np.tensordot(np.arange(K.shape[0], dtype=float), K, axes=(0, 0))
    assert np.abs(got + Kp / p.dt).max() < 1e-12 * np.abs(got).max()


def test_excitation_dc(s120):
    w, rwg, p, K = s120
    W = mfie.excitation(rwg, p, [0, 0, 1], [1, 0, 0], w.sigma, w.t_d, np.arange(-40, 90))
    WF = mfie.excitation_fd(rwg, p, [0, 0, 1], [1, 0, 0])
    lhs = w.dt * W.sum(0)
    rhs = 1j * p.wc * w.sigma * math.sqrt(2 * math.pi) * np.exp(-1j * p.wc * w.t_d) * WF
    assert np.linalg.norm(lhs - rhs) < 1e-12 * np.linalg.norm(rhs)


def test_cfie_march_decays_where_efie_grows():
    """chi = 3 on the 120-RWG sphere (CPPIF Q = 2, beta = 1/4): the EFIE march grows after the
    pulse (the broadband growth of Sec. 3.1.1), the CFIE (alpha = 0.5, Sec. 5.1) march decays
    by more than 15 orders of magnitude over 200 steps."""
    w = make_workload("sphere480", band_frac=0.5)
    rwg = build_rwg(*icosphere(1, 1.0))
    p = efie.Params(dt=w.dt, f_c=w.f_c, Q=2)
    Z = efie.fill_dense(rwg, p)
    K = mfie.fill_dense(rwg, p, n_delays=Z.shape[0] - 1)
    eta = math.sqrt(p.mu / p.eps)
    steps = np.arange(1, 201)
    V = efie.excitation(rwg, p, w.khat, w.phat, w.sigma, w.t_d, steps)[:, 0]
    W = mfie.excitation(rwg, p, w.khat[0], w.phat[0], w.sigma, w.t_d, steps)
    from oracle import march

    ne = np.linalg.norm(march.march_dense(Z, V[:, None])[:, 0], axis=1)
    nc = np.linalg.norm(march.march_dense(0.5 * Z + 0.5 * eta * K, (0.5 * V + 0.5 * eta * W)[:, None])[:, 0], axis=1)
    assert ne[-1] > ne[:60].max()
    assert nc[-1] < 1e-15 * nc.max()
