"""Pins of the homogeneous background medium (Sec. 2.1: relative permittivity eps_r and
permeability mu_r; light speed c0/n, n = sqrt(eps_r mu_r)).

Exact scaling laws, from the definitions of Eq. 1 and Eq. 4:
* Z_m(medium; dt, f_c) = Z_m(vacuum; dt/n, n f_c) / eps_r for every delay m (the time
  factors see R/(c dt) and k R unchanged, D^2 T scales by n^2 and mu/(4 pi) by mu_r, the
  scalar term by 1/eps_r), the same for the AIM operator;
* V_l(medium; sigma, t_d, dt, f_c) = V_l(vacuum; sigma/n, t_d/n, dt/n, n f_c) / n;
* the frequency-domain EFIE matrix Z(medium, w) = sqrt(mu_r/eps_r) Z(vacuum, n w).
"""
import math

import numpy as np
import pytest

from oracle import aim as oaim
from oracle import efie
from oracle.rwg import build_rwg
from paper_1408_7060_gb300.inputs import icosphere, make_workload

EPS_R, MU_R = 2.25, 1.7
NIDX = math.sqrt(EPS_R * MU_R)


@pytest.fixture(scope="module")
def s480():
    """The 480-RWG sphere's pulse and grid on the 120-RWG icosphere (sub 1)."""
    w = make_workload("sphere480", band_frac=0.2)
    w.mesh = icosphere(1, 1.0)
    return w, build_rwg(*w.mesh)


def test_impedance_matrices_scale(s480):
    w, rwg = s480
    pm = efie.Params(dt=w.dt, f_c=w.f_c, Q=2, eps_r=EPS_R, mu_r=MU_R)
    pv = efie.Params(dt=w.dt / NIDX, f_c=w.f_c * NIDX, Q=2)
    Zm, Zv = efie.fill_dense(rwg, pm), efie.fill_dense(rwg, pv)
    assert Zm.shape == Zv.shape
    assert np.abs(Zm - Zv / EPS_R).max() < 1e-12 * np.abs(Zm).max()
    Fm = efie.fill_dense(rwg, pm, freq=True)
    Fv = efie.fill_dense(rwg, efie.Params(dt=w.dt, f_c=w.f_c * NIDX), freq=True)
    assert np.abs(Fm - math.sqrt(MU_R / EPS_R) * Fv).max() < 1e-12 * np.abs(Fm).max()


def test_excitation_scales(s480):
    w, rwg = s480
    steps = np.arange(1, 40)
    pm = efie.Params(dt=w.dt, f_c=w.f_c, Q=2, eps_r=EPS_R, mu_r=MU_R)
    pv = efie.Params(dt=w.dt / NIDX, f_c=w.f_c * NIDX, Q=2)
    Vm = efie.excitation(rwg, pm, w.khat, w.phat, w.sigma, w.t_d, steps)
    Vv = efie.excitation(rwg, pv, w.khat, w.phat, w.sigma / NIDX, w.t_d / NIDX, steps)
    assert np.abs(Vm - Vv / NIDX).max() < 1e-12 * np.abs(Vm).max()


def test_aim_operator_scales(s480):
    w, rwg = s480
    pm = efie.Params(dt=w.dt, f_c=w.f_c, Q=2, eps_r=EPS_R, mu_r=MU_R)
    pv = efie.Params(dt=w.dt / NIDX, f_c=w.f_c * NIDX, Q=2)
    Am = oaim.AimOracle(rwg, w.grid_n, w.h, w.origin, w.near_radius, pm)
    Av = oaim.AimOracle(rwg, w.grid_n, w.h, w.origin, w.near_radius, pv)
    assert Am.n_delays == Av.n_delays
    for m in (0, 1, Am.n_delays):
        D = Am.dense(m)
        assert np.abs(D - Av.dense(m) / EPS_R).max() < 1e-11 * np.abs(D).max(), m
