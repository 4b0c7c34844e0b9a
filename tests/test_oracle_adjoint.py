"""Pins of the oracle's far-field objective and its adjoint gradient."""
import math

import numpy as np
import pytest

from oracle import adjoint, efie, march
from oracle.constants import MU0
from oracle.rwg import build_rwg
from paper_1408_7060_gb300.inputs import icosphere


@pytest.fixture(scope="module")
def small():
    V, F = icosphere(1, 1.0)
    rwg = build_rwg(V, F)
    p = efie.Params(dt=1.0 / (4 * 0.1 * 150e6), f_c=150e6, Q=2)
    return rwg, p


def test_constant_envelope_is_time_harmonic(small):
    """a_i = 1 for all i: the CPPIF partition of unity gives e(t) = 1, so the tested
    incident field is the time-harmonic one, V_l = j w_c V^FD (independent code path)."""
    rwg, p = small
    s = list(range(-8, 8))
    B = adjoint.incident_taps(rwg, p, [0, 0, 1.0], [1.0, 0, 0], s)
    a = np.ones(60, dtype=complex)
    V = adjoint.excitation_from_samples(B, s, a, -20, 30)
    VF = efie.excitation_fd(rwg, p, [0, 0, 1.0], [1.0, 0, 0])[0]
    for l in range(1, 30):
        assert np.linalg.norm(V[l - 1] - 1j * p.wc * VF) < 1e-12 * np.linalg.norm(VF) * p.wc


def test_constant_current_far_field(small):
    """I_l = I for all l: sum_s (DT)(s + w) = j w_c, so F = -j w mu/(4 pi) (radiation vector)."""
    rwg, p = small
    rng = np.random.default_rng(0)
    I = rng.standard_normal(rwg.ns) + 1j * rng.standard_normal(rwg.ns)
    rh = np.array([[0.3, -0.4, math.sqrt(1 - 0.25)]])
    e1 = np.cross(rh[0], [0, 0, 1.0])
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(rh[0], e1)
    s = list(range(-8, 8))
    A = adjoint.farfield_taps(rwg, p, rh, e1, e2, s)
    Ih = np.tile(I, (40, 1))
    F = adjoint.farfield(A, s, Ih, [20])[0, 0]
    R = efie.far_field_fd(rwg, p, I, rh)[0]
    ref = -1j * p.wc * MU0 / (4 * math.pi) * np.array([R @ e1, R @ e2])
    assert np.abs(F - ref).max() < 1e-12 * np.abs(ref).max()


def test_gradient_central_differences(small):
    """J is quadratic in a: central differences are exact up to rounding."""
    rwg, p = small
    Z = efie.fill_dense(rwg, p)
    sB = list(range(-6, 6))
    B = adjoint.incident_taps(rwg, p, [0, 0, 1.0], [1.0, 0, 0], sB)
    rh = np.array([[0, 0, -1.0], [1.0, 0, 0]])
    e1 = np.array([[1.0, 0, 0], [0, 1.0, 0]])
    e2 = np.array([[0, 1.0, 0], [0, 0, 1.0]])
    sA = list(range(-6, 6))
    A = adjoint.farfield_taps(rwg, p, rh, e1, e2, sA)
    rng = np.random.default_rng(1)
    n_steps, i0 = 25, -2
    a = rng.standard_normal(20) + 1j * rng.standard_normal(20)
    n_range = list(range(-5, n_steps + 6))
    J, g = adjoint.gradient(Z, B, sB, A, sA, a, i0, n_steps, n_range)

    def Jof(aa):
        V = adjoint.excitation_from_samples(B, sB, aa, i0, n_steps)
        I = march.march_dense(Z, V[:, None, :])[:, 0, :]
        return adjoint.objective(adjoint.farfield(A, sA, I, n_range))

    assert abs(Jof(a) - J) < 1e-12 * J
    for _ in range(4):
        d = rng.standard_normal(20) + 1j * rng.standard_normal(20)
        eps = 1e-3
        fd = (Jof(a + eps * d) - Jof(a - eps * d)) / (2 * eps)
        assert abs(fd - 2 * np.real(np.vdot(g, d))) < 1e-9 * abs(fd) + 1e-12 * J
