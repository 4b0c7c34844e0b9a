"""The RCS pipeline of Sec. 2.4 on the GPU (aim_march_spectrum, aim_rcs) against the
oracle, and the RCS of the complex64 ET-AIM march against the Mie series in the
dB-error norm of Eq. 2.

* aim_march_spectrum on the 480-RWG sphere (complex128, 150 MHz +-5 %): the frequency-
  domain currents at f_c and f_c +- f_bw/2 equal the oracle's transform of its own
  ET-AIM march (dense LU of the AIM operator) within the march's solver tolerance, and
  the transform of the library's aim_march currents of the same march to rounding;
* aim_rcs of those currents equals the oracle's frequency-domain far field to rounding;
* the 7680-RWG sphere (complex64 grid path, FP64 refinement, 600 MHz +-30 %): the RCS
  of the march over the whole sphere of directions agrees with the Mie series at f_c and
  f_c +- f_bw/2 within the dB-error bound 1e-2.
"""
import math

import numpy as np
import pytest

from oracle import aim as oaim
from oracle import efie, march, mie, rcs
from oracle.rwg import build_rwg
from paper_1408_7060_gb300.inputs import make_workload

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b))


@pytest.fixture(scope="module")
def s480_narrow():
    w = make_workload("sphere480", band_frac=0.05, n_t=60)
    rwg = build_rwg(*w.mesh)
    p = efie.Params(dt=w.dt, f_c=w.f_c, Q=w.order)
    A = oaim.AimOracle(rwg, w.grid_n, w.h, w.origin, w.near_radius, p)
    ZA = np.stack([A.dense(m) for m in range(A.n_delays + 1)])
    V = efie.excitation(rwg, p, w.khat, w.phat, w.sigma, w.t_d, np.arange(1, w.n_t + 1))
    I_ref = march.march_dense(ZA, V)[:, 0]
    freqs = np.array([w.f_c, w.f_c + 0.5 * w.f_bw, w.f_c - 0.5 * w.f_bw])
    return w, rwg, p, I_ref, freqs


def oracle_spec(w, p, I, freqs):
    out = []
    for f in freqs:
        Om = 2 * math.pi * (f - w.f_c)
        out.append(rcs.envelope_spectrum(I, p.dt, p.Q, Om) / rcs.incident_spectrum(w.sigma, w.t_d, w.f_c, Om))
    return np.array(out)


def test_march_spectrum_vs_oracle(s480_narrow):
    from paper_1408_7060_gb300 import AimContext

    w, rwg, p, I_ref, freqs = s480_narrow
    with AimContext.from_workload(w, precision="c128") as c:
        spec, st, rc = c.march_spectrum(w.khat, w.phat, w.sigma, w.t_d, w.n_t, 1e-10, freqs)
        cur, _, _ = c.march(w.khat, w.phat, w.sigma, w.t_d, w.n_t, 1e-10)
    assert st["last_step"] == w.n_t and spec.shape == (3, 1, rwg.ns)
    ref = oracle_spec(w, p, I_ref, freqs)
    mine = oracle_spec(w, p, cur[:, 0], freqs)
    for i in range(len(freqs)):
        assert rel(spec[i, 0], mine[i]) < 1e-12, i   # the same march, transformed
        assert rel(spec[i, 0], ref[i]) < 1e-7, i     # the oracle's march (LU)


def test_rcs_vs_oracle_far_field(s480_narrow):
    from paper_1408_7060_gb300 import AimContext
    from paper_1408_7060_gb300.rcs import sphere_grid

    w, rwg, p, I_ref, freqs = s480_narrow
    spec = oracle_spec(w, p, I_ref, freqs)[:, None, :]
    rh, eth, wt, th, ph = sphere_grid(8, 10)
    eph = np.cross(rh, eth)
    with AimContext.from_workload(w, precision="c128") as c:
        s_th = c.rcs(freqs, spec, rh, eth)
        s_ph = c.rcs(freqs, spec, rh, eph)
    for i, f in enumerate(freqs):
        pf = efie.Params(dt=p.dt, f_c=f, Q=p.Q)
        for got, pol in ((s_th, eth), (s_ph, eph)):
            ref = efie.rcs_fd(rwg, pf, spec[i, 0], rh, pol)
            assert np.abs(got[i, 0] - ref).max() < 1e-11 * ref.max(), (i, f)


def test_sphere7680_rcs_vs_mie():
    from paper_1408_7060_gb300 import AimContext
    from paper_1408_7060_gb300.rcs import sphere_grid

    w = make_workload("sphere7680", precond="sai", refine=4)
    w.precond_radius = 2.5 * w.near_radius
    n_t = int(2 * w.t_d / w.dt) + 40
    freqs = np.array([w.f_c, w.f_c + 0.5 * w.f_bw, w.f_c - 0.5 * w.f_bw])
    rh, eth, wt, th, ph = sphere_grid(24, 24)
    with AimContext.from_workload(w) as c:
        spec, st, rc = c.march_spectrum(w.khat, w.phat, w.sigma, w.t_d, n_t, w.tol, freqs)
        sig = c.rcs(freqs, spec, rh, eth)
    assert st["last_step"] == n_t
    errs = []
    for i, f in enumerate(freqs):
        k = 2 * math.pi * f / 299792458.0
        s_mie = mie.rcs(k, k, th, "E") * np.cos(ph) ** 2
        errs.append(mie.db_error(sig[i, 0], s_mie, wt))
    print("7680-RWG sphere, RCS dB error of Eq. 2 vs Mie at f_c, f_c + f_bw/2, f_c - f_bw/2:",
          " ".join(f"{e:.2e}" for e in errs))
    assert max(errs) < 1e-2
