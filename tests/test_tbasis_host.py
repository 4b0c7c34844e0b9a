"""The library's temporal basis on the host (aim_time_factor, no GPU): the time factors its
setup kernels tabulate Z_m with -- the CPPIF of Eq. 3 and the extrapolated BLIF of Sec. 3.1.2,
values and three derivatives -- against the oracle, and its argument checks."""
import numpy as np
import pytest

from oracle import blif, tbasis


@pytest.mark.parametrize("M,beta", [(3, 0.25), (3, 1 / 15), (2, 0.3), (5, 0.1), (4, 0.02)])
def test_blif_time_factors_match_oracle(M, beta):
    from paper_1408_7060_gb300 import abi

    rng = np.random.default_rng(11)
    E = blif.extrapolation(M, beta)
    for m in range(M + 3):
        x = np.concatenate([rng.uniform(0.0, M + m + 1, 300), [0.0, 1e-9, float(m), float(m + M)]])
        got = abi.aim_time_factor(m, x, "blif", M, beta)
        for d in range(4):
            ref = blif.T_eff(m, m - x, M, beta, E, d)
            # the extrapolation weights' conditioning grows as the band narrows (beta = 0.02)
            tol = 1e-12 if beta > 0.05 else 2e-12
            assert np.abs(got[:, d] - ref).max() <= tol * max(1.0, np.abs(ref).max()), (m, d)


@pytest.mark.parametrize("Q", [1, 2, 3, 4])
def test_cppif_time_factors_match_oracle(Q):
    from paper_1408_7060_gb300 import abi

    x = np.random.default_rng(12).uniform(0.0, 9.0, 400)
    for m in range(7):
        got = abi.aim_time_factor(m, x, "cppif", Q)
        for d in range(4):
            ref = tbasis.T(m - x, Q, d)
            assert np.abs(got[:, d] - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max()), (m, d)


def test_arguments_rejected():
    from paper_1408_7060_gb300 import abi

    for kw in (dict(basis="blif", order=3, blif_band=0.5), dict(basis="blif", order=6, blif_band=0.2),
               dict(basis="blif", order=1, blif_band=0.2), dict(basis="cppif", order=5)):
        with pytest.raises(abi.AimError):
            abi.aim_time_factor(0, [0.5], **kw)
    with pytest.raises(abi.AimError):
        abi.aim_time_factor(-1, [0.5])
