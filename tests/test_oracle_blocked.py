"""Pins of the oracle's multilevel blocked delay sums (Sec. 4, stage ii): the blocked
schedule gives the direct sums sum_{m=1..N_g} g[m] s[n-m] to rounding for any N_g and
march length (every source/observer pair with a delay 1..N_g lies in exactly one
square), and each square's observers lie at or after the step that forms it."""
import numpy as np
import pytest

from oracle import blocked


@pytest.mark.parametrize("ng,nt", [(1, 9), (2, 17), (3, 40), (6, 64), (7, 100), (16, 70), (31, 130)])
def test_blocked_equals_direct(ng, nt):
    rng = np.random.default_rng(ng * 1000 + nt)
    g = rng.standard_normal((ng + 1, 3)) + 1j * rng.standard_normal((ng + 1, 3))
    s = rng.standard_normal((nt, 3)) + 1j * rng.standard_normal((nt, 3))
    ref = blocked.direct_delay_sums(g, s)
    got = blocked.blocked_delay_sums(g, s)
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


def test_pairs_covered_once_and_causal():
    for ng in (1, 3, 6, 7, 31):
        P = blocked.top_level(ng)
        assert (1 << P) >= ng and (P == 0 or (1 << (P - 1)) < ng)
        nt = 4 * (1 << P) + 3
        cover = np.zeros((nt + 2 * (1 << P), nt), dtype=int)
        for e in range(1, nt + 1):
            b = blocked.square_size(e, P)
            assert e % b == 0
            for i in range(b):
                for j in range(e - b, e):
                    if 1 <= e + i - j <= ng:
                        cover[e + i, j] += 1
        for n in range(nt):
            for j in range(nt):
                assert cover[n, j] == (1 if 1 <= n - j <= ng else 0), (ng, n, j)
