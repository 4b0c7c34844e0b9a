"""Multilevel blocked evaluation of the delayed sums of the right-hand side (Sec. 4,
stage ii; the blocked space-time FFT scheme the paper takes from TD-AIM).

Test infrastructure: only the tests, the smoke check and the benchmark's CPU baseline use it.

The right-hand side of Eq. 5 needs, at every step n (0-based) and at every point of the
grid's spatial spectrum, the temporal convolution

    y[n] = sum_{m=1..N_g} g[m] s[n - m]

of the source spectra s with the kernel spectra g.  Stage ii radiates the sources "at
the present and some of the future time steps": after the sample s[e-1] is known, the
block of the last b sources s[e-b .. e-1] is convolved at once with the kernel and its
contributions to the next b observers y[e .. e+b-1] are added to them.  Reading of the
schedule (the paper defers it to its reference [2]): the strictly lower triangle of
source/observer pairs is tiled by squares; a pair (n', n) inside one top block of
B = 2^P >= N_g steps belongs to the square of the highest bit p in which n' and n differ
(b = 2^p sources below the boundary e, b observers from e), and a pair of adjacent top
blocks to the square of size B at their boundary; pairs further apart have delays above
N_g.  So the square formed after s[e-1] has size b = 2^min(ctz(e), P).  Each square is
one linear convolution of b samples with the taps g[1 .. 2b-1], done by temporal FFTs of
length 2b (no wrap-around reaches the b outputs kept); over a march this costs O(log^2 N_g)
per step and spatial point instead of the N_g of the direct sum.
"""
from __future__ import annotations

import numpy as np


def direct_delay_sums(g: np.ndarray, s: np.ndarray) -> np.ndarray:
    """y[n] = sum_{m=1..N_g} g[m] s[n-m] (s[n] = 0 for n < 0); g: [N_g + 1, ...] (g[0]
    unused), s: [N_t, ...] -> y: [N_t, ...]."""
    ng = len(g) - 1
    y = np.zeros(s.shape, dtype=complex)
    for n in range(len(s)):
        for m in range(1, ng + 1):
            if n - m >= 0:
                y[n] += g[m] * s[n - m]
    return y


def top_level(ng: int) -> int:
    """P with 2^P the smallest power of two >= N_g."""
    P = 0
    while (1 << P) < ng:
        P += 1
    return P


def square_size(e: int, P: int) -> int:
    """Size b of the square formed once e samples are known (e >= 1)."""
    p = 0
    while p < P and (e >> p) & 1 == 0:
        p += 1
    return 1 << p


def blocked_delay_sums(g: np.ndarray, s: np.ndarray) -> np.ndarray:
    """The same sums by the multilevel blocked schedule, in march order: y[n] is complete
    before s[n] is used (the observers of every square lie at or after its boundary)."""
    ng = len(g) - 1
    nt = len(s)
    P = top_level(ng)
    y = np.zeros((nt + 2 * (1 << P),) + s.shape[1:], dtype=complex)
    for e in range(1, nt + 1):          # s[e-1] has just been solved
        b = square_size(e, P)
        h = np.zeros((2 * b,) + g.shape[1:], dtype=complex)  # taps g[1 .. 2b-1]
        k = np.arange(1, min(2 * b - 1, ng) + 1)
        h[k] = g[k]
        a = np.zeros((2 * b,) + s.shape[1:], dtype=complex)
        a[:b] = s[e - b:e]              # b divides e, so e >= b
        c = np.fft.ifft(np.fft.fft(a, axis=0) * np.fft.fft(h, axis=0), axis=0)
        y[e:e + b] += c[b:2 * b]
    return y[:nt]
