"""The ring-fraction statistic of the long-run tests (tests/golden/
make_longrun.py): the spectral power of a field split over Chebyshev rings
max(|mx|, |my|) = 0, [1, 2), [2, 4), ... of doubling radius."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))
from make_longrun import ring_fractions  # noqa: E402


def test_a_plane_wave_puts_all_its_power_in_its_ring():
    n = 64
    x = np.arange(n)
    for (mx, my), ring in [((0, 0), 0), ((1, 0), 1), ((0, -1), 1), ((3, -2), 2), ((-7, 5), 3), ((12, 31), 5),
                           ((-32, 0), 5), ((16, -16), 5), ((8, 0), 4)]:
        E = np.exp(2j * np.pi * (mx * x[None, :] + my * x[:, None]) / n)
        f = ring_fractions(np.abs(np.fft.fft2(E)) ** 2)
        assert len(f) == 6                               # DC and rings up to [16, 32]
        assert abs(f[ring] - 1.0) < 1e-12 and abs(sum(f) - 1.0) < 1e-12, ((mx, my), f)


def test_fractions_sum_to_one_and_follow_the_ring_areas_for_white_noise():
    n = 256
    S = np.ones((n, n))
    f = ring_fractions(S)
    assert abs(sum(f) - 1.0) < 1e-12
    # bins with max(|m|) = r number 8r for r >= 1 (signed frequencies -n/2..n/2-1; n/2 appears once per axis)
    counts = np.zeros(len(f))
    m = np.abs(np.fft.fftfreq(n, 1.0 / n)).astype(int)
    rho = np.maximum(m[:, None], m[None, :])
    counts[0] = 1
    for k in range(1, len(f)):
        lo, hi = 2 ** (k - 1), 2 ** k
        counts[k] = np.count_nonzero((rho >= lo) & ((rho < hi) if k < len(f) - 1 else (rho <= n // 2)))
    assert counts.sum() == n * n
    assert np.allclose(f, counts / (n * n), rtol=0, atol=1e-15)
