"""Host-side analysis of the instability studies (no GPU): the spectral measures used by the time-step
scan (Sec. 5) and by the App. I runs."""
import numpy as np

from paper_1009_2727_gb300 import stability


def test_nyquist_fraction_separates_odd_even_from_smooth_fields():
    k = np.arange(400)
    smooth = np.sin(2 * np.pi * k / 80.0)
    odd_even = np.cos(np.pi * k)
    assert stability.nyquist_fraction(smooth, 10) < 1e-3
    assert stability.nyquist_fraction(odd_even, 10) > 0.99
    mix = smooth + 0.1 * odd_even
    f = stability.nyquist_fraction(mix, 10)
    # one-sided spectrum: the sine's power 1/2 splits over +-k and counts half; the Nyquist bin counts whole:
    # 0.01 / (0.25 + 0.01) = 0.038, up to the window's leakage
    assert 0.03 < f < 0.05
    assert stability.nyquist_fraction(np.zeros(100), 10) == 0.0


def test_high_k_power_splits_at_quarter_nyquist():
    nx, nz = 8, 256
    z = np.arange(nz + 1)
    low = np.tile(np.sin(2 * np.pi * z * 4 / 256.0), (nx + 1, 1))       # k dz = 0.098
    high = np.tile(np.cos(0.9 * np.pi * z), (nx + 1, 1))              # k dz = 0.9 pi
    hk, lk = stability.high_k_power(low, 2)
    assert hk < 1e-3 * lk
    hk, lk = stability.high_k_power(high, 2)
    assert lk < 1e-2 * hk
