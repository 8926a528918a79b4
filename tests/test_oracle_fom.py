"""Pins of the figures-of-merit oracle (Sec. 4.1) against hand values and
closed forms."""
import math

import numpy as np
import pytest

from oracle import figures_of_merit as F


def test_nofv_endpoints_and_midpoint():
    assert F.nofv(7.0, 7.0, 3.0) == 1.0
    assert F.nofv(3.0, 7.0, 3.0) == 0.0
    assert F.nofv(5.0, 7.0, 3.0) == 0.5


def test_psnr_hand_value():
    f = np.array([1.0, 2.0, 3.0, 4.0])
    t = np.array([1.0, 2.0, 3.0, 6.0])
    assert F.mse(f, t) == 1.0                    # (4 - 6)^2 / 4
    assert F.psnr(f, t, 10.0) == pytest.approx(20.0, abs=1e-12)


def test_psnr_of_constant_offset():
    rng = np.random.default_rng(0)
    t = rng.uniform(0, 4, 1000)
    for c in (0.5, 0.01):
        assert F.psnr(t + c, t, 4.0) == pytest.approx(20 * math.log10(4.0 / c), rel=1e-12)


def test_relative_contrast_hand_value_and_invariances():
    f = np.array([3.0, 3.0, 1.0, 1.0, 9.0])
    h = np.array([1, 1, 0, 0, 0], bool)
    b = np.array([0, 0, 1, 1, 0], bool)
    assert F.relative_contrast(f, h, b) == 2.0   # |3 - 1| / 1
    assert F.relative_contrast(5.0 * f, h, b) == pytest.approx(2.0, rel=1e-15)
    assert F.relative_contrast(f + 1.0, h, b) == pytest.approx(1.0, rel=1e-15)  # |4-2|/2
    assert F.nrc(f, f, h, b) == 1.0
    assert F.nrc(f + 1.0, f, h, b) == pytest.approx(0.5, rel=1e-15)


def test_central_line_profile_of_ramp():
    n = 6
    f = np.arange(n * n, dtype=np.float64)
    assert np.array_equal(F.central_line_profile(f, n), np.arange(3 * n, 4 * n))


def test_disk_roi_area_and_symmetry():
    n = 256
    m = F.disk_roi(n, 0.0, 0.0, 40.0).reshape(n, n)
    assert abs(m.sum() - math.pi * 40 ** 2) < 4 * 40       # lattice points in a disk
    assert np.array_equal(m, m[::-1, :]) and np.array_equal(m, m[:, ::-1])
    off = F.disk_roi(n, 30.0, -20.0, 5.0).reshape(n, n)
    r, c = np.nonzero(off)
    assert abs((c + 0.5 - n / 2).mean() - 30.0) < 1e-9 and abs((r + 0.5 - n / 2).mean() + 20.0) < 1e-9
