"""FP64 CPU oracle of the figures of merit used to compare reconstructions
(Sec. 4.1): NOFV, PSNR, NRC and the central line profile.

TEST INFRASTRUCTURE ONLY, like the rest of this package: only the tests,
the package smoke check and the benchmark's CPU-baseline leg may import it.

Definitions, restated from the paper:

* NOFV(f^k) = (Phi(f^k) - Phi_ref) / (Phi_0 - Phi_ref), with Phi_0 the
  objective of the initial image and Phi_ref a reference objective value.
* MSE(f^k) = ||f^k - f_true||^2 / d and PSNR = 10 log10(MAX^2 / MSE), MAX the
  largest possible pixel value.
* RC = |E_H - E_B| / E_B with E_H, E_B the mean activities over a hot region
  ROI_H and a background region ROI_B; NRC(f^k) = RC(f^k) / RC(f_true).
* CLP: the pixel values along the central line of the image.

Readings where the paper leaves a choice open: MAX is an input (the caller
decides the largest possible value, e.g. the maximum of the ground truth);
the central line is image row floor(N/2) of the row-major image; the ROIs
are given as boolean masks of equal size.
"""
from __future__ import annotations

import math

import numpy as np


def nofv(phi_k: float, phi_0: float, phi_ref: float) -> float:
    return (float(phi_k) - float(phi_ref)) / (float(phi_0) - float(phi_ref))


def mse(f: np.ndarray, f_true: np.ndarray) -> float:
    e = np.asarray(f, np.float64) - np.asarray(f_true, np.float64)
    return float(np.dot(e, e) / e.size)


def psnr(f: np.ndarray, f_true: np.ndarray, max_value: float) -> float:
    return 10.0 * math.log10(float(max_value) ** 2 / mse(f, f_true))


def relative_contrast(f: np.ndarray, roi_h: np.ndarray, roi_b: np.ndarray) -> float:
    f = np.asarray(f, np.float64)
    e_h = float(f[np.asarray(roi_h, bool)].mean())
    e_b = float(f[np.asarray(roi_b, bool)].mean())
    return abs(e_h - e_b) / e_b


def nrc(f: np.ndarray, f_true: np.ndarray, roi_h: np.ndarray, roi_b: np.ndarray) -> float:
    return relative_contrast(f, roi_h, roi_b) / relative_contrast(f_true, roi_h, roi_b)


def central_line_profile(f: np.ndarray, n: int) -> np.ndarray:
    return np.asarray(f, np.float64).reshape(n, n)[n // 2].copy()


def disk_roi(n: int, cx: float, cy: float, r: float) -> np.ndarray:
    """Pixels whose centres lie within radius r of (cx, cy) (pixel units,
    origin at the image centre, x along columns, y along rows)."""
    c = np.arange(n, dtype=np.float64) + 0.5 - n / 2.0
    x = c[None, :]
    y = c[:, None]
    return (((x - cx) ** 2 + (y - cy) ** 2) <= r * r).reshape(-1)
