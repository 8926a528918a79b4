"""Seeded synthetic PET workloads: system matrix, phantoms, sinograms.

This module only *makes inputs*.  It holds none of the reconstruction
method's arithmetic (no preconditioner, no regulariser, no momentum, no
initial-image rule); the FP64 oracle and the CUDA library both take its
arrays as given.

Data model (Sec. 2.1, Eq. "model-Poisson"): g = Poisson(A f_true + gamma).

Geometry (replaces the paper's 2D ring simulation of Sec. 4.1, whose
area-integral projector is not fully specified): parallel beam, angles
phi_a = a*pi/n_angles, detector bins of width one pixel centred on the
rotation axis, an N x N image of unit pixels centred at the origin.
A_ij = length of ray i inside pixel j (Siddon traversal, computed in FP64,
stored rounded to nearest FP32).  Rays are ordered angle-major
(i = a*n_bins + b); pixels row-major (j = r*N + c, r along +y, c along +x).

Phantoms: random ellipses (a body ellipse inside the inscribed disk plus
5-10 overwriting ellipses, activity U(0, 4)), optional hot lesions at 4:1
over the local background, and the paper's uniform phantom (uniform disk
with six hot disks of radii 4..14 px at 4:1, Sec. 4.1).  Counts: f_true is
scaled so that sum(A f_true + gamma) = C with gamma uniform at 10 % of the
mean projection, then g is drawn with NumPy's PCG64.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np
import scipy.sparse as sp

BASE_SEED = 13344


@dataclasses.dataclass(frozen=True)
class Geometry:
    n: int          # image side N (d = N*N)
    n_angles: int   # number of projection angles (NPA)
    n_bins: int     # detector bins per angle

    @property
    def d(self) -> int:
        return self.n * self.n

    @property
    def m(self) -> int:
        return self.n_angles * self.n_bins


# Named geometries of the reconstruction workloads (image side, angles, bins).
GEOMETRIES = {
    "64": Geometry(64, 90, 95),
    "128": Geometry(128, 90, 185),
    "256": Geometry(256, 180, 367),
    "400": Geometry(400, 288, 575),
    "512": Geometry(512, 360, 731),
}


def seed_for(config: int, slice_index: int = 0) -> int:
    """Seed rule shared by every generator call: 13344 + 1000*config + slice."""
    return BASE_SEED + 1000 * int(config) + int(slice_index)


# --------------------------------------------------------------------------
# System matrix
# --------------------------------------------------------------------------

def _ray_segments(n: int, phi: float, s: np.ndarray):
    """Siddon traversal of the rays {s*nrm + t*u} through the N x N square.

    Returns (ray_index, pixel_index, length) in FP64 for all rays of one
    angle, rays in the order of ``s`` and segments in traversal order.
    """
    h = n / 2.0
    cs, sn = math.cos(phi), math.sin(phi)
    if abs(cs) < 1e-12:
        cs = 0.0
    if abs(sn) < 1e-12:
        sn = 0.0
    x0 = -s * sn  # a point of each ray (t = 0)
    y0 = s * cs
    nb = s.shape[0]
    edges = np.arange(n + 1, dtype=np.float64) - h
    big = np.inf
    # slab entry/exit per axis
    if cs != 0.0:
        tx = (edges[None, :] - x0[:, None]) / cs
        tx_lo = np.minimum(tx[:, 0], tx[:, -1])
        tx_hi = np.maximum(tx[:, 0], tx[:, -1])
    else:
        tx = None
        inside = (x0 >= -h) & (x0 < h)  # half-open: a ray on the +h edge misses
        tx_lo = np.where(inside, -big, big)
        tx_hi = np.where(inside, big, -big)
    if sn != 0.0:
        ty = (edges[None, :] - y0[:, None]) / sn
        ty_lo = np.minimum(ty[:, 0], ty[:, -1])
        ty_hi = np.maximum(ty[:, 0], ty[:, -1])
    else:
        ty = None
        inside = (y0 >= -h) & (y0 < h)
        ty_lo = np.where(inside, -big, big)
        ty_hi = np.where(inside, big, -big)
    t_lo = np.maximum(tx_lo, ty_lo)
    t_hi = np.minimum(tx_hi, ty_hi)
    hit = t_hi > t_lo + 1e-12
    if not np.any(hit):
        return (np.zeros(0, np.int64),) * 2 + (np.zeros(0),)
    rays = np.nonzero(hit)[0]
    t_lo = t_lo[rays]
    t_hi = t_hi[rays]
    parts = [t_lo[:, None], t_hi[:, None]]
    if tx is not None:
        parts.append(tx[rays])
    if ty is not None:
        parts.append(ty[rays])
    t = np.concatenate(parts, axis=1)
    t = np.clip(t, t_lo[:, None], t_hi[:, None])
    t.sort(axis=1)
    seg = np.diff(t, axis=1)
    tm = 0.5 * (t[:, 1:] + t[:, :-1])
    xm = x0[rays][:, None] + tm * cs
    ym = y0[rays][:, None] + tm * sn
    c = np.floor(xm + h).astype(np.int64)
    r = np.floor(ym + h).astype(np.int64)
    keep = seg > 1e-9
    np.clip(c, 0, n - 1, out=c)
    np.clip(r, 0, n - 1, out=r)
    ray_idx = np.broadcast_to(rays[:, None], seg.shape)[keep]
    pix = (r * n + c)[keep]
    return ray_idx, pix, seg[keep]


def siddon_matrix(geom: Geometry) -> sp.csr_matrix:
    """Parallel-beam Siddon system matrix as canonical CSR (sorted columns).

    Values are intersection lengths in pixel units rounded to FP32; indices
    are int32.  Rows of rays that miss the image are empty.  With an even
    number of angles NPA, angle a + NPA/2 is angle a turned a quarter turn:
    its ray at bin nb-1-b is the ray of angle a at bin b turned about the
    image centre, which moves pixel (r, c) to (N-1-c, r).  Those rows are
    built from the traversal of angle a by that turn, so the matrix has the
    scanner's symmetry exactly (traversing them directly differs only by the
    FP64 rounding of the angle's sine and cosine: a few values per thousand
    rows, by a few FP32 units in the last place).
    """
    n, na, nb = geom.n, geom.n_angles, geom.n_bins
    s = np.arange(nb, dtype=np.float64) - (nb - 1) / 2.0
    rows, cols, vals = [], [], []
    half = na // 2 if na % 2 == 0 else na
    for a in range(half):
        ray, pix, seg = _ray_segments(n, a * math.pi / na, s)
        rows.append(ray + a * nb)
        cols.append(pix)
        vals.append(seg)
    if half < na:
        for a in range(half):
            ray = rows[a] - a * nb
            pix = cols[a]
            rows.append((a + half) * nb + (nb - 1 - ray))
            cols.append((n - 1 - pix % n) * n + pix // n)
            vals.append(vals[a])
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    # a ray never visits a pixel twice (convex cells) but merge defensively
    mat = sp.coo_matrix((vals, (rows, cols)), shape=(geom.m, geom.d)).tocsr()
    mat.sum_duplicates()
    mat.sort_indices()
    out = sp.csr_matrix(
        (mat.data.astype(np.float32), mat.indices.astype(np.int32),
         mat.indptr.astype(np.int32)), shape=mat.shape)
    return out


def chord_length(n: int, phi: float, s: np.ndarray) -> np.ndarray:
    """Closed-form length of the line {p : <p, (-sin, cos)> = s} inside the
    square [-N/2, N/2]^2 (the Radon transform of the square's indicator is a
    trapezoid in s).  Used to pin the generator."""
    h = n / 2.0
    c, sn = abs(math.cos(phi)), abs(math.sin(phi))
    s = np.abs(np.asarray(s, dtype=np.float64))
    if c < 1e-12 or sn < 1e-12:
        return np.where(s < h, 2.0 * h, 0.0)
    inner = h * abs(c - sn)
    outer = h * (c + sn)
    plateau = 2.0 * h / max(c, sn)
    ramp = (outer - s) / (c * sn)
    return np.where(s <= inner, plateau, np.where(s < outer, ramp, 0.0))


# --------------------------------------------------------------------------
# Phantoms
# --------------------------------------------------------------------------

def _pixel_centres(n: int):
    h = n / 2.0
    coords = np.arange(n, dtype=np.float64) + 0.5 - h
    x = np.broadcast_to(coords[None, :], (n, n))  # column index -> x
    y = np.broadcast_to(coords[:, None], (n, n))  # row index -> y
    return x, y


def _ellipse_mask(x, y, cx, cy, ax, ay, ang):
    ca, sa = math.cos(ang), math.sin(ang)
    xr = (x - cx) * ca + (y - cy) * sa
    yr = -(x - cx) * sa + (y - cy) * ca
    return (xr / ax) ** 2 + (yr / ay) ** 2 <= 1.0


def ellipse_phantom(n: int, rng: np.random.Generator, lesions: bool) -> np.ndarray:
    """Random-ellipse phantom, FP64 [N*N], unscaled (body activity 1)."""
    x, y = _pixel_centres(n)
    R = n / 2.0
    img = np.zeros((n, n))
    ang = rng.uniform(0.0, math.pi)
    ax = rng.uniform(0.80, 0.95) * R
    ay = rng.uniform(0.60, 0.85) * R
    body = _ellipse_mask(x, y, 0.0, 0.0, ax, ay, ang)
    img[body] = 1.0
    for _ in range(int(rng.integers(5, 11))):
        rad = 0.7 * R * math.sqrt(rng.uniform())
        th = rng.uniform(0.0, 2 * math.pi)
        cx, cy = rad * math.cos(th), rad * math.sin(th)
        ex = rng.uniform(0.05, 0.4) * R
        ey = rng.uniform(0.05, 0.4) * R
        m = _ellipse_mask(x, y, cx, cy, ex, ey, rng.uniform(0.0, math.pi)) & body
        img[m] = rng.uniform(0.0, 4.0)
    if lesions:
        for _ in range(int(rng.integers(3, 7))):
            rad = 0.6 * R * math.sqrt(rng.uniform())
            th = rng.uniform(0.0, 2 * math.pi)
            cx, cy = rad * math.cos(th), rad * math.sin(th)
            pr = rng.uniform(2.0, 6.0)
            m = ((x - cx) ** 2 + (y - cy) ** 2 <= pr * pr) & body
            ci = min(max(int(math.floor(cy + R)), 0), n - 1)
            cj = min(max(int(math.floor(cx + R)), 0), n - 1)
            bg = img[ci, cj] if img[ci, cj] > 0 else 1.0
            img[m] = 4.0 * bg
    return img.reshape(-1)


def uniform_phantom(n: int) -> np.ndarray:
    """Uniform disk with six hot disks of radii 4,6,8,10,12,14 px at 4:1
    (Sec. 4.1), radii scaled with N/256.  FP64 [N*N], background 1."""
    x, y = _pixel_centres(n)
    R = n / 2.0
    img = np.zeros((n, n))
    img[x ** 2 + y ** 2 <= (0.85 * R) ** 2] = 1.0
    scale = n / 256.0
    for k, rad in enumerate((4, 6, 8, 10, 12, 14)):
        th = 2 * math.pi * k / 6.0
        cx, cy = 0.5 * R * math.cos(th), 0.5 * R * math.sin(th)
        rr = max(rad * scale, 1.0)
        img[(x - cx) ** 2 + (y - cy) ** 2 <= rr * rr] = 4.0
    return img.reshape(-1)


# --------------------------------------------------------------------------
# Sinograms
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Slice:
    f_true: np.ndarray   # FP64 [d]
    g: np.ndarray        # FP32 [m] Poisson counts
    gamma: np.ndarray    # FP32 [m] background mean (uniform)
    counts: float        # total expected counts C


def make_slice(A: sp.csr_matrix, geom: Geometry, counts: float, seed: int,
               phantom: str = "ellipses") -> Slice:
    """One seeded slice: phantom -> scaled so sum(A f + gamma) = counts,
    gamma = 10 % of the mean projection, g ~ Poisson(A f + gamma)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if phantom == "ellipses":
        f = ellipse_phantom(geom.n, rng, lesions=False)
    elif phantom == "lesions":
        f = ellipse_phantom(geom.n, rng, lesions=True)
    elif phantom == "uniform":
        f = uniform_phantom(geom.n)
    else:
        raise ValueError(f"unknown phantom {phantom!r}")
    A64 = A.astype(np.float64)
    proj = A64 @ f
    f = f * (counts / (1.1 * proj.sum()))
    proj = A64 @ f
    gamma = np.full(geom.m, 0.1 * proj.mean())
    g = rng.poisson(proj + gamma).astype(np.float32)
    return Slice(f_true=f, g=g, gamma=gamma.astype(np.float32), counts=float(counts))


def ellipsoid_volume(n: int, nz: int, rng: np.random.Generator) -> np.ndarray:
    """Random-ellipsoid volume, FP64 [nz, N*N], unscaled (body activity 1):
    a body ellipsoid that every slice cuts (z semi-axis longer than half the
    stack), 5-10 inner ellipsoids with activity U(0, 4), slice thickness one
    pixel."""
    x, y = _pixel_centres(n)
    R = n / 2.0
    zc = np.arange(nz, dtype=np.float64) + 0.5 - nz / 2.0
    vol = np.zeros((nz, n, n))

    def ellipsoid(cx, cy, cz, ax, ay, az, ang):
        ca, sa = math.cos(ang), math.sin(ang)
        xr = (x - cx) * ca + (y - cy) * sa
        yr = -(x - cx) * sa + (y - cy) * ca
        inplane = (xr / ax) ** 2 + (yr / ay) ** 2
        return inplane[None, :, :] + ((zc - cz) / az)[:, None, None] ** 2 <= 1.0

    body = ellipsoid(0.0, 0.0, 0.0, rng.uniform(0.80, 0.95) * R, rng.uniform(0.60, 0.85) * R,
                     rng.uniform(0.6, 1.0) * nz + 1.0, rng.uniform(0.0, math.pi))
    vol[body] = 1.0
    for _ in range(int(rng.integers(5, 11))):
        rad = 0.7 * R * math.sqrt(rng.uniform())
        th = rng.uniform(0.0, 2 * math.pi)
        m = ellipsoid(rad * math.cos(th), rad * math.sin(th), rng.uniform(-0.4, 0.4) * nz,
                      rng.uniform(0.05, 0.4) * R, rng.uniform(0.05, 0.4) * R,
                      rng.uniform(0.1, 0.5) * nz + 1.0, rng.uniform(0.0, math.pi)) & body
        vol[m] = rng.uniform(0.0, 4.0)
    return vol.reshape(nz, n * n)


@dataclasses.dataclass
class Volume:
    f_true: np.ndarray   # FP64 [nz, d]
    g: np.ndarray        # FP32 [nz, m] Poisson counts, slice by slice
    gamma: np.ndarray    # FP32 [nz, m] background mean (uniform over the volume)
    counts: float        # total expected counts over the volume


def make_volume(A: sp.csr_matrix, geom: Geometry, nz: int, counts: float, seed: int) -> Volume:
    """One seeded volume of nz slices sharing A: ellipsoid phantom scaled so
    the volume's expected counts are `counts`, gamma = 10 % of the mean
    projection over the volume, g_z ~ Poisson(A f_z + gamma) per slice."""
    rng = np.random.Generator(np.random.PCG64(seed))
    f = ellipsoid_volume(geom.n, nz, rng)
    A64 = A.astype(np.float64)
    proj = (A64 @ f.T).T
    f = f * (counts / (1.1 * proj.sum()))
    proj = (A64 @ f.T).T
    gamma = np.full((nz, geom.m), 0.1 * proj.mean())
    g = rng.poisson(proj + gamma).astype(np.float32)
    return Volume(f_true=f, g=g, gamma=gamma.astype(np.float32), counts=float(counts))


def log_uniform_counts(rng: np.random.Generator, lo: float, hi: float, k: int) -> np.ndarray:
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=k))


# --------------------------------------------------------------------------
# Small dense problems (for brute-force checks)
# --------------------------------------------------------------------------

def dense_problem(n: int, m: int, seed: int, counts: float = 2e3):
    """Small full-column-rank problem with a dense positive A (m x n*n)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = n * n
    A = rng.uniform(0.05, 1.0, size=(m, d))
    A = A.astype(np.float32).astype(np.float64)
    f = rng.uniform(0.2, 1.0, size=d)
    proj = A @ f
    f *= counts / (1.1 * proj.sum())
    proj = A @ f
    gamma = np.full(m, 0.1 * proj.mean())
    g = rng.poisson(proj + gamma).astype(np.float64)
    return A, f, g, gamma


_MATRIX_CACHE: dict = {}


def system_matrix(name: str) -> sp.csr_matrix:
    """Memoised Siddon matrix of a named geometry."""
    if name not in _MATRIX_CACHE:
        _MATRIX_CACHE[name] = siddon_matrix(GEOMETRIES[name])
    return _MATRIX_CACHE[name]
