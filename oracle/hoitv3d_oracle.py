"""FP64 CPU oracle of the 3-D SHOITV regulariser and of APPGA on a volume.

TEST INFRASTRUCTURE ONLY.  Only the test suite and the CPU-baseline legs of
the benchmark may import this module.  The product path (the CUDA library
and its binding) never imports, links or calls it, and this module imports
nothing from the product path.

The paper writes HOITV out in 2-D only (Sec. 2.1) and leaves the 3-D form to
other work.  This module takes the Kronecker generalisation of the paper's
2-D operators as its reading (also listed in the design notes):

* A volume of Nz slices of N x N pixels is vectorised slice by slice,
  j = z N^2 + r N + c, and D is the paper's backward difference matrix of the
  size of each axis (row 1 zero).
* Axis differences: Dc = I_Nz (x) I_N (x) D_N, Dr = I_Nz (x) D_N (x) I_N,
  Dz = D_Nz (x) I_N (x) I_N.
* B1 = [Dc ; Dr ; Dz]: three first-order components per voxel.
* B2: the paper's four 2-D blocks -Dc^T Dc, -Dr^T Dc, -Dr^T Dr, -Dr Dc^T
  (that is I (x) (-D^T D), (-D^T) (x) D, (-D^T D) (x) I and D (x) (-D^T) in
  each slice), then -Dz^T Dz and, for the two pairs (z, c) and (z, r), the
  same two mixed forms -Dz^T Dc, -Dz Dc^T, -Dz^T Dr, -Dz Dr^T: nine
  second-order components per voxel.
* phi~1 = lambda1 sum over voxels of s_eps(3-vector), phi~2 = lambda2 sum of
  s_eps(9-vector) (Eq. def:smoothL2 on the larger groups).

With Nz = 1 every z-term vanishes (D_1 = 0), so the regulariser is the 2-D
one of each slice; the set of components is closed under permuting the axes.
Both facts are checked in the tests against the independently pinned 2-D
oracle and by transposing volumes.

The volume problem: every slice z has its own sinogram g_z and background
gamma_z and the same system matrix A, so F(f) = sum_z F(f_z) (Eq.
FidelityTerm per slice); APPGA (Eq. APPGAiter with the EM preconditioner of
Eq. EM) runs on the whole volume with one momentum sequence and one stopping
test on the volume's objective.
"""
from __future__ import annotations

import math
from typing import List, Optional

import numpy as np
import scipy.sparse as sp

from oracle.appga_oracle import (KAPPA, Params, Result, difference_matrix, grad_s_eps,
                                 initial_image, s_eps, thetas_for)

N1, N2 = 3, 9  # components of the first- and second-order groups


# --------------------------------------------------------------------------
# 3-D difference operators
# --------------------------------------------------------------------------

def axis_differences(nz: int, nr: int, nc: Optional[int] = None):
    """Dc, Dr, Dz for a volume of nz slices of nr x nc pixels (nc = nr when
    not given; the solver's volumes are square in-plane, rectangular boxes
    serve the sampled checks)."""
    nc = nr if nc is None else nc
    I = lambda k: sp.identity(k, format="csr", dtype=np.float64)
    Dc = sp.kron(sp.kron(I(nz), I(nr)), difference_matrix(nc)).tocsr()
    Dr = sp.kron(sp.kron(I(nz), difference_matrix(nr)), I(nc)).tocsr()
    Dz = sp.kron(sp.kron(difference_matrix(nz), I(nr)), I(nc)).tocsr()
    return Dc, Dr, Dz


def b1_matrix3(nz: int, nr: int, nc: Optional[int] = None) -> sp.csr_matrix:
    """B1 = [Dc ; Dr ; Dz]  (3 dv x dv)."""
    Dc, Dr, Dz = axis_differences(nz, nr, nc)
    return sp.vstack([Dc, Dr, Dz]).tocsr()


def b2_matrix3(nz: int, nr: int, nc: Optional[int] = None) -> sp.csr_matrix:
    """The nine second-order blocks (9 dv x dv), in the order listed above."""
    Dc, Dr, Dz = axis_differences(nz, nr, nc)
    Dct, Drt, Dzt = Dc.T.tocsr(), Dr.T.tocsr(), Dz.T.tocsr()
    blocks = [-(Dct @ Dc), -(Drt @ Dc), -(Drt @ Dr), -(Dr @ Dct),
              -(Dzt @ Dz), -(Dzt @ Dc), -(Dz @ Dct), -(Dzt @ Dr), -(Dz @ Drt)]
    return sp.vstack(blocks).tocsr()


def b_matrix3(nz: int, nr: int, nc: Optional[int] = None) -> sp.csr_matrix:
    """B = [B1 ; B2]  (12 dv x dv)."""
    return sp.vstack([b1_matrix3(nz, nr, nc), b2_matrix3(nz, nr, nc)]).tocsr()


# --------------------------------------------------------------------------
# Regulariser on the 3- and 9-component groups
# --------------------------------------------------------------------------

def _groups3(u: np.ndarray, dv: int):
    u1 = np.stack([u[q * dv:(q + 1) * dv] for q in range(N1)], axis=1)
    u2 = np.stack([u[(N1 + q) * dv:(N1 + q + 1) * dv] for q in range(N2)], axis=1)
    return u1, u2


def phi_tilde3(u: np.ndarray, dv: int, lam1: float, lam2: float, eps: float) -> float:
    """lam1 sum_voxels s_eps(first-order triple) + lam2 sum s_eps(second-order 9-vector)."""
    u1, u2 = _groups3(u, dv)
    return lam1 * float(np.sum(s_eps(u1, eps))) + lam2 * float(np.sum(s_eps(u2, eps)))


def grad_phi_tilde3(u: np.ndarray, dv: int, lam1: float, lam2: float, eps: float) -> np.ndarray:
    """Gradient of phi~ at u: lam * x / max(group norm, eps), group by group."""
    u1, u2 = _groups3(u, dv)
    v1 = lam1 * grad_s_eps(u1, eps)
    v2 = lam2 * grad_s_eps(u2, eps)
    return np.concatenate([v1[:, q] for q in range(N1)] + [v2[:, q] for q in range(N2)])


class Regulariser3D:
    """phi~(B f) and B^T grad phi~(B f) for volumes of nz x nr x nc
    (nc = nr when not given)."""

    def __init__(self, nz: int, nr: int, nc: Optional[int] = None):
        self.nz, self.nr = int(nz), int(nr)
        self.nc = self.nr if nc is None else int(nc)
        self.dv = self.nz * self.nr * self.nc
        self.B = b_matrix3(self.nz, self.nr, self.nc)
        self.Bt = self.B.T.tocsr()

    def value(self, f, lam1, lam2, eps) -> float:
        return phi_tilde3(self.B @ np.ravel(f), self.dv, lam1, lam2, eps)

    def grad(self, f, lam1, lam2, eps) -> np.ndarray:
        return self.Bt @ grad_phi_tilde3(self.B @ np.ravel(f), self.dv, lam1, lam2, eps)


# --------------------------------------------------------------------------
# The volume problem and APPGA on it
# --------------------------------------------------------------------------

class VolumeProblem:
    """Slices z = 0..nz-1 with sinograms g[z], backgrounds gamma[z] and the
    same A (m x N^2).  Volumes are arrays of shape [nz, N^2]."""

    def __init__(self, A, g, gamma, n: int):
        self.A = sp.csr_matrix(A, dtype=np.float64)
        self.At = self.A.T.tocsr()
        self.g = np.atleast_2d(np.asarray(g, dtype=np.float64))
        self.gamma = np.atleast_2d(np.asarray(gamma, dtype=np.float64))
        self.nz = self.g.shape[0]
        self.n = int(n)
        self.d = self.n * self.n
        assert self.A.shape == (self.g.shape[1], self.d) and self.gamma.shape == self.g.shape
        self.reg = Regulariser3D(self.nz, self.n)

    def fidelity(self, f: np.ndarray) -> float:
        """sum_z <A f_z, 1> - <ln(A f_z + gamma_z), g_z>."""
        y = (self.A @ f.T).T
        return float(np.sum(y) - np.sum(np.log(y + self.gamma) * self.g))

    def objective(self, f, lam1, lam2, eps) -> float:
        if np.any(f < 0):
            return math.inf
        return self.fidelity(f) + self.reg.value(f, lam1, lam2, eps)

    def em_lambda(self) -> np.ndarray:
        """Lambda_j = (A^T 1)_j if positive, else 1: the same for every slice."""
        s = self.At @ np.ones(self.A.shape[0])
        return np.where(s > 0, s, 1.0)


def appga_volume_step(prob: VolumeProblem, f_k: np.ndarray, f_km1: np.ndarray, theta: float,
                      params: Params, lam: np.ndarray):
    """One APPGA map on the volume (arrays [nz, d]).  Returns (f^{k+1}, guard hits).

    f~ = f^k + theta (f^k - f^{k-1})
    grad_z = A^T (1 - g_z / den_z) + (B^T grad phi~(B f~))_z,
    den_z = max(A f~_z + gamma_z, kappa gamma_z)
    f^{k+1} = max(f~ - beta (f^k / Lambda) grad, 0)
    """
    f_tl = f_k + theta * (f_k - f_km1)
    y = (prob.A @ f_tl.T).T
    den = np.maximum(y + prob.gamma, KAPPA * prob.gamma)
    hits = int(np.count_nonzero(y + prob.gamma < KAPPA * prob.gamma))
    grad_F = (prob.At @ (1.0 - prob.g / den).T).T
    grad_R = prob.reg.grad(f_tl, params.lambda1, params.lambda2, params.eps).reshape(f_k.shape)
    p = params.beta * f_k / lam[None, :]
    return np.maximum(f_tl - p * (grad_F + grad_R), 0.0), hits


def initial_volume(prob: VolumeProblem, n_angles: int) -> np.ndarray:
    """TMC_z * 1_disk for every slice, TMC_z from that slice's counts (Sec. 4.1)."""
    return np.stack([initial_image(prob.g[z], prob.gamma[z], prob.n, n_angles)
                     for z in range(prob.nz)])


def appga_volume(prob: VolumeProblem, params: Params, f_init: Optional[np.ndarray] = None,
                 n_angles: Optional[int] = None, track_phi: bool = True) -> Result:
    """APPGA on the volume from f^0 = f^1 = f_init (default: per-slice
    TMC * 1_disk); the optional stopping test uses the volume's objective."""
    f_k = (initial_volume(prob, n_angles) if f_init is None
           else np.array(f_init, dtype=np.float64).reshape(prob.nz, prob.d))
    f_km1 = f_k.copy()
    lam = prob.em_lambda()
    thetas = thetas_for(params, params.max_iters, 1)
    phis: List[float] = []
    want = track_phi or params.rel_obj_tol > 0
    if want:
        phis.append(prob.objective(f_k, params.lambda1, params.lambda2, params.eps))
    hits, done = 0, 0
    for it in range(params.max_iters):
        f_next, h = appga_volume_step(prob, f_k, f_km1, thetas[it], params, lam)
        hits += h
        f_km1, f_k = f_k, f_next
        done += 1
        if want:
            phis.append(prob.objective(f_k, params.lambda1, params.lambda2, params.eps))
            if params.rel_obj_tol > 0 and abs(phis[-1] - phis[-2]) <= params.rel_obj_tol * abs(phis[-2]):
                break
    return Result(f=f_k, f_prev=f_km1, iters=done, phi=phis, guard_hits=hits, thetas=thetas[:done])
