"""FP64 CPU oracle of the fixed-point proximity algorithm (FPPA) and its
momentum-accelerated form (AFPPA) for the non-smooth HOITV model (the
paper's extension of the GN momentum, Sec. 4.4; model Eq. model:HOTV).

TEST INFRASTRUCTURE ONLY, like the rest of this package: only the tests,
the package smoke check and the benchmark's CPU-baseline leg may import it.

Model: minimise F(f) + lam1 sum_i ||(B1 f)_i||_2 + lam2 sum_i ||(B2 f)_i||_2
over f >= 0, the groups being the pairs (x_i, x_{d+i}) of B1 f and the
quadruples (x_i, x_{d+i}, x_{2d+i}, x_{3d+i}) of B2 f (Sec. 2.1).

AFPPA iteration (the paper's scheme, step by step):

    f~ = f^k + theta_k (f^k - f^{k-1}),  b~, c~ likewise (dual fields)
    f^{k+1} = max(f~ - P (grad F(f~) + B1^T b~ + B2^T c~), 0)
    b^{k+1} = rho1 (I - prox_{(lam1/rho1) ||.||}) (b~/rho1 + B1 (2 f^{k+1} - f~))
    c^{k+1} = rho2 (I - prox_{(lam2/rho2) ||.||}) (c~/rho2 + B2 (2 f^{k+1} - f~))

with P the EM preconditioner beta diag(f^k / Lambda) (Eq. EM) and
rho1 = 1 / (2 * 8 * p_max), rho2 = 1 / (2 * 64 * p_max), p_max the largest
entry of P.  FPPA is theta_k = 0.

Readings where the paper leaves a choice open (each also in the design notes):

* The prox in the dual updates is that of the plain group l2 sum scaled by
  lam/rho (the printed phi_1, phi_2 already carry lam, which would count it
  twice).  Since I - prox_{t||.||} is the projection onto the l2 ball of
  radius t, group by group,
      rho (I - prox_{(lam/rho)||.||})(z) = rho proj_{ball(lam/rho)}(z)
                                         = proj_{ball(lam)}(rho z),
  so every dual group stays in the ball of radius lam.
* P is recomputed from f^k every iteration (as in APPGA), and so are rho1
  and rho2 from its largest entry; ``p_fixed`` fixes P (and the rhos).  If
  the iterate has become all zero (P = 0, an absorbing state of the EM
  preconditioner) the previous rhos are kept.
* The duals start at zero: b^0 = b^1 = 0, c^0 = c^1 = 0; f^0 = f^1 = f_init.
* The ratio uses the same guarded denominator as APPGA (kappa gamma).
* RE(k) = ||f^k - f^{k-1}||_2 / ||f^k||_2 is recorded for every new iterate.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

from .appga_oracle import KAPPA, Params, Problem, b1_matrix, b2_matrix, initial_image, thetas_for


def ball_projection(z: np.ndarray, d: int, ncomp: int, radius: float) -> np.ndarray:
    """Projects each group (z_i, z_{d+i}, ..., z_{(ncomp-1)d+i}) of z onto the
    l2 ball of the given radius."""
    g = np.stack([z[q * d:(q + 1) * d] for q in range(ncomp)], axis=1)
    nrm = np.sqrt(np.sum(g * g, axis=1))
    scale = np.where(nrm > radius, radius / np.where(nrm > 0, nrm, 1.0), 1.0)
    g = g * scale[:, None]
    return np.concatenate([g[:, q] for q in range(ncomp)])


def group_norm_sum(u: np.ndarray, d: int, ncomp: int) -> float:
    g = np.stack([u[q * d:(q + 1) * d] for q in range(ncomp)], axis=1)
    return float(np.sum(np.sqrt(np.sum(g * g, axis=1))))


def hoitv_objective(prob: Problem, f: np.ndarray, lam1: float, lam2: float) -> float:
    """F(f) + lam1 sum ||(B1 f)_i|| + lam2 sum ||(B2 f)_i||  (f >= 0)."""
    B1 = b1_matrix(prob.n)
    B2 = b2_matrix(prob.n)
    return (prob.fidelity(f) + lam1 * group_norm_sum(B1 @ f, prob.d, 2)
            + lam2 * group_norm_sum(B2 @ f, prob.d, 4))


@dataclasses.dataclass
class AfppaResult:
    f: np.ndarray
    f_prev: np.ndarray
    b: np.ndarray
    c: np.ndarray
    iters: int
    re: List[float]          # RE of f^2, f^3, ...
    rho1: List[float]
    rho2: List[float]
    guard_hits: int


def afppa(prob: Problem, params: Params, f_init: Optional[np.ndarray] = None,
          n_angles: Optional[int] = None, p_fixed: Optional[np.ndarray] = None) -> AfppaResult:
    """params: lambda1, lambda2, beta, max_iters, momentum ("gn", "none" =
    FPPA, "nesterov"), omega, a, b, precond_freeze_iter (eps is not used)."""
    if f_init is None:
        f_init = initial_image(prob.g, prob.gamma, prob.n, n_angles)
    d = prob.d
    B1 = b1_matrix(prob.n)
    B2 = b2_matrix(prob.n)
    f_k = np.array(f_init, dtype=np.float64)
    f_km1 = f_k.copy()
    b_k = np.zeros(2 * d)
    b_km1 = b_k.copy()
    c_k = np.zeros(4 * d)
    c_km1 = c_k.copy()
    lam = prob.em_lambda()
    thetas = thetas_for(params, params.max_iters, 1)
    re: List[float] = []
    rho1s: List[float] = []
    rho2s: List[float] = []
    hits = 0
    p_frozen = None
    for it in range(params.max_iters):
        k = 1 + it
        th = thetas[it]
        f_tl = f_k + th * (f_k - f_km1)
        b_tl = b_k + th * (b_k - b_km1)
        c_tl = c_k + th * (c_k - c_km1)
        if p_fixed is not None:
            p_vec = p_fixed
        elif params.precond_freeze_iter >= 0 and k > params.precond_freeze_iter:
            p_vec = p_frozen
        else:
            p_vec = params.beta * f_k / lam
            if params.precond_freeze_iter >= 0 and k == params.precond_freeze_iter:
                p_frozen = p_vec.copy()
        p_max = float(np.max(p_vec))
        if p_max > 0.0 or not rho1s:
            rho1 = 1.0 / (2.0 * 8.0 * p_max)
            rho2 = 1.0 / (2.0 * 64.0 * p_max)
        # (an all-zero iterate has P = 0 and stays at zero: the rhos are kept)
        y = prob.A @ f_tl
        den = np.maximum(y + prob.gamma, KAPPA * prob.gamma)
        hits += int(np.count_nonzero(y + prob.gamma < KAPPA * prob.gamma))
        grad_F = prob.At @ (prob.ones_m - prob.g / den)
        f_next = np.maximum(f_tl - p_vec * (grad_F + B1.T @ b_tl + B2.T @ c_tl), 0.0)
        u = 2.0 * f_next - f_tl
        b_next = rho1 * ball_projection(b_tl / rho1 + B1 @ u, d, 2, params.lambda1 / rho1)
        c_next = rho2 * ball_projection(c_tl / rho2 + B2 @ u, d, 4, params.lambda2 / rho2)
        nrm = float(np.linalg.norm(f_next))
        re.append(float(np.linalg.norm(f_next - f_k)) / nrm if nrm > 0 else 0.0)
        rho1s.append(rho1)
        rho2s.append(rho2)
        f_km1, f_k = f_k, f_next
        b_km1, b_k = b_k, b_next
        c_km1, c_k = c_k, c_next
    return AfppaResult(f=f_k, f_prev=f_km1, b=b_k, c=c_k, iters=params.max_iters, re=re,
                       rho1=rho1s, rho2=rho2s, guard_hits=hits)
