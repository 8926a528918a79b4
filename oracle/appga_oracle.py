"""FP64 CPU oracle of APPGA for SHOITV-regularised PET reconstruction.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
the CPU-baseline leg of the benchmark may import this module.  The product
path (the CUDA library and its binding) never imports, links or calls it,
and this module imports nothing from the product path.

Everything is plain NumPy / SciPy in float64, written step by step in the
paper's notation so it can be checked against the paper by eye:

* F(f) = <Af, 1> - <ln(Af + gamma), g>                    (Eq. FidelityTerm)
* D, B1, B2 built literally as Kronecker products          (Sec. 2.1)
* s_eps and its gradient x / max(||x||, eps)               (Eq. def:smoothL2, Eq. gradenvL2)
* phi = F + phi~ o B,  Phi = phi + iota                    (Eq. def:phi)
* prox of iota under any diagonal metric = max(x, 0)       (Eq. cloformproiota)
* GN momentum theta_k = (t_{k-1}-1)/t_k, t_k = a k^w + b   (Eq. GNtheta)
* EM preconditioner P = beta diag(f^k / Lambda)            (Eq. EM)
* APPGA iteration                                          (Eq. APPGAiter)
* initial image TMC * 1_disk                               (Sec. 4.1)

Readings where the paper is silent (each also listed in the design notes):

* Pixels are vectorised row-major (j = r*N + c), so I (x) D differences
  along c.  The regulariser is invariant under transposing the image, so
  this choice does not change phi.
* The preconditioner uses the non-extrapolated iterate f^k, recomputed every
  iteration until ``precond_freeze_iter`` (then frozen), as Eq. EM states.
* Momentum can make A f~ + gamma non-positive; the ratio uses the guarded
  denominator max(A f~ + gamma, kappa * gamma) with kappa = 1e-3 and counts
  the guarded bins.  Phi itself is only evaluated at f >= 0, where no guard
  is needed when gamma > 0.
* The disk of the initial image holds the pixels whose centres satisfy
  x^2 + y^2 <= (N/2)^2; ACTc = sum(g) - sum(gamma); NPA = number of angles.
* The "K iterations" of a run are K applications of the APPGA map, starting
  from f^0 = f^1 = f_init, so the result is f^{K+1}.

Pins (tests/test_oracle.py, tests/golden/): the difference operators against
hand-written matrices and a pixel-loop definition; phi~ and its gradient on a
hand-worked 3 x 3 image with lambda1 != lambda2 and both s_eps branches; the
Lambda_j = 1 branch of Eq. EM, the preconditioner freeze and the relative-
objective stop on hand-solved one- and four-pixel problems in exact rational
arithmetic; MLEM as the unregularised momentum-free step; finite
differences; KKT against L-BFGS-B; the momentum closed forms.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np
import scipy.sparse as sp

KAPPA = 1e-3  # guard factor of the Poisson-ratio denominator (reading above)


# --------------------------------------------------------------------------
# Difference operators (Sec. 2.1)
# --------------------------------------------------------------------------

def difference_matrix(n: int) -> sp.csr_matrix:
    """Backward difference D (N x N): D_jj = 1, D_j,j-1 = -1 for j = 2..N
    (1-based); every other entry, including all of row 1, is zero."""
    rows, cols, vals = [], [], []
    for j in range(1, n):  # 0-based rows 1..N-1 == paper rows 2..N
        rows += [j, j]
        cols += [j, j - 1]
        vals += [1.0, -1.0]
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n), dtype=np.float64)


def b1_matrix(n: int) -> sp.csr_matrix:
    """First-order differences B1 = [I (x) D ; D (x) I]  (2d x d)."""
    D = difference_matrix(n)
    I = sp.identity(n, format="csr", dtype=np.float64)
    return sp.vstack([sp.kron(I, D), sp.kron(D, I)]).tocsr()


def b2_matrix(n: int) -> sp.csr_matrix:
    """Second-order differences
    B2 = [I (x) (-D^T D) ; (-D^T) (x) D ; (-D^T D) (x) I ; D (x) (-D^T)]  (4d x d)."""
    D = difference_matrix(n)
    Dt = D.T.tocsr()
    I = sp.identity(n, format="csr", dtype=np.float64)
    mDtD = -(Dt @ D)
    return sp.vstack([sp.kron(I, mDtD), sp.kron(-Dt, D),
                      sp.kron(mDtD, I), sp.kron(D, -Dt)]).tocsr()


def b_matrix(n: int) -> sp.csr_matrix:
    """B = [B1 ; B2]  (6d x d)."""
    return sp.vstack([b1_matrix(n), b2_matrix(n)]).tocsr()


# --------------------------------------------------------------------------
# Smoothed l2 norm and the SHOITV regulariser (Eq. def:smoothL2, Sec. 2.1-2.2)
# --------------------------------------------------------------------------

def s_eps(x: np.ndarray, eps: float) -> np.ndarray:
    """s_eps applied to each row of x (shape [groups, comps])."""
    nrm = np.sqrt(np.sum(x * x, axis=1))
    return np.where(nrm > eps, nrm - eps / 2.0, nrm * nrm / (2.0 * eps))


def grad_s_eps(x: np.ndarray, eps: float) -> np.ndarray:
    """Gradient of s_eps per row: x / max(||x||_2, eps)."""
    nrm = np.sqrt(np.sum(x * x, axis=1))
    return x / np.maximum(nrm, eps)[:, None]


def _groups(u: np.ndarray, d: int):
    """Split u in R^{6d} into the first-order pairs (x_i, x_{d+i}) and the
    second-order quadruples (x_{2d+i}, ..., x_{5d+i})."""
    u1 = np.stack([u[0:d], u[d:2 * d]], axis=1)
    u2 = np.stack([u[2 * d:3 * d], u[3 * d:4 * d], u[4 * d:5 * d], u[5 * d:6 * d]], axis=1)
    return u1, u2


def phi_tilde(u: np.ndarray, d: int, lam1: float, lam2: float, eps: float) -> float:
    """phi~(u) = lam1 sum_i s_eps(pair_i) + lam2 sum_i s_eps(quad_i)."""
    u1, u2 = _groups(u, d)
    return lam1 * float(np.sum(s_eps(u1, eps))) + lam2 * float(np.sum(s_eps(u2, eps)))


def grad_phi_tilde(u: np.ndarray, d: int, lam1: float, lam2: float, eps: float) -> np.ndarray:
    """Gradient of phi~ at u (Sec. 2.2): lam * x / max(group norm, eps)."""
    u1, u2 = _groups(u, d)
    v1 = lam1 * grad_s_eps(u1, eps)
    v2 = lam2 * grad_s_eps(u2, eps)
    return np.concatenate([v1[:, 0], v1[:, 1], v2[:, 0], v2[:, 1], v2[:, 2], v2[:, 3]])


# --------------------------------------------------------------------------
# Problem
# --------------------------------------------------------------------------

class Problem:
    """A (m x d, promoted to float64), g, gamma and the image side N."""

    def __init__(self, A, g, gamma, n: int):
        if sp.issparse(A):
            self.A = sp.csr_matrix(A, dtype=np.float64)
        else:
            self.A = sp.csr_matrix(np.asarray(A, dtype=np.float64))
        self.At = self.A.T.tocsr()
        self.g = np.asarray(g, dtype=np.float64)
        self.gamma = np.asarray(gamma, dtype=np.float64)
        self.n = int(n)
        self.d = self.n * self.n
        assert self.A.shape == (self.g.shape[0], self.d)
        self.B = b_matrix(self.n)
        self.Bt = self.B.T.tocsr()
        self.ones_m = np.ones(self.A.shape[0])

    # ---- fidelity (Eq. FidelityTerm) and its gradient (Sec. 2.2) ----
    def fidelity(self, f: np.ndarray) -> float:
        y = self.A @ f
        return float(np.dot(y, self.ones_m) - np.dot(np.log(y + self.gamma), self.g))

    def grad_fidelity(self, f: np.ndarray) -> np.ndarray:
        y = self.A @ f
        return self.At @ (self.ones_m - self.g / (y + self.gamma))

    # ---- phi = F + phi~ o B (Eq. def:phi) ----
    def phi(self, f, lam1, lam2, eps) -> float:
        return self.fidelity(f) + phi_tilde(self.B @ f, self.d, lam1, lam2, eps)

    def grad_phi(self, f, lam1, lam2, eps) -> np.ndarray:
        return self.grad_fidelity(f) + self.Bt @ grad_phi_tilde(self.B @ f, self.d, lam1, lam2, eps)

    def objective(self, f, lam1, lam2, eps) -> float:
        """Phi = phi + iota (iota = +inf off the nonnegative orthant)."""
        if np.any(f < 0):
            return math.inf
        return self.phi(f, lam1, lam2, eps)

    def em_lambda(self) -> np.ndarray:
        """Lambda_j = (A^T 1)_j if positive, else 1 (Sec. 4.1, Eq. EM)."""
        s = self.At @ self.ones_m
        return np.where(s > 0, s, 1.0)


# --------------------------------------------------------------------------
# Momentum (Eq. GNtheta; Nesterov's recursion of Sec. 4.3)
# --------------------------------------------------------------------------

def gn_t(k: int, a: float, b: float, omega: float) -> float:
    return a * float(k) ** omega + b


def gn_theta(k: int, a: float, b: float, omega: float) -> float:
    """theta_k = (t_{k-1} - 1) / t_k with t_k = a k^omega + b, k >= 1."""
    return (gn_t(k - 1, a, b, omega) - 1.0) / gn_t(k, a, b, omega)


def nesterov_thetas(K: int) -> List[float]:
    """theta_1..theta_K of Nesterov's rule t_k = (1 + sqrt(1 + 4 t_{k-1}^2))/2,
    t_0 = 1."""
    out, t_prev = [], 1.0
    for _ in range(K):
        t = (1.0 + math.sqrt(1.0 + 4.0 * t_prev * t_prev)) / 2.0
        out.append((t_prev - 1.0) / t)
        t_prev = t
    return out


# --------------------------------------------------------------------------
# Initial image (Sec. 4.1)
# --------------------------------------------------------------------------

def disk_mask(n: int) -> np.ndarray:
    """Pixels whose centres lie in the inscribed disk x^2 + y^2 <= (N/2)^2."""
    c = np.arange(n, dtype=np.float64) + 0.5 - n / 2.0
    x = c[None, :]
    y = c[:, None]
    return ((x * x + y * y) <= (n / 2.0) ** 2).reshape(-1)


def initial_image(g, gamma, n: int, n_angles: int) -> np.ndarray:
    """TMC * 1_disk with TMC = ACTc / (NPFOV * NPA), ACTc = sum g - sum gamma."""
    disk = disk_mask(n)
    actc = float(np.sum(np.asarray(g, np.float64)) - np.sum(np.asarray(gamma, np.float64)))
    tmc = actc / (float(disk.sum()) * float(n_angles))
    return np.where(disk, tmc, 0.0)


# --------------------------------------------------------------------------
# APPGA (Eq. APPGAiter with Eq. EM) and PPGA (Eq. PPGAiter)
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Params:
    lambda1: float = 0.1
    lambda2: float = 0.05
    eps: float = 1e-3
    omega: float = 0.5
    a: float = 0.125
    b: float = 1.0
    beta: float = 1.0
    max_iters: int = 100
    rel_obj_tol: float = 0.0        # 0 = never stop early
    precond_freeze_iter: int = -1   # -1 = recompute P from f^k every iteration
    momentum: str = "gn"            # "gn", "none" (PPGA) or "nesterov"


@dataclasses.dataclass
class Result:
    f: np.ndarray                   # the last iterate f^{K+1}
    f_prev: np.ndarray              # f^K
    iters: int                      # number of APPGA maps applied
    phi: List[float]                # Phi(f^1), Phi(f^2), ... (if tracked)
    guard_hits: int                 # guarded ratio denominators
    thetas: List[float]


def thetas_for(params: Params, K: int, k0: int = 1) -> List[float]:
    if params.momentum == "none":
        return [0.0] * K
    if params.momentum == "nesterov":
        return nesterov_thetas(k0 + K - 1)[k0 - 1:]
    return [gn_theta(k, params.a, params.b, params.omega) for k in range(k0, k0 + K)]


def appga_step(prob: Problem, f_k: np.ndarray, f_km1: np.ndarray, theta: float,
               params: Params, lam: np.ndarray, p_vec: Optional[np.ndarray] = None):
    """One APPGA map.  Returns (f^{k+1}, guard hits).

    f~ = f^k + theta (f^k - f^{k-1})
    grad = A^T (1 - g / den) + B^T grad phi~(B f~),  den = max(A f~ + gamma, kappa gamma)
    P = beta f^k / Lambda (or the given frozen diagonal ``p_vec``)
    f^{k+1} = max(f~ - P grad, 0)
    """
    f_tl = f_k + theta * (f_k - f_km1)
    y = prob.A @ f_tl
    den = np.maximum(y + prob.gamma, KAPPA * prob.gamma)
    hits = int(np.count_nonzero(y + prob.gamma < KAPPA * prob.gamma))
    grad_F = prob.At @ (prob.ones_m - prob.g / den)
    grad_R = prob.Bt @ grad_phi_tilde(prob.B @ f_tl, prob.d, params.lambda1, params.lambda2, params.eps)
    if p_vec is None:
        p_vec = params.beta * f_k / lam
    return np.maximum(f_tl - p_vec * (grad_F + grad_R), 0.0), hits


def appga(prob: Problem, params: Params, f_init: Optional[np.ndarray] = None,
          n_angles: Optional[int] = None, f_prev: Optional[np.ndarray] = None,
          k0: int = 1, p_fixed: Optional[np.ndarray] = None,
          track_phi: bool = True) -> Result:
    """Run APPGA from f^{k0-1} = f_prev (default f_init), f^{k0} = f_init.

    ``p_fixed`` replaces the EM preconditioner by a fixed positive diagonal
    (the setting of the convergence theory, Sec. 3).
    """
    if f_init is None:
        f_init = initial_image(prob.g, prob.gamma, prob.n, n_angles)
    f_k = np.array(f_init, dtype=np.float64)
    f_km1 = f_k.copy() if f_prev is None else np.array(f_prev, dtype=np.float64)
    lam = prob.em_lambda()
    thetas = thetas_for(params, params.max_iters, k0)
    phis: List[float] = []
    if track_phi or params.rel_obj_tol > 0:
        phis.append(prob.objective(f_k, params.lambda1, params.lambda2, params.eps))
    hits = 0
    p_frozen = None
    done = 0
    for it in range(params.max_iters):
        k = k0 + it
        if p_fixed is not None:
            p_vec = p_fixed
        elif params.precond_freeze_iter >= 0 and k > params.precond_freeze_iter:
            if p_frozen is None:
                raise RuntimeError("freeze iteration precedes the start iteration")
            p_vec = p_frozen
        else:
            p_vec = params.beta * f_k / lam
            if params.precond_freeze_iter >= 0 and k == params.precond_freeze_iter:
                p_frozen = p_vec.copy()
        f_next, h = appga_step(prob, f_k, f_km1, thetas[it], params, lam, p_vec)
        hits += h
        f_km1, f_k = f_k, f_next
        done += 1
        if track_phi or params.rel_obj_tol > 0:
            phis.append(prob.objective(f_k, params.lambda1, params.lambda2, params.eps))
            if params.rel_obj_tol > 0 and abs(phis[-1] - phis[-2]) <= params.rel_obj_tol * abs(phis[-2]):
                break
    return Result(f=f_k, f_prev=f_km1, iters=done, phi=phis, guard_hits=hits, thetas=thetas[:done])


def mlem_step(prob: Problem, f: np.ndarray) -> np.ndarray:
    """Classical MLEM update (f / A^T 1) * A^T (g / (A f + gamma)), used as an
    independent closed form for the unregularised, momentum-free step.

    A pixel that no ray sees, (A^T 1)_j = 0, has no data: the update there is
    0/0, and such a pixel keeps its value (the sensitivity-zero convention;
    the EM-preconditioned step does the same, since its fidelity gradient is
    zero there and Lambda_j = 1 by Eq. EM)."""
    s = prob.At @ prob.ones_m
    back = prob.At @ (prob.g / (prob.A @ f + prob.gamma))
    seen = s > 0
    out = f.copy()
    out[seen] = f[seen] / s[seen] * back[seen]
    return out


def lipschitz_bound(prob: Problem, lam1: float, lam2: float, eps: float) -> float:
    """Upper bound on L_phi on the nonnegative orthant:
    ||A||_2^2 max(g / gamma^2) + (lam1 ||B1||^2 + lam2 ||B2||^2) / eps with
    ||B1||^2 <= 8 and ||B2||^2 <= 64; the smoothed-norm gradient is
    (1/eps)-Lipschitz (the paper's 2/eps bound is also valid)."""
    A = prob.A.toarray() if prob.A.shape[0] * prob.A.shape[1] <= 4_000_000 else None
    if A is None:
        raise ValueError("lipschitz_bound is for small problems")
    a2 = np.linalg.norm(A, 2) ** 2
    return a2 * float(np.max(prob.g / prob.gamma ** 2)) + (8 * lam1 + 64 * lam2) / eps
