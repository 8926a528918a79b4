"""Pins of the FPPA / AFPPA oracle for the non-smooth HOITV model (Sec. 4.4
extension of the GN momentum): closed forms, a special case that reduces to
MLEM, a minimiser known in closed form, and the dual invariants."""
import numpy as np
import pytest
import scipy.optimize as so

from oracle import afppa_oracle as AF
from oracle import appga_oracle as O
from paper_2409_13344_gb300 import workload as W


def test_ball_projection_hand_cases():
    d = 3
    z = np.array([3.0, 0.0, 0.3, 4.0, 0.0, 0.4])   # groups (3,4), (0,0), (0.3,0.4)
    p = AF.ball_projection(z, d, 2, 1.0)
    np.testing.assert_allclose(p, [0.6, 0.0, 0.3, 0.8, 0.0, 0.4], rtol=0, atol=1e-15)


def test_dual_update_is_rho_times_identity_minus_prox():
    # rho (I - prox_{(lam/rho)||.||})(z), with the prox written out as group
    # soft-thresholding, equals the projection of rho z onto the ball of radius lam
    rng = np.random.default_rng(0)
    d, ncomp, lam, rho = 50, 4, 0.3, 2.5
    z = rng.normal(0, 0.2, ncomp * d)
    g = np.stack([z[q * d:(q + 1) * d] for q in range(ncomp)], axis=1)
    nrm = np.linalg.norm(g, axis=1)
    t = lam / rho
    prox = g * np.maximum(1.0 - t / np.maximum(nrm, 1e-300), 0.0)[:, None]
    lhs = rho * (g - prox)
    lhs = np.concatenate([lhs[:, q] for q in range(ncomp)])
    np.testing.assert_allclose(lhs, AF.ball_projection(rho * z, d, ncomp, lam), atol=1e-15)


def _dense():
    A, _, g, gamma = W.dense_problem(8, 96, seed=11)
    return O.Problem(A, g, gamma, 8)


def test_unregularised_fppa_is_mlem():
    # lam1 = lam2 = 0: the duals stay 0 and, with theta = 0 and beta = 1, each
    # FPPA map is one MLEM update (closed form)
    prob = _dense()
    x0 = np.full(prob.d, float(np.sum(prob.g)) / float(np.sum(prob.A.toarray())))
    f = x0.copy()
    for _ in range(5):
        f = O.mlem_step(prob, f)
    par = O.Params(lambda1=0.0, lambda2=0.0, momentum="none", max_iters=5)
    res = AF.afppa(prob, par, f_init=x0)
    np.testing.assert_allclose(res.f, f, rtol=1e-13)
    assert not res.b.any() and not res.c.any()


def test_fppa_reaches_the_constant_minimiser_for_strong_penalties():
    # With large lam the HOITV minimiser is a constant image c* 1, where c*
    # minimises the 1-D fidelity c sum(A 1) - sum g ln(c (A 1) + gamma)
    prob = _dense()
    a1 = prob.A.toarray().sum(axis=1)
    cstar = so.brentq(lambda c: a1.sum() - np.sum(prob.g * a1 / (c * a1 + prob.gamma)),
                      1e-9, 1e6, xtol=1e-15, rtol=1e-15)
    x0 = np.full(prob.d, float(np.sum(prob.g)) / float(np.sum(prob.A.toarray())))
    par = O.Params(lambda1=100.0, lambda2=100.0, momentum="none", max_iters=3000)
    res = AF.afppa(prob, par, f_init=x0)
    assert np.max(np.abs(res.f - cstar)) <= 1e-8 * cstar
    # the duals are in their balls and certify stationarity: grad F + B^T [b; c] = 0
    B1, B2 = O.b1_matrix(8), O.b2_matrix(8)
    r = prob.grad_fidelity(res.f) + B1.T @ res.b + B2.T @ res.c
    assert np.max(np.abs(r)) <= 1e-6 * np.max(np.abs(prob.grad_fidelity(x0)))


def test_duals_stay_in_their_balls_and_momentum_variants_run():
    A = W.system_matrix("64")
    geom = W.GEOMETRIES["64"]
    sl = W.make_slice(A, geom, 1e5, W.seed_for(1))
    prob = O.Problem(A, sl.g, sl.gamma, geom.n)
    for mom in ("none", "gn", "nesterov"):
        par = O.Params(lambda1=0.05, lambda2=0.02, momentum=mom, omega=0.5, max_iters=30)
        res = AF.afppa(prob, par, n_angles=geom.n_angles)
        d = prob.d
        nb = np.hypot(res.b[:d], res.b[d:])
        nc = np.sqrt(sum(res.c[q * d:(q + 1) * d] ** 2 for q in range(4)))
        assert nb.max() <= 0.05 * (1 + 1e-12) and nc.max() <= 0.02 * (1 + 1e-12)
        assert np.all(res.f >= 0) and len(res.re) == 30
        assert all(r1 > 0 for r1 in res.rho1)


def test_fppa_objective_decreases_on_siddon_slice():
    A = W.system_matrix("64")
    geom = W.GEOMETRIES["64"]
    sl = W.make_slice(A, geom, 1e5, W.seed_for(1))
    prob = O.Problem(A, sl.g, sl.gamma, geom.n)
    par = O.Params(lambda1=0.05, lambda2=0.02, momentum="none", beta=0.3, max_iters=60)
    f0 = O.initial_image(sl.g, sl.gamma, geom.n, geom.n_angles)
    res = AF.afppa(prob, par, f_init=f0)
    assert AF.hoitv_objective(prob, res.f, 0.05, 0.02) < AF.hoitv_objective(prob, f0, 0.05, 0.02)
    assert res.re[-1] < res.re[0]
