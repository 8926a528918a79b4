"""GPU parity of every hot-path step and of the solver against the FP64
oracle, through the C ABI (sm_103a library).

Tolerances (derived in the design notes):
  y = A f (double-float accumulation)        rel 1e-11 per bin
  w = 1 - g/den (FP32 output)                rel 5e-7 per bin
  A^T w (FP32 accumulation)                  |err| <= 2e-6 * (A^T |w|)_j
  B^T grad phi~(B f) (FP32 stencil)          |err| <= 2e-6 (lam1 + lam2) + 1e-5 |ref|
  one fused APPGA map                        rel L2 1e-6
  Phi (FP64 objective on identical images)   rel 1e-9
  APPGA trajectories, FP32 images            rel L2 1e-5
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import appga_oracle as O
from paper_2409_13344_gb300 import workload as W

from fp32_spread import oracle_fp32_noisy

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def A():
    from paper_2409_13344_gb300 import build
    build.build()
    from paper_2409_13344_gb300 import appga
    if not torch.cuda.is_available():
        pytest.fail("the -m gpu tests need a CUDA device")
    return appga


@pytest.fixture(scope="module")
def ctx(A):
    c = A.Context(0)
    yield c
    c.close()


DEV = "cuda:0"

# a ragged geometry: N not a multiple of the 32-pixel tile, odd bin count
RAGGED = W.Geometry(40, 48, 59)
SPARSE = W.Geometry(16, 10, 8)      # many empty rows and never-hit pixels
TINY = W.Geometry(1, 3, 3)          # d = 1: B = 0


_cache = {}


def problem(name_or_geom, counts=1e5, seed=None, phantom="ellipses"):
    if isinstance(name_or_geom, str):
        geom = W.GEOMETRIES[name_or_geom]
        Amat = W.system_matrix(name_or_geom)
    else:
        geom = name_or_geom
        key = (geom.n, geom.n_angles, geom.n_bins)
        if key not in _cache:
            _cache[key] = W.siddon_matrix(geom)
        Amat = _cache[key]
    seed = W.seed_for(1) if seed is None else seed
    sl = W.make_slice(Amat, geom, counts, seed, phantom=phantom)
    return geom, Amat, sl


def to_dev(x, dtype=torch.float32):
    return torch.as_tensor(np.asarray(x), dtype=dtype).to(DEV)


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def bf16_round(x):
    """FP32 -> BF16 (round to nearest even) -> FP32, in NumPy."""
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32)


@pytest.fixture(scope="module")
def mats(A, ctx):
    out = {}
    for key in ("64", RAGGED, SPARSE, TINY):
        geom, Amat, _ = problem(key)
        out[key if isinstance(key, str) else (key.n, key.n_angles, key.n_bins)] = \
            A.Matrix(ctx, Amat, geom.n, geom.n_angles, bf16=True)
    yield out
    for m in out.values():
        m.close()


def mkey(k):
    return k if isinstance(k, str) else (k.n, k.n_angles, k.n_bins)


GEOMS = ["64", RAGGED, SPARSE, TINY]


# ------------------------------------------------------------- step a1-a2

@pytest.mark.parametrize("gk", GEOMS, ids=["64", "ragged40", "sparse16", "tiny1"])
def test_forward_ratio(A, ctx, mats, gk):
    geom, Amat, sl = problem(gk)
    mat = mats[mkey(gk)]
    rng = np.random.default_rng(7)
    f = (sl.f_true * rng.uniform(0.5, 1.5, geom.d)).astype(np.float32)
    f[rng.uniform(size=geom.d) < 0.1] *= -40.0  # drive some bins into the guard
    y = torch.empty(geom.m, dtype=torch.float64, device=DEV)
    w = torch.empty(geom.m, dtype=torch.float32, device=DEV)
    A.appga_forward_ratio(ctx.handle, mat.handle, to_dev(f), to_dev(sl.g), to_dev(sl.gamma), y, w)
    torch.cuda.synchronize()
    A64 = Amat.astype(np.float64)
    y_ref = A64 @ f.astype(np.float64)
    gam = sl.gamma.astype(np.float64)
    den = np.maximum(y_ref + gam, O.KAPPA * gam)
    w_ref = 1.0 - sl.g / den
    yg = y.cpu().numpy()
    np.testing.assert_allclose(yg, y_ref, rtol=1e-11, atol=1e-300)
    np.testing.assert_allclose(w.cpu().numpy(), w_ref, rtol=5e-7, atol=1e-30)
    assert np.any(y_ref + gam < O.KAPPA * gam) or gk is TINY or gk is SPARSE


@pytest.mark.parametrize("gk", ["64", RAGGED], ids=["64", "ragged40"])
def test_data_term(A, ctx, mats, gk):
    geom, Amat, sl = problem(gk)
    f = sl.f_true.astype(np.float32)
    y = torch.empty(geom.m, dtype=torch.float64, device=DEV)
    data = torch.zeros(1, dtype=torch.float64, device=DEV)
    A.appga_forward_ratio(ctx.handle, mats[mkey(gk)].handle, to_dev(f), to_dev(sl.g),
                          to_dev(sl.gamma), y, None, data)
    torch.cuda.synchronize()
    prob = O.Problem(Amat, sl.g, sl.gamma, geom.n)
    ref = prob.fidelity(f.astype(np.float64))
    assert abs(float(data.item()) - ref) <= 1e-11 * abs(ref)


# ------------------------------------------------------------------ step a3

@pytest.mark.parametrize("gk", GEOMS, ids=["64", "ragged40", "sparse16", "tiny1"])
def test_backproject(A, ctx, mats, gk):
    geom, Amat, _ = problem(gk)
    rng = np.random.default_rng(3)
    w = rng.uniform(-1, 1, geom.m).astype(np.float32)
    out = torch.empty(geom.d, dtype=torch.float32, device=DEV)
    A.appga_backproject(ctx.handle, mats[mkey(gk)].handle, to_dev(w), out)
    torch.cuda.synchronize()
    At = Amat.astype(np.float64).T.tocsr()
    ref = At @ w.astype(np.float64)
    scale = At @ np.abs(w.astype(np.float64))
    err = np.abs(out.cpu().numpy() - ref)
    assert np.all(err <= 2e-6 * scale + 1e-30)


def test_adjoint_identity_device(A, ctx, mats):
    # <A x, z> = <x, A^T z> with both products from the device kernels
    geom, Amat, sl = problem("64")
    mat = mats["64"]
    rng = np.random.default_rng(11)
    x = rng.uniform(0, 1, geom.d).astype(np.float32)
    z = rng.uniform(-1, 1, geom.m).astype(np.float32)
    y = torch.empty(geom.m, dtype=torch.float64, device=DEV)
    A.appga_forward_ratio(ctx.handle, mat.handle, to_dev(x), to_dev(sl.g), to_dev(sl.gamma), y)
    bt = torch.empty(geom.d, dtype=torch.float32, device=DEV)
    A.appga_backproject(ctx.handle, mat.handle, to_dev(z), bt)
    torch.cuda.synchronize()
    lhs = float(np.dot(y.cpu().numpy(), z.astype(np.float64)))
    rhs = float(np.dot(x.astype(np.float64), bt.cpu().numpy().astype(np.float64)))
    assert abs(lhs - rhs) <= 1e-5 * np.sum(np.abs(z)) * np.max(y.cpu().numpy())


# ------------------------------------------------------------------ step a4

@pytest.mark.parametrize("n", [1, 2, 3, 5, 31, 33, 64, 100])
@pytest.mark.parametrize("eps", [1e-3, 0.3])
def test_shoitv_grad(A, ctx, n, eps):
    rng = np.random.default_rng(n)
    F = rng.uniform(0, 1, (n, n))
    F[: n // 2, : n // 3] = 0.25          # flat block: quadratic branch of s_eps
    F = F.astype(np.float32)
    lam1, lam2 = 0.1, 0.05
    out = torch.empty(n * n, dtype=torch.float32, device=DEV)
    A.appga_shoitv_grad(ctx.handle, n, to_dev(F.reshape(-1)), lam1, lam2, eps, out)
    torch.cuda.synchronize()
    B = O.b_matrix(n)
    ref = B.T @ O.grad_phi_tilde(B @ F.reshape(-1).astype(np.float64), n * n, lam1, lam2, eps)
    err = np.abs(out.cpu().numpy() - ref)
    assert np.all(err <= 2e-6 * (lam1 + lam2) + 1e-5 * np.abs(ref)), float(err.max())


def test_shoitv_adjoint_symmetry(A, ctx):
    # transposing the image transposes B^T grad phi~(B f) (block swap 3<->5, 4<->6)
    n = 48
    rng = np.random.default_rng(5)
    F = rng.uniform(0, 1, (n, n)).astype(np.float32)
    outs = []
    for X in (F, np.ascontiguousarray(F.T)):
        o = torch.empty(n * n, dtype=torch.float32, device=DEV)
        A.appga_shoitv_grad(ctx.handle, n, to_dev(X.reshape(-1)), 0.2, 0.1, 1e-2, o)
        outs.append(o.cpu().numpy().reshape(n, n))
    np.testing.assert_allclose(outs[0], outs[1].T, atol=2e-6)


# ----------------------------------------------------- fused map a0+a3+a4+a5

@pytest.mark.parametrize("gk", ["64", RAGGED, SPARSE], ids=["64", "ragged40", "sparse16"])
def test_pixel_update(A, ctx, mats, gk):
    geom, Amat, sl = problem(gk)
    prob = O.Problem(Amat, sl.g, sl.gamma, geom.n)
    rng = np.random.default_rng(2)
    f_cur = (sl.f_true * rng.uniform(0.8, 1.2, geom.d) + 1e-3).astype(np.float32)
    f_prev = (sl.f_true * rng.uniform(0.8, 1.2, geom.d) + 1e-3).astype(np.float32)
    theta = 0.7
    f_tl = f_cur.astype(np.float64) + theta * (f_cur.astype(np.float64) - f_prev)
    y = prob.A @ f_tl
    den = np.maximum(y + prob.gamma, O.KAPPA * prob.gamma)
    w = (1.0 - prob.g / den).astype(np.float32)
    p = A.default_params(lambda1=0.1, lambda2=0.05, eps=1e-3, beta=1.0)
    out = torch.empty(geom.d, dtype=torch.float32, device=DEV)
    A.appga_pixel_update(ctx.handle, mats[mkey(gk)].handle, to_dev(f_prev), to_dev(f_cur),
                         to_dev(w), theta, p, out)
    torch.cuda.synchronize()
    grad = prob.At @ w.astype(np.float64) + prob.Bt @ O.grad_phi_tilde(
        prob.B @ f_tl, prob.d, 0.1, 0.05, 1e-3)
    ref = np.maximum(f_tl - 1.0 * f_cur / prob.em_lambda() * grad, 0.0)
    assert rel_l2(out.cpu().numpy(), ref) <= 1e-6


# ------------------------------------------------------------------ step a6

@pytest.mark.parametrize("gk", ["64", RAGGED, "256"], ids=["64", "ragged40", "256"])
def test_objective(A, ctx, gk):
    geom, Amat, sl = problem(gk, counts=1e6 if gk == "256" else 1e5)
    mat = A.Matrix(ctx, Amat, geom.n, geom.n_angles)
    rng = np.random.default_rng(9)
    f = (sl.f_true * rng.uniform(0.9, 1.1, geom.d)).astype(np.float32)
    p = A.default_params(lambda1=0.1, lambda2=0.05, eps=1e-3)
    phi = A.appga_objective(ctx.handle, mat.handle, to_dev(f), to_dev(sl.g), to_dev(sl.gamma), p)
    ref = O.Problem(Amat, sl.g, sl.gamma, geom.n).objective(f.astype(np.float64), 0.1, 0.05, 1e-3)
    assert abs(phi - ref) <= 1e-9 * abs(ref), (phi, ref)
    mat.close()


def test_initial_image(A, ctx, mats):
    geom, Amat, sl = problem("64")
    out = torch.empty(geom.d, dtype=torch.float32, device=DEV)
    A.appga_initial_image(ctx.handle, mats["64"].handle, to_dev(sl.g), to_dev(sl.gamma), out)
    torch.cuda.synchronize()
    ref = O.initial_image(sl.g, sl.gamma, geom.n, geom.n_angles)
    got = out.cpu().numpy()
    np.testing.assert_array_equal(got > 0, ref > 0)
    np.testing.assert_allclose(got, ref, rtol=1e-7)


# ---------------------------------------------------------------- solver

def run_gpu(A, ctx, mat, sl, **kw):
    p = A.default_params(**kw)
    f = torch.empty(mat.d, dtype=torch.float32, device=DEV)
    st = A.appga_reconstruct(ctx.handle, mat.handle, to_dev(sl.g), to_dev(sl.gamma), None, p, f)
    return f.cpu().numpy(), st


def run_oracle(geom, Amat, sl, **kw):
    prob = O.Problem(Amat, sl.g, sl.gamma, geom.n)
    par = O.Params(**kw)
    return prob, O.appga(prob, par, n_angles=geom.n_angles, track_phi=par.rel_obj_tol > 0)


@pytest.mark.parametrize("omega", [0.25, 0.5, 1.0])
def test_trajectory_64_short(A, ctx, mats, omega):
    geom, Amat, sl = problem("64")
    f, st = run_gpu(A, ctx, mats["64"], sl, max_iters=30, omega=omega, track_objective=1)
    prob, ref = run_oracle(geom, Amat, sl, max_iters=30, omega=omega)
    assert st.iters == 30 and st.result_k == 31
    assert rel_l2(f, ref.f) <= 1e-5
    phi_same = prob.objective(f.astype(np.float64), 0.1, 0.05, 1e-3)
    assert abs(st.phi - phi_same) <= 1e-9 * abs(phi_same)


@pytest.mark.parametrize("gk,kw", [
    ("64", dict(beta=0.1)),
    (RAGGED, dict(beta=0.03)),
    # pixels no ray sees have Lambda = 1 (Eq. EM) and a huge step; without the
    # regulariser their gradient is zero and the run stays well conditioned
    (SPARSE, dict(beta=1.0, lambda1=0.0, lambda2=0.0)),
], ids=["64", "ragged40", "sparse16"])
def test_trajectory_long_small_step(A, ctx, mats, gk, kw):
    # beta small enough that p_max meets the step-size condition on the small
    # grids; with beta = 1 they amplify rounding (see the design notes)
    geom, Amat, sl = problem(gk)
    f, st = run_gpu(A, ctx, mats[mkey(gk)], sl, max_iters=150, omega=1.0, **kw)
    _, ref = run_oracle(geom, Amat, sl, max_iters=150, omega=1.0, **kw)
    assert rel_l2(f, ref.f) <= 1e-5


def test_trajectory_tiny(A, ctx, mats):
    geom, Amat, sl = problem(TINY)
    f, st = run_gpu(A, ctx, mats[mkey(TINY)], sl, max_iters=20)
    _, ref = run_oracle(geom, Amat, sl, max_iters=20)
    assert rel_l2(f, ref.f) <= 1e-6


@pytest.mark.parametrize("momentum,mname", [(1, "none"), (2, "nesterov")])
def test_momentum_variants(A, ctx, mats, momentum, mname):
    geom, Amat, sl = problem("64")
    f, _ = run_gpu(A, ctx, mats["64"], sl, max_iters=40, momentum=momentum)
    _, ref = run_oracle(geom, Amat, sl, max_iters=40, momentum=mname)
    assert rel_l2(f, ref.f) <= 1e-5


def test_preconditioner_freeze(A, ctx, mats):
    geom, Amat, sl = problem("64")
    f, _ = run_gpu(A, ctx, mats["64"], sl, max_iters=40, precond_freeze_iter=6)
    _, ref = run_oracle(geom, Amat, sl, max_iters=40, precond_freeze_iter=6)
    assert rel_l2(f, ref.f) <= 1e-5


def test_stopping_rule(A, ctx, mats):
    geom, Amat, sl = problem("64")
    tol = 1e-6
    f, st = run_gpu(A, ctx, mats["64"], sl, max_iters=400, beta=0.1, omega=1.0, rel_obj_tol=tol,
                    graph_iters=8)
    prob, ref = run_oracle(geom, Amat, sl, max_iters=400, beta=0.1, omega=1.0, rel_obj_tol=tol)
    assert st.stopped_early == 1 and ref.iters < 400
    assert abs(st.iters - ref.iters) <= 1
    # the test can fire one map apart on FP32 and FP64 objectives; the image
    # is compared with the oracle's iterate after the GPU's own map count
    if st.iters != ref.iters:
        _, ref = run_oracle(geom, Amat, sl, max_iters=st.iters, beta=0.1, omega=1.0)
    assert rel_l2(f, ref.f) <= 1e-5
    phi_same = prob.objective(f.astype(np.float64), 0.1, 0.05, 1e-3)
    assert abs(st.phi - phi_same) <= 1e-9 * abs(phi_same)


@pytest.mark.parametrize("track", [0, 1])
def test_zero_maps_returns_the_initial_image(A, ctx, mats, track):
    # max_iters = 0: the result is f^1 = f_init, with Phi(f^1) when tracked
    geom, Amat, sl = problem("64")
    f, st = run_gpu(A, ctx, mats["64"], sl, max_iters=0, track_objective=track)
    f0 = O.initial_image(sl.g, sl.gamma, geom.n, geom.n_angles)
    assert st.iters == 0 and st.result_k == 1 and st.stopped_early == 0
    np.testing.assert_allclose(f, f0, rtol=1e-7)
    if track:
        prob = O.Problem(Amat, sl.g, sl.gamma, geom.n)
        phi0 = prob.objective(f.astype(np.float64), 0.1, 0.05, 1e-3)
        assert abs(st.phi - phi0) <= 1e-9 * abs(phi0)
        assert math.isnan(st.phi_prev)
    else:
        assert math.isnan(st.phi)


@pytest.mark.parametrize("iters,graph_iters", [(1, 0), (5, 0), (17, 0), (23, 4), (31, 16)])
def test_exact_map_counts(A, ctx, mats, iters, graph_iters):
    # a run of K maps replays whole graphs plus power-of-two remainders and
    # must apply exactly K maps, with Phi of the result and of the map before
    geom, Amat, sl = problem("64")
    f, st = run_gpu(A, ctx, mats["64"], sl, max_iters=iters, graph_iters=graph_iters,
                    track_objective=1)
    prob = O.Problem(Amat, sl.g, sl.gamma, geom.n)
    ref = O.appga(prob, O.Params(max_iters=iters), n_angles=geom.n_angles, track_phi=True)
    assert st.iters == iters and st.result_k == iters + 1
    assert rel_l2(f, ref.f) <= 1e-5
    phi_same = prob.objective(f.astype(np.float64), 0.1, 0.05, 1e-3)
    assert abs(st.phi - phi_same) <= 1e-9 * abs(phi_same)
    # Phi of the previous iterate, against the oracle's value at f^K
    assert abs(st.phi_prev - ref.phi[-2]) <= 1e-8 * abs(ref.phi[-2])


def test_guard_hits_counted(A, ctx, mats):
    # resume from a state whose extrapolation f~ is strongly negative somewhere
    geom, Amat, sl = problem("64")
    rng = np.random.default_rng(4)
    f_cur = np.maximum(sl.f_true, 1e-3).astype(np.float32)
    f_prev = f_cur.copy()
    hot = rng.uniform(size=geom.d) < 0.05
    f_prev[hot] += 60.0 * f_cur.max()
    p = A.default_params(max_iters=1, omega=1.0)
    out = torch.empty(geom.d, dtype=torch.float32, device=DEV)
    k0 = 50
    st = A.appga_resume(ctx.handle, mats["64"].handle, to_dev(sl.g), to_dev(sl.gamma),
                        to_dev(f_prev), to_dev(f_cur), k0, p, None, out)
    prob = O.Problem(Amat, sl.g, sl.gamma, geom.n)
    th = O.gn_theta(k0, 0.125, 1.0, 1.0)
    f_next, hits = O.appga_step(prob, f_cur.astype(np.float64), f_prev.astype(np.float64), th,
                                O.Params(), prob.em_lambda())
    assert hits > 0 and st.guard_hits == hits
    assert rel_l2(out.cpu().numpy(), f_next) <= 1e-5


ODD_ORBITS = W.Geometry(18, 12, 27)  # 81 pixel orbits: the last pixel block is partial


@pytest.mark.parametrize("gk", ["64", RAGGED, SPARSE, ODD_ORBITS],
                         ids=["64", "ragged40", "sparse16", "orbits81"])
@pytest.mark.parametrize("bf16", [False, True], ids=["fp32", "bf16"])
def test_quarter_turn_fold(A, ctx, gk, bf16):
    # The Siddon matrices have the scanner's quarter-turn symmetry, so the
    # solver loop streams the folded halves of A and A^T; turned off, it
    # streams the whole matrices.  Both are the same method: images agree to
    # FP32 rounding of the sums, and both match the oracle.
    geom, Amat, sl = problem(gk)
    mf = A.Matrix(ctx, Amat, geom.n, geom.n_angles, bf16=bf16)
    mu = A.Matrix(ctx, Amat, geom.n, geom.n_angles, bf16=bf16, fold=False)
    try:
        assert mf.info().quarter_turn_folded == 1
        assert mu.info().quarter_turn_folded == 0
        kw = dict(max_iters=30, track_objective=1, beta=0.1,
                  a_precision=A.APPGA_PREC_BF16 if bf16 else A.APPGA_PREC_FP32)
        ff, sf = run_gpu(A, ctx, mf, sl, **kw)
        fu, su = run_gpu(A, ctx, mu, sl, **kw)
        assert sf.iters == su.iters == 30
        assert rel_l2(ff, fu) <= 2e-6
        assert abs(sf.phi - su.phi) <= 1e-9 * abs(su.phi)
        Aref = Amat
        if bf16:
            Aref = Amat.copy()
            Aref.data = bf16_round(Amat.data)
        prob, ref = run_oracle(geom, Aref, sl, max_iters=30, beta=0.1)
        assert rel_l2(ff, ref.f) <= 1e-5
        # the folded loop's resume continues an uninterrupted run bit for bit
        g, gamma = to_dev(sl.g), to_dev(sl.gamma)
        p = A.default_params(max_iters=30, beta=0.1, a_precision=kw["a_precision"])
        full = torch.empty(geom.d, dtype=torch.float32, device=DEV)
        A.appga_reconstruct(ctx.handle, mf.handle, g, gamma, None, p, full)
        f0 = torch.empty_like(full)
        A.appga_initial_image(ctx.handle, mf.handle, g, gamma, f0)
        p13 = A.default_params(max_iters=13, beta=0.1, a_precision=kw["a_precision"])
        p17 = A.default_params(max_iters=17, beta=0.1, a_precision=kw["a_precision"])
        a_prev, a_cur, out = (torch.empty_like(full) for _ in range(3))
        A.appga_resume(ctx.handle, mf.handle, g, gamma, f0, f0, 1, p13, a_prev, a_cur)
        A.appga_resume(ctx.handle, mf.handle, g, gamma, a_prev, a_cur, 14, p17, None, out)
        assert torch.equal(out, full)
    finally:
        mf.close()
        mu.close()


def test_quarter_turn_fold_only_where_it_holds(A, ctx, mats):
    assert mats["64"].info().quarter_turn_folded == 1
    assert mats[mkey(TINY)].info().quarter_turn_folded == 0  # odd side
    geom, Amat, sl = problem("64")
    B = Amat.copy()
    B.data = B.data.copy()
    B.data[12345] = np.nextafter(B.data[12345], np.float32(10.0))  # one value bit
    mb = A.Matrix(ctx, B, geom.n, geom.n_angles)
    try:
        assert mb.info().quarter_turn_folded == 0
        f, st = run_gpu(A, ctx, mb, sl, max_iters=20, beta=0.1)
        prob, ref = run_oracle(geom, B, sl, max_iters=20, beta=0.1)
        assert rel_l2(f, ref.f) <= 1e-5
    finally:
        mb.close()


def test_repeated_short_calls_replay_one_graph(A, ctx, mats):
    # a short call whose arguments repeat runs as one captured graph from its
    # second time on: the results and statistics stay those of the first
    # call bit for bit, inputs changed in place are read at each replay, and
    # a longer call in between (which regrows the momentum table) leaves
    # the short calls correct
    geom, Amat, sl = problem("64")
    mat = mats["64"]
    g, gamma = to_dev(sl.g), to_dev(sl.gamma)
    p = A.default_params(max_iters=20, track_objective=1)
    outs, stats = [], []
    for _ in range(4):
        out = torch.empty(geom.d, dtype=torch.float32, device=DEV)
        st = A.appga_reconstruct(ctx.handle, mat.handle, g, gamma, None, p, out)
        outs.append(out.clone())
        stats.append((st.iters, st.result_k, st.phi, st.phi_prev, st.guard_hits, st.flags))
    # the same output buffer each time
    out = torch.empty(geom.d, dtype=torch.float32, device=DEV)
    runs = []
    for _ in range(3):
        st = A.appga_reconstruct(ctx.handle, mat.handle, g, gamma, None, p, out)
        runs.append((out.clone(), st.phi, st.iters))
    for o, phi, it in runs:
        assert torch.equal(o, runs[0][0]) and phi == runs[0][1] and it == 20
    assert torch.equal(runs[0][0], outs[0])
    for st in stats[1:]:
        assert st == stats[0]
    # inputs changed in place are read at the next replay
    g2_host = (sl.g * 1.5).astype(np.float32)
    g.copy_(torch.from_numpy(g2_host).to(DEV))
    st2 = A.appga_reconstruct(ctx.handle, mat.handle, g, gamma, None, p, out)
    fresh = torch.empty_like(out)
    st_ref = A.appga_reconstruct(ctx.handle, mat.handle, to_dev(g2_host), gamma, None, p, fresh)
    assert torch.equal(out, fresh) and st2.phi == st_ref.phi
    # a long call regrows the momentum table; the short call stays correct
    A.appga_reconstruct(ctx.handle, mat.handle, g, gamma, None,
                        A.default_params(max_iters=1500), torch.empty_like(out))
    for _ in range(2):
        st3 = A.appga_reconstruct(ctx.handle, mat.handle, g, gamma, None, p, out)
        assert torch.equal(out, fresh) and st3.phi == st_ref.phi
    # the host-buffer entry point with a pinned result buffer
    gh = torch.from_numpy(g2_host).pin_memory()
    gamh = torch.from_numpy(sl.gamma).pin_memory()
    fh = torch.empty(geom.d, dtype=torch.float32).pin_memory()
    for _ in range(3):
        sth = A.appga_reconstruct_host(ctx.handle, mat.handle, gh, gamh, None, p, fh)
        np.testing.assert_array_equal(fh.numpy(), fresh.cpu().numpy())
        assert sth.phi == st_ref.phi


def test_resume_is_bitwise_continuation(A, ctx, mats):
    geom, Amat, sl = problem("64")
    mat = mats["64"]
    g, gamma = to_dev(sl.g), to_dev(sl.gamma)
    p40 = A.default_params(max_iters=40)
    full = torch.empty(geom.d, dtype=torch.float32, device=DEV)
    A.appga_reconstruct(ctx.handle, mat.handle, g, gamma, None, p40, full)
    p20 = A.default_params(max_iters=20)
    a_prev = torch.empty_like(full)
    a_cur = torch.empty_like(full)
    # first half from the initial image
    f_init = torch.empty_like(full)
    A.appga_initial_image(ctx.handle, mat.handle, g, gamma, f_init)
    st1 = A.appga_resume(ctx.handle, mat.handle, g, gamma, f_init, f_init, 1, p20, a_prev, a_cur)
    assert st1.result_k == 21
    out = torch.empty_like(full)
    st2 = A.appga_resume(ctx.handle, mat.handle, g, gamma, a_prev, a_cur, 21, p20, None, out)
    assert st2.result_k == 41
    assert torch.equal(out, full)


def test_deterministic_and_host_entry(A, ctx, mats):
    geom, Amat, sl = problem("64")
    mat = mats["64"]
    p = A.default_params(max_iters=25, track_objective=1)
    f1, s1 = run_gpu(A, ctx, mat, sl, max_iters=25, track_objective=1)
    f2, s2 = run_gpu(A, ctx, mat, sl, max_iters=25, track_objective=1)
    np.testing.assert_array_equal(f1, f2)
    assert s1.phi == s2.phi
    out = np.empty(geom.d, np.float32)
    s3 = A.appga_reconstruct_host(ctx.handle, mat.handle, sl.g, sl.gamma, None, p, out)
    np.testing.assert_array_equal(out, f1)
    assert s3.phi == s1.phi


@pytest.mark.parametrize("what", ["g_nan", "g_neg", "gamma_zero", "f_neg"])
def test_invalid_inputs_rejected(A, ctx, mats, what):
    geom, Amat, sl = problem("64")
    g = sl.g.copy()
    gamma = sl.gamma.copy()
    f_init = None
    if what == "g_nan":
        g[5] = np.nan
    elif what == "g_neg":
        g[5] = -1.0
    elif what == "gamma_zero":
        gamma[7] = 0.0
    else:
        f_init = to_dev(np.full(geom.d, -1.0, np.float32))
    p = A.default_params(max_iters=5)
    out = torch.empty(geom.d, dtype=torch.float32, device=DEV)
    with pytest.raises(A.AppgaError) as ei:
        A.appga_reconstruct(ctx.handle, mats["64"].handle, to_dev(g), to_dev(gamma), f_init, p, out)
    assert ei.value.status == A.APPGA_EDOMAIN
    # the context stays usable
    f, st = run_gpu(A, ctx, mats["64"], sl, max_iters=3)
    assert np.all(np.isfinite(f))


def test_bf16_matrix(A, ctx, mats):
    geom, Amat, sl = problem("64")
    f, _ = run_gpu(A, ctx, mats["64"], sl, max_iters=30, a_precision=1)
    _, ref32 = run_oracle(geom, Amat, sl, max_iters=30)
    Ab = sp.csr_matrix((bf16_round(Amat.data), Amat.indices, Amat.indptr), shape=Amat.shape)
    _, refb = run_oracle(geom, Ab, sl, max_iters=30)
    assert rel_l2(f, refb.f) <= 1e-5
    assert rel_l2(f, ref32.f) <= 1e-3


def test_kernel_times(A, ctx, mats):
    geom, Amat, sl = problem("64")
    p = A.default_params(track_objective=1)
    tp, tf = A.appga_kernel_times(ctx.handle, mats["64"].handle, to_dev(sl.g), to_dev(sl.gamma),
                                  p, 20)
    assert tp > 0 and tf > 0


# ------------------------------------------------- full-size (256^2) parity

@pytest.fixture(scope="module")
def m256(A, ctx):
    geom, Amat, _ = problem("256", counts=1e6)
    mat = A.Matrix(ctx, Amat, geom.n, geom.n_angles, bf16=True)
    yield mat
    mat.close()


def test_full_size_forward_and_backproject(A, ctx, m256):
    geom, Amat, sl = problem("256", counts=1e6, phantom="lesions")
    f = sl.f_true.astype(np.float32)
    y = torch.empty(geom.m, dtype=torch.float64, device=DEV)
    w = torch.empty(geom.m, dtype=torch.float32, device=DEV)
    A.appga_forward_ratio(ctx.handle, m256.handle, to_dev(f), to_dev(sl.g), to_dev(sl.gamma), y, w)
    bp = torch.empty(geom.d, dtype=torch.float32, device=DEV)
    A.appga_backproject(ctx.handle, m256.handle, w, bp)
    torch.cuda.synchronize()
    A64 = Amat.astype(np.float64)
    y_ref = A64 @ f.astype(np.float64)
    np.testing.assert_allclose(y.cpu().numpy(), y_ref, rtol=1e-11, atol=1e-300)
    wv = w.cpu().numpy().astype(np.float64)
    ref = A64.T @ wv
    assert np.all(np.abs(bp.cpu().numpy() - ref) <= 2e-6 * (A64.T @ np.abs(wv)) + 1e-30)


@pytest.mark.parametrize("counts,omega,iters,beta", [
    (1e6, 0.5, 500, 1.0),    # the benchmarked configuration
    (1e6, 1.0, 500, 1.0),
    (1e6, 0.25, 500, 1.0),
    (5e6, 1.0, 300, 0.1),
    (5e6, 0.5, 30, 1.0),
])
def test_full_size_trajectory(A, ctx, m256, counts, omega, iters, beta):
    # 256^2, 180 x 367, lesion phantom, objective tracked
    geom, Amat, sl = problem("256", counts=counts, phantom="lesions")
    f, st = run_gpu(A, ctx, m256, sl, max_iters=iters, omega=omega, beta=beta, track_objective=1)
    prob, ref = run_oracle(geom, Amat, sl, max_iters=iters, omega=omega, beta=beta)
    assert st.iters == iters
    assert rel_l2(f, ref.f) <= 1e-5
    phi_same = prob.objective(f.astype(np.float64), 0.1, 0.05, 1e-3)
    assert abs(st.phi - phi_same) <= 1e-9 * abs(phi_same)


@pytest.mark.parametrize("omega", [0.25, 1.0])
def test_full_size_5e6_beta1_500_maps(A, ctx, m256, omega):
    # 256^2 at 5e6 counts with beta = 1 over the workload's 500 maps.  The EM
    # step here breaks the step-size condition of Thm. 10 (p_max <= 1/L) and
    # the FP64 oracle itself does not fix the image to 1e-5 from FP32-sized
    # rounding: the oracle-side pin (tests/test_oracle.py) shows a 2^-24
    # perturbation of f^1 growing past 1e-5.  So the GPU's distance from the
    # oracle is bounded by a stated multiple (10x) of the oracle's own spread
    # under FP32-sized noise on every iterate, and the objective is compared.
    geom, Amat, sl = problem("256", counts=5e6, phantom="lesions")
    f, st = run_gpu(A, ctx, m256, sl, max_iters=500, omega=omega, track_objective=1)
    prob = O.Problem(Amat, sl.g, sl.gamma, geom.n)
    par = O.Params(max_iters=500, omega=omega)
    f0 = O.initial_image(sl.g, sl.gamma, geom.n, geom.n_angles)
    ref = O.appga(prob, par, f_init=f0, track_phi=False)
    noisy = oracle_fp32_noisy(prob, par, f0, seed=1)
    spread = rel_l2(noisy, ref.f)
    dist = rel_l2(f, ref.f)
    assert spread > 1e-6
    assert dist <= 10.0 * spread, (dist, spread)
    phi_ref = prob.objective(ref.f, 0.1, 0.05, 1e-3)
    phi_same = prob.objective(f.astype(np.float64), 0.1, 0.05, 1e-3)
    assert abs(st.phi - phi_same) <= 1e-9 * abs(phi_same)
    # the objective is flat where the trajectories part
    assert abs(st.phi - phi_ref) <= 1e-7 * abs(phi_ref)


def _bf16_matrix(Amat):
    return sp.csr_matrix((bf16_round(Amat.data), Amat.indices, Amat.indptr), shape=Amat.shape)


def test_full_size_bf16_single_slice(A, ctx, m256):
    # 256^2 with the BF16 copy of A (FP32 accumulation) over the benchmarked
    # 500-map run.  Against the FP64 oracle on the BF16-rounded matrix (the
    # method's arithmetic): 1e-5.  Against the FP64 oracle on the FP32 matrix
    # the distance includes the matrix rounding itself, which the two FP64
    # oracles alone already show: about 1.3e-3 after 100 maps and 1.8e-3 after
    # 500 here, above the 1e-3 that holds on the 64^2 grid over 30 maps.  The
    # GPU may add no more than the FP32 arithmetic's share to it.
    geom, Amat, sl = problem("256", counts=1e6, phantom="lesions")
    f, st = run_gpu(A, ctx, m256, sl, max_iters=500, a_precision=1, track_objective=1)
    _, ref32 = run_oracle(geom, Amat, sl, max_iters=500)
    Ab = _bf16_matrix(Amat)
    probb, refb = run_oracle(geom, Ab, sl, max_iters=500)
    rounding = rel_l2(refb.f, ref32.f)
    assert 1e-4 < rounding < 5e-3
    assert rel_l2(f, refb.f) <= 1e-5
    assert rel_l2(f, ref32.f) <= rounding + 2e-5
    phi_same = probb.objective(f.astype(np.float64), 0.1, 0.05, 1e-3)
    assert abs(st.phi - phi_same) <= 1e-9 * abs(phi_same)


def test_largest_geometry_single_slice_sampled(A, ctx):
    # 512^2, 360 x 731 (120.2M nnz): the largest workload geometry through the
    # single-slice solver; a few maps against the FP64 oracle, with the
    # objective tracked
    geom, Amat, sl = problem("512", counts=1e6, phantom="lesions")
    mat = A.Matrix(ctx, Amat, geom.n, geom.n_angles)
    try:
        # the Siddon matrix has the quarter-turn symmetry: the loop is folded
        assert mat.info().quarter_turn_folded == 1
        f, st = run_gpu(A, ctx, mat, sl, max_iters=4, omega=1.0, track_objective=1)
        prob, ref = run_oracle(geom, Amat, sl, max_iters=4, omega=1.0)
        assert st.iters == 4
        assert rel_l2(f, ref.f) <= 1e-5
        phi_same = prob.objective(f.astype(np.float64), 0.1, 0.05, 1e-3)
        assert abs(st.phi - phi_same) <= 1e-9 * abs(phi_same)
        # 30 maps folded and over the whole matrices agree to FP32 rounding
        mu = A.Matrix(ctx, Amat, geom.n, geom.n_angles, fold=False)
        try:
            assert mu.info().quarter_turn_folded == 0
            ff, sf = run_gpu(A, ctx, mat, sl, max_iters=30, omega=1.0, track_objective=1)
            fu, su = run_gpu(A, ctx, mu, sl, max_iters=30, omega=1.0, track_objective=1)
            assert rel_l2(ff, fu) <= 2e-6
            assert abs(sf.phi - su.phi) <= 1e-9 * abs(su.phi)
        finally:
            mu.close()
    finally:
        mat.close()


def test_objective_on_every_visible_device(A):
    # The double-float logarithm's constant tables and the kernels' function
    # attributes are set up per device on first use there: the objective of
    # the same inputs is the same on device 0 and on device 1 (where a second
    # device is visible; a one-GPU machine skips this).
    if torch.cuda.device_count() < 2:
        pytest.skip("one CUDA device visible")
    geom, Amat, sl = problem("64")
    vals = []
    for dev in (0, 1):
        c = A.Context(dev)
        mat = A.Matrix(c, Amat, geom.n, geom.n_angles)
        d = f"cuda:{dev}"
        f = torch.from_numpy(sl.f_true.astype(np.float32)).to(d)
        vals.append(A.appga_objective(c.handle, mat.handle, f, torch.from_numpy(sl.g).to(d),
                                      torch.from_numpy(sl.gamma).to(d), A.default_params()))
        mat.close()
        c.close()
    prob = O.Problem(Amat, sl.g, sl.gamma, geom.n)
    ref = prob.objective(sl.f_true.astype(np.float32).astype(np.float64), 0.1, 0.05, 1e-3)
    assert vals[0] == vals[1]
    assert abs(vals[1] - ref) <= 1e-9 * abs(ref)
