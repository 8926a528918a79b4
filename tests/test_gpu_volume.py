"""GPU parity of the 3-D SHOITV path through the C ABI against the FP64 oracle
(oracle/hoitv3d_oracle.py): the stand-alone 3-D gradient and regulariser,
APPGA on volumes (several z-tiles with a ragged last tile, padded slot
widths), the joint stopping test, one slice against the 2-D paths, and a
sampled check of one map on the 64-slice 256 x 256 volume the benchmark
times.

Tolerances: the FP32 3-D stencil as the 2-D one, |err| <= 4e-6 (lam1 + lam2)
+ 1e-5 |ref| (twelve fields and their adjoints instead of six); the
regulariser value (double-float sums of FP32 terms) rel 2e-6; images after
APPGA maps rel L2 1e-5; the volume's Phi on identical images rel 1e-9.
"""
import numpy as np
import pytest

from oracle import appga_oracle as O
from oracle import hoitv3d_oracle as H
from paper_2409_13344_gb300 import workload as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = "cuda:0"
RAGGED = W.Geometry(40, 48, 59)


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


_mats = {}


def matrix(A, ctx, name):
    if name not in _mats:
        geom = W.GEOMETRIES[name] if isinstance(name, str) else name
        Amat = W.system_matrix(name) if isinstance(name, str) else W.siddon_matrix(geom)
        _mats[name] = (geom, Amat, A.Matrix(ctx, Amat, geom.n, geom.n_angles, bf16=True))
    return _mats[name]


def dev(x, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype).to(DEV)


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def grad3d(A, ctx, V, lam1, lam2, eps):
    nz, n, _ = V.shape
    out = torch.empty(V.size, dtype=torch.float32, device=DEV)
    reg = torch.zeros(1, dtype=torch.float64, device=DEV)
    A.appga_shoitv3d_grad(ctx.handle, n, nz, dev(V.reshape(-1)), lam1, lam2, eps, out, reg)
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(V.shape), float(reg.item())


# ------------------------------------------------------- stand-alone stencil

@pytest.mark.parametrize("nz,n,eps", [(1, 37, 1e-3), (5, 33, 1e-3), (11, 40, 0.05),
                                      (17, 64, 1e-3), (128, 24, 1e-2)])
def test_stencil3d_against_oracle(A, ctx, nz, n, eps):
    rng = np.random.default_rng(nz * 100 + n)
    V = rng.uniform(0.0, 1.0, (nz, n, n))
    V[: max(1, nz // 2), : n // 2, : n // 3] = 0.25    # flat block: quadratic branch of s_eps
    V = V.astype(np.float32)
    lam1, lam2 = 0.1, 0.05
    got, reg = grad3d(A, ctx, V, lam1, lam2, eps)
    R = H.Regulariser3D(nz, n)
    V64 = V.astype(np.float64)
    ref = R.grad(V64, lam1, lam2, eps).reshape(V.shape)
    err = np.abs(got - ref)
    assert np.all(err <= 4e-6 * (lam1 + lam2) + 1e-5 * np.abs(ref)), float(err.max())
    ref_val = R.value(V64, lam1, lam2, eps)
    assert abs(reg - ref_val) <= 2e-6 * abs(ref_val), (reg, ref_val)


def test_stencil3d_one_slice_is_2d(A, ctx):
    n = 45
    rng = np.random.default_rng(3)
    F = rng.uniform(0.0, 2.0, (1, n, n)).astype(np.float32)
    got, _ = grad3d(A, ctx, F, 0.2, 0.1, 1e-2)
    out2 = torch.empty(n * n, dtype=torch.float32, device=DEV)
    A.appga_shoitv_grad(ctx.handle, n, dev(F.reshape(-1)), 0.2, 0.1, 1e-2, out2)
    torch.cuda.synchronize()
    np.testing.assert_allclose(got.reshape(-1), out2.cpu().numpy(), rtol=1e-5, atol=1e-6)


def test_stencil3d_axis_swap(A, ctx):
    # a cube with r and z swapped gives the swapped gradient (the component
    # set is closed under axis permutations)
    n = 24
    rng = np.random.default_rng(6)
    V = rng.uniform(0.0, 1.0, (n, n, n)).astype(np.float32)
    g0, r0 = grad3d(A, ctx, V, 0.2, 0.3, 1e-2)
    g1, r1 = grad3d(A, ctx, np.ascontiguousarray(np.transpose(V, (1, 0, 2))), 0.2, 0.3, 1e-2)
    np.testing.assert_allclose(np.transpose(g1, (1, 0, 2)), g0, rtol=0, atol=4e-6)
    assert abs(r0 - r1) <= 2e-6 * abs(r0)


def test_stencil3d_rejects_bad_sizes(A, ctx):
    V = torch.zeros(8 * 8 * 2, dtype=torch.float32, device=DEV)
    out = torch.empty_like(V)
    for n_side, nz, eps in ((8, 0, 1e-3), (8, 129, 1e-3), (0, 2, 1e-3), (8, 2, 0.0)):
        with pytest.raises(A.AppgaError):
            A.appga_shoitv3d_grad(ctx.handle, n_side, nz, V, 0.1, 0.05, eps, out)


# ---------------------------------------------------------------- solver

def volume_problem(A, ctx, geom_key, nz, counts, seed_slice=0):
    geom, Amat, mat = matrix(A, ctx, geom_key)
    vol = W.make_volume(Amat, geom, nz, counts, W.seed_for(6, seed_slice))
    return geom, Amat, mat, vol


def run_volume(A, ctx, mat, vol, **kw):
    nz = vol.g.shape[0]
    f = torch.empty((nz, mat.d), dtype=torch.float32, device=DEV)
    p = A.default_params(**kw)
    st = A.appga_reconstruct_volume(ctx.handle, mat.handle, nz, dev(vol.g), dev(vol.gamma), None,
                                    p, f)
    torch.cuda.synchronize()
    return f.cpu().numpy(), st


@pytest.mark.parametrize("gk,nz,iters,beta", [("64", 5, 30, 1.0), ("64", 33, 12, 1.0),
                                               (RAGGED, 9, 40, 0.1)],
                         ids=["64x5", "64x33", "ragged40x9"])
def test_volume_against_oracle(A, ctx, gk, nz, iters, beta):
    geom, Amat, mat, vol = volume_problem(A, ctx, gk, nz, 8e4 * nz)
    f, st = run_volume(A, ctx, mat, vol, max_iters=iters, beta=beta, omega=0.5,
                       track_objective=1)
    prob = H.VolumeProblem(Amat, vol.g, vol.gamma, geom.n)
    ref = H.appga_volume(prob, O.Params(max_iters=iters, beta=beta, omega=0.5),
                         n_angles=geom.n_angles, track_phi=False)
    assert st.iters == iters and st.result_k == iters + 1 and not st.stopped_early
    assert rel_l2(f, ref.f) <= 1e-5, rel_l2(f, ref.f)
    for z in (0, nz // 2, nz - 1):
        assert rel_l2(f[z], ref.f[z]) <= 1e-5
    phi_same = prob.objective(f.astype(np.float64), 0.1, 0.05, 1e-3)
    assert abs(st.phi - phi_same) <= 1e-9 * abs(phi_same), (st.phi, phi_same)


def test_volume_joint_stop_matches_oracle(A, ctx):
    geom, Amat, mat, vol = volume_problem(A, ctx, "64", 6, 5e5, seed_slice=1)
    tol = 1e-6
    prob = H.VolumeProblem(Amat, vol.g, vol.gamma, geom.n)
    ref = H.appga_volume(prob, O.Params(max_iters=400, beta=0.5, omega=1.0, rel_obj_tol=tol),
                         n_angles=geom.n_angles)
    assert ref.iters < 400
    # the oracle's stopping decision is not within rounding of the tolerance
    ratios = [abs(ref.phi[i + 1] - ref.phi[i]) / abs(ref.phi[i]) for i in range(len(ref.phi) - 1)]
    assert all(abs(r / tol - 1.0) > 1e-3 for r in ratios)
    f, st = run_volume(A, ctx, mat, vol, max_iters=400, beta=0.5, omega=1.0, rel_obj_tol=tol)
    assert st.stopped_early == 1
    assert st.iters == ref.iters, (st.iters, ref.iters)
    assert rel_l2(f, ref.f) <= 1e-5
    phi_same = prob.objective(f.astype(np.float64), 0.1, 0.05, 1e-3)
    assert abs(st.phi - phi_same) <= 1e-9 * abs(phi_same)


def test_volume_one_slice_matches_single_slice_solver(A, ctx):
    geom, Amat, mat, vol = volume_problem(A, ctx, "64", 1, 1e5, seed_slice=2)
    f, st = run_volume(A, ctx, mat, vol, max_iters=25, track_objective=1)
    out = torch.empty(mat.d, dtype=torch.float32, device=DEV)
    p = A.default_params(max_iters=25, track_objective=1)
    st2 = A.appga_reconstruct(ctx.handle, mat.handle, dev(vol.g[0]), dev(vol.gamma[0]), None, p, out)
    torch.cuda.synchronize()
    assert rel_l2(f[0], out.cpu().numpy().astype(np.float64)) <= 2e-6
    assert abs(st.phi - st2.phi) <= 1e-9 * abs(st2.phi)


def test_volume_deterministic_and_zero_iterations(A, ctx):
    geom, Amat, mat, vol = volume_problem(A, ctx, "64", 7, 3e5, seed_slice=3)
    f1, _ = run_volume(A, ctx, mat, vol, max_iters=15)
    f2, _ = run_volume(A, ctx, mat, vol, max_iters=15)
    assert np.array_equal(f1, f2)
    f0, st0 = run_volume(A, ctx, mat, vol, max_iters=0)
    prob = H.VolumeProblem(Amat, vol.g, vol.gamma, geom.n)
    init = H.initial_volume(prob, geom.n_angles)
    assert st0.iters == 0
    np.testing.assert_allclose(f0, init, rtol=1e-6, atol=1e-12)


def test_volume_rejects_bad_arguments(A, ctx):
    geom, Amat, mat, vol = volume_problem(A, ctx, "64", 2, 1e5)
    f = torch.empty((129, mat.d), dtype=torch.float32, device=DEV)
    g = torch.ones((129, mat.m), dtype=torch.float32, device=DEV)
    with pytest.raises(A.AppgaError):
        A.appga_reconstruct_volume(ctx.handle, mat.handle, 129, g, g, None,
                                   A.default_params(max_iters=1), f)
    bad = vol.gamma.copy()
    bad[1, 5] = 0.0
    with pytest.raises(A.AppgaError):
        A.appga_reconstruct_volume(ctx.handle, mat.handle, 2, dev(vol.g), dev(bad), None,
                                   A.default_params(max_iters=1), f[:2])


# ------------------------------------------ full size: 64 slices of 256 x 256

def _box(V, z, r, c, h=3):
    nz, n, _ = V.shape
    z0, z1 = max(0, z - h), min(nz, z + h + 1)
    r0, r1 = max(0, r - h), min(n, r + h + 1)
    c0, c1 = max(0, c - h), min(n, c + h + 1)
    return V[z0:z1, r0:r1, c0:c1], (z - z0, r - r0, c - c0)


def _sample_voxels(nz, n, rng, k=120):
    pts = [(0, 0, 0), (nz - 1, n - 1, n - 1), (0, n - 1, 0), (nz - 1, 0, n - 1),
           (nz // 2, 0, n // 2), (nz // 2, n // 2, n - 1), (1, 1, 1), (nz - 2, n - 2, n - 2)]
    pts += [tuple(int(v) for v in (rng.integers(nz), rng.integers(n), rng.integers(n)))
            for _ in range(k)]
    return pts


def _local_grad(V, z, r, c, lam1, lam2, eps):
    """The oracle's gradient at one voxel from the box within 3 voxels of it:
    the box edges that are not volume edges lie beyond the stencil's reach."""
    box, (bz, br, bc) = _box(V, z, r, c)
    R = H.Regulariser3D(*box.shape)
    return R.grad(box, lam1, lam2, eps).reshape(box.shape)[bz, br, bc]


def test_full_size_one_map_sampled(A, ctx):
    nz = 64
    geom, Amat, mat, vol = volume_problem(A, ctx, "256", nz, 6.4e7, seed_slice=4)
    f, st = run_volume(A, ctx, mat, vol, max_iters=1)
    assert st.iters == 1
    n, d = geom.n, geom.d
    # f^2 = max(f~ - beta (f^1/Lambda)(A^T w + grad R), 0) with f~ = f^1 (theta_1 = 0);
    # the slices' data terms from the 2-D oracle, the 3-D gradient from boxes
    f1 = np.stack([O.initial_image(vol.g[z], vol.gamma[z], n, geom.n_angles) for z in range(nz)])
    probs = {}
    V = f1.reshape(nz, n, n)
    rng = np.random.default_rng(11)
    pts = _sample_voxels(nz, n, rng)
    gradF = {}
    for z in sorted({p[0] for p in pts}):
        prob = O.Problem(Amat, vol.g[z], vol.gamma[z], n) if not probs else probs[0]
        probs.setdefault(0, prob)
        y = prob.A @ f1[z]
        gam = vol.gamma[z].astype(np.float64)
        den = np.maximum(y + gam, O.KAPPA * gam)
        gradF[z] = prob.At @ (1.0 - vol.g[z].astype(np.float64) / den)
    lam = probs[0].em_lambda()
    scale = np.max(np.abs(f1))
    for (z, r, c) in pts:
        j = r * n + c
        gR = _local_grad(V, z, r, c, 0.1, 0.05, 1e-3)
        ref = max(f1[z, j] - 1.0 * f1[z, j] / lam[j] * (gradF[z][j] + gR), 0.0)
        assert abs(f[z, j] - ref) <= 1e-5 * scale, (z, r, c, f[z, j], ref)


def test_full_size_stencil_sampled(A, ctx):
    nz, n = 64, 256
    rng = np.random.default_rng(21)
    V = rng.uniform(0.0, 1.0, (nz, n, n)).astype(np.float32)
    V[:, 100:140, 60:200] = 0.5
    got, _ = grad3d(A, ctx, V, 0.1, 0.05, 1e-3)
    V64 = V.astype(np.float64)
    for (z, r, c) in _sample_voxels(nz, n, rng):
        ref = _local_grad(V64, z, r, c, 0.1, 0.05, 1e-3)
        assert abs(got[z, r, c] - ref) <= 4e-6 * 0.15 + 1e-5 * abs(ref), (z, r, c)
