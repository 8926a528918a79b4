"""GPU parity of the batched (K slices, one matrix) solver through the C ABI:
every slice against the FP64 oracle, against the single-slice GPU path, and
independence of a slice's result from the rest of the batch."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import appga_oracle as O
from paper_2409_13344_gb300 import workload as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = "cuda:0"


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


def slices(geom, Amat, K, counts=None, config=3, phantom="ellipses"):
    rng = np.random.default_rng(99)
    if counts is None:
        counts = W.log_uniform_counts(rng, 5e4, 5e5, K)
    return [W.make_slice(Amat, geom, float(c), W.seed_for(config, i), phantom=phantom)
            for i, c in enumerate(counts)]


def run_batched(A, ctx, mat, sls, **kw):
    K = len(sls)
    g = torch.from_numpy(np.stack([s.g for s in sls])).to(DEV)
    gam = torch.from_numpy(np.stack([s.gamma for s in sls])).to(DEV)
    f = torch.empty((K, mat.d), dtype=torch.float32, device=DEV)
    p = A.default_params(**kw)
    st = A.appga_reconstruct_batched(ctx.handle, mat.handle, K, g, gam, None, p, f)
    return f.cpu().numpy(), st


def oracle(geom, Amat, sl, **kw):
    prob = O.Problem(Amat, sl.g, sl.gamma, geom.n)
    par = O.Params(**kw)
    return prob, O.appga(prob, par, n_angles=geom.n_angles, track_phi=par.rel_obj_tol > 0)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("K", [1, 3, 33, 100])
def test_batched_vs_oracle_64(A, ctx, K):
    geom, Amat, mat = matrix(A, ctx, "64")
    sls = slices(geom, Amat, K)
    f, st = run_batched(A, ctx, mat, sls, max_iters=30, omega=0.5, track_objective=1)
    check = range(K) if K <= 3 else [0, K // 2, K - 1]
    for i in check:
        prob, ref = oracle(geom, Amat, sls[i], max_iters=30, omega=0.5)
        assert st[i].iters == 30
        assert rel(f[i], ref.f) <= 1e-5, (i, rel(f[i], ref.f))
        phi_same = prob.objective(f[i].astype(np.float64), 0.1, 0.05, 1e-3)
        assert abs(st[i].phi - phi_same) <= 1e-9 * abs(phi_same)


def test_batched_matches_single_slice_path(A, ctx):
    geom, Amat, mat = matrix(A, ctx, "64")
    sls = slices(geom, Amat, 4)
    fb, _ = run_batched(A, ctx, mat, sls, max_iters=40, beta=0.1, omega=1.0)
    for i, sl in enumerate(sls):
        p = A.default_params(max_iters=40, beta=0.1, omega=1.0)
        out = torch.empty(geom.d, dtype=torch.float32, device=DEV)
        A.appga_reconstruct(ctx.handle, mat.handle, torch.from_numpy(sl.g).to(DEV),
                            torch.from_numpy(sl.gamma).to(DEV), None, p, out)
        assert rel(fb[i], out.cpu().numpy().astype(np.float64)) <= 2e-6


def test_slice_result_independent_of_batch_mates(A, ctx):
    # the same slice, alone among different batch mates, gives the same image
    geom, Amat, mat = matrix(A, ctx, "64")
    base = slices(geom, Amat, 6)
    other = slices(geom, Amat, 6, config=7)
    mix = [base[0], other[1], base[2], other[3], other[4], base[5]]
    f1, s1 = run_batched(A, ctx, mat, base, max_iters=25, track_objective=1)
    f2, s2 = run_batched(A, ctx, mat, mix, max_iters=25, track_objective=1)
    for i in (0, 2, 5):
        np.testing.assert_array_equal(f1[i], f2[i])
        assert s1[i].phi == s2[i].phi


def test_batched_ragged_geometry(A, ctx):
    geom = W.Geometry(40, 48, 59)
    geom, Amat, mat = matrix(A, ctx, geom)
    sls = slices(geom, Amat, 5, counts=[2e4, 3e4, 5e4, 1e4, 4e4])
    f, st = run_batched(A, ctx, mat, sls, max_iters=100, beta=0.03, omega=1.0)
    for i in range(5):
        _, ref = oracle(geom, Amat, sls[i], max_iters=100, beta=0.03, omega=1.0)
        assert rel(f[i], ref.f) <= 1e-5


def test_batched_per_slice_stopping(A, ctx):
    geom, Amat, mat = matrix(A, ctx, "64")
    sls = slices(geom, Amat, 4)
    f, st = run_batched(A, ctx, mat, sls, max_iters=400, beta=0.1, omega=1.0, rel_obj_tol=1e-6)
    iters = []
    for i in range(4):
        prob, ref = oracle(geom, Amat, sls[i], max_iters=400, beta=0.1, omega=1.0,
                           rel_obj_tol=1e-6)
        assert st[i].stopped_early == 1
        assert abs(st[i].iters - ref.iters) <= 1, (i, st[i].iters, ref.iters)
        # FP32 and FP64 objectives can fire the test one map apart: compare
        # with the oracle's iterate after the slice's own map count
        if st[i].iters != ref.iters:
            _, ref = oracle(geom, Amat, sls[i], max_iters=st[i].iters, beta=0.1, omega=1.0)
        assert rel(f[i], ref.f) <= 1e-5
        iters.append(st[i].iters)
    assert len(set(iters)) > 1  # slices really stop at different iterations


def test_batched_bf16(A, ctx):
    geom, Amat, mat = matrix(A, ctx, "64")
    sls = slices(geom, Amat, 3)
    f, _ = run_batched(A, ctx, mat, sls, max_iters=30, a_precision=1)
    u = Amat.data.view(np.uint32).astype(np.uint64)
    ub = (((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)).view(np.float32)
    Ab = sp.csr_matrix((ub, Amat.indices, Amat.indptr), shape=Amat.shape)
    for i in range(3):
        _, refb = oracle(geom, Ab, sls[i], max_iters=30)
        _, ref32 = oracle(geom, Amat, sls[i], max_iters=30)
        assert rel(f[i], refb.f) <= 1e-5
        assert rel(f[i], ref32.f) <= 1e-3


def test_batched_full_size_256(A, ctx):
    # 64 slices of 256^2 sharing one A, per-slice counts log-uniform 1e5..1e7
    geom, Amat, mat = matrix(A, ctx, "256")
    rng = np.random.default_rng(3)
    counts = W.log_uniform_counts(rng, 1e5, 1e7, 64)
    sls = slices(geom, Amat, 64, counts=counts, phantom="lesions")
    f, st = run_batched(A, ctx, mat, sls, max_iters=60, beta=0.1, omega=1.0, track_objective=1)
    for i in (0, 31, 63):
        prob, ref = oracle(geom, Amat, sls[i], max_iters=60, beta=0.1, omega=1.0)
        assert rel(f[i], ref.f) <= 1e-5, (i, rel(f[i], ref.f))
        phi_same = prob.objective(f[i].astype(np.float64), 0.1, 0.05, 1e-3)
        assert abs(st[i].phi - phi_same) <= 1e-9 * abs(phi_same)


def _bf16(Amat):
    u = Amat.data.view(np.uint32).astype(np.uint64)
    ub = (((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)).view(np.float32)
    return sp.csr_matrix((ub, Amat.indices, Amat.indptr), shape=Amat.shape)


def test_batched_full_size_256_bf16(A, ctx):
    # the benchmarked batch (64 slices of 256^2, counts 1e5..1e7) with the
    # BF16 copy of A: sampled slices against the FP64 oracle on the BF16-
    # rounded matrix (1e-5) and on the FP32 matrix (the matrix rounding's own
    # effect, measured between the two oracles, plus the arithmetic's share)
    geom, Amat, mat = matrix(A, ctx, "256")
    rng = np.random.default_rng(3)
    counts = W.log_uniform_counts(rng, 1e5, 1e7, 64)
    sls = slices(geom, Amat, 64, counts=counts, phantom="lesions")
    f, st = run_batched(A, ctx, mat, sls, max_iters=60, beta=0.1, omega=1.0, track_objective=1,
                        a_precision=1)
    Ab = _bf16(Amat)
    for i in (0, 40, 63):
        probb, refb = oracle(geom, Ab, sls[i], max_iters=60, beta=0.1, omega=1.0)
        _, ref32 = oracle(geom, Amat, sls[i], max_iters=60, beta=0.1, omega=1.0)
        rounding = rel(refb.f, ref32.f)
        assert rel(f[i], refb.f) <= 1e-5, (i, rel(f[i], refb.f))
        assert rel(f[i], ref32.f) <= rounding + 2e-5, (i, rel(f[i], ref32.f), rounding)
        phi_same = probb.objective(f[i].astype(np.float64), 0.1, 0.05, 1e-3)
        assert abs(st[i].phi - phi_same) <= 1e-9 * abs(phi_same)


def test_batched_large_512_bf16_sampled(A, ctx):
    # 120 slices of 512^2 with the BF16 copy of A (the large-batch leg's BF16
    # variant): a few maps, sampled slices against the BF16-matrix oracle
    geom, Amat, mat = matrix(A, ctx, "512")
    rng = np.random.default_rng(6)
    counts = W.log_uniform_counts(rng, 1e4, 1e7, 120)
    picks = {3: None, 118: None}
    for i in picks:
        picks[i] = W.make_slice(Amat, geom, float(counts[i]), W.seed_for(5, i), phantom="lesions")
    base = W.make_slice(Amat, geom, 1e6, W.seed_for(5, 1001), phantom="lesions")
    sls = [picks.get(i, base) for i in range(120)]
    f, st = run_batched(A, ctx, mat, sls, max_iters=3, omega=1.0, a_precision=1)
    Ab = _bf16(Amat)
    for i, sl in picks.items():
        _, refb = oracle(geom, Ab, sl, max_iters=3, omega=1.0)
        assert st[i].iters == 3
        assert rel(f[i], refb.f) <= 1e-5, (i, rel(f[i], refb.f))


def test_batched_rejects_bad_input(A, ctx):
    geom, Amat, mat = matrix(A, ctx, "64")
    sls = slices(geom, Amat, 2)
    sls[1].g[3] = np.nan
    with pytest.raises(A.AppgaError) as ei:
        run_batched(A, ctx, mat, sls, max_iters=5)
    assert ei.value.status == A.APPGA_EDOMAIN


def _reset_schedule(A, mat, K, prec=0):
    A.appga_batch_schedule_set(mat.handle, A.appga_batch_tuning(K=K, a_precision=prec))


def test_launch_schedule_never_changes_images(A, ctx):
    # sub-batches, SpMV / back-projection / stencil grids: the same images bit for bit
    geom, Amat, mat = matrix(A, ctx, "64")
    sls = slices(geom, Amat, 40)
    f0, _ = run_batched(A, ctx, mat, sls, max_iters=20, omega=1.0)
    try:
        for sch in (dict(chunk=32), dict(spmv_per_sm=3, pixel_per_sm=5, stencil_per_sm=1),
                    dict(chunk=32, spmv_per_sm=16, pixel_per_sm=16, stencil_per_sm=16),
                    dict(gather_rows_fw=4), dict(gather_rows_px=4),
                    dict(chunk=32, gather_rows_fw=4, gather_rows_px=4, spmv_per_sm=5)):
            A.appga_batch_schedule_set(mat.handle, A.appga_batch_tuning(K=40, a_precision=0, **sch))
            got = A.appga_batch_schedule_get(mat.handle, 40)
            assert (got.chunk, got.spmv_per_sm) == (sch.get("chunk", 0), sch.get("spmv_per_sm", 0))
            assert (got.gather_rows_fw, got.gather_rows_px) == (sch.get("gather_rows_fw", 0),
                                                                sch.get("gather_rows_px", 0))
            f1, _ = run_batched(A, ctx, mat, sls, max_iters=20, omega=1.0)
            np.testing.assert_array_equal(f1, f0)
    finally:
        _reset_schedule(A, mat, 40)


def test_autotune_batched(A, ctx):
    geom, Amat, mat = matrix(A, ctx, "128")
    sls = slices(geom, Amat, 64)
    g = torch.from_numpy(np.stack([s.g for s in sls])).to(DEV)
    gam = torch.from_numpy(np.stack([s.gamma for s in sls])).to(DEV)
    f0, _ = run_batched(A, ctx, mat, sls, max_iters=12)
    try:
        t = A.appga_autotune_batched(ctx.handle, mat.handle, 64, g, gam, A.default_params())
        assert t.K == 64 and 0 < t.us_per_slice_iter <= t.us_per_slice_iter_default
        kept = A.appga_batch_schedule_get(mat.handle, 64)
        assert (kept.spmv_per_sm, kept.stencil_per_sm, kept.pixel_per_sm, kept.chunk) == (
            t.spmv_per_sm, t.stencil_per_sm, t.pixel_per_sm, t.chunk)
        assert t.gather_rows_fw in (4, 8) and t.gather_rows_px in (4, 8)
        assert (kept.gather_rows_fw or 8, kept.gather_rows_px or 8) == (t.gather_rows_fw,
                                                                        t.gather_rows_px)
        f1, _ = run_batched(A, ctx, mat, sls, max_iters=12)
        np.testing.assert_array_equal(f1, f0)
    finally:
        _reset_schedule(A, mat, 64)


def test_batch_schedule_rejects_bad_values(A, ctx):
    geom, Amat, mat = matrix(A, ctx, "64")
    for bad in (dict(K=0), dict(K=129), dict(K=8, chunk=48), dict(K=8, spmv_per_sm=17),
                dict(K=8, pixel_per_sm=-1), dict(K=8, a_precision=3),
                dict(K=8, gather_rows_fw=6), dict(K=8, gather_rows_px=16)):
        with pytest.raises(A.AppgaError) as ei:
            A.appga_batch_schedule_set(mat.handle, A.appga_batch_tuning(**bad))
        assert ei.value.status == A.APPGA_EINVAL


def test_batched_large_512_sampled(A, ctx):
    # 120 slices of 512^2 (360 x 731, 120.2M nnz) in one batch (Kp = 128),
    # dynamic-frame counts 1e4..1e7, omega 1: a few maps, sampled slices
    # against the FP64 oracle
    geom, Amat, mat = matrix(A, ctx, "512")
    rng = np.random.default_rng(5)
    counts = W.log_uniform_counts(rng, 1e4, 1e7, 120)
    picks = {0: None, 77: None, 119: None}
    for i in picks:
        picks[i] = W.make_slice(Amat, geom, float(counts[i]), W.seed_for(5, i), phantom="lesions")
    base = W.make_slice(Amat, geom, 1e6, W.seed_for(5, 1000), phantom="lesions")
    sls = [picks.get(i, base) for i in range(120)]
    f, st = run_batched(A, ctx, mat, sls, max_iters=3, omega=1.0)
    for i, sl in picks.items():
        _, ref = oracle(geom, Amat, sl, max_iters=3, omega=1.0)
        assert st[i].iters == 3
        assert rel(f[i], ref.f) <= 1e-5, (i, rel(f[i], ref.f))


def test_gather_probe(A, ctx):
    """The gather-bandwidth probe runs for every width and rejects others."""
    geom, Amat, mat = matrix(A, ctx, "64")
    for w in (32, 64, 128):
        fwd, bwd = A.appga_gather_probe(ctx.handle, mat.handle, w, 3)
        assert np.isfinite(fwd) and fwd > 0 and np.isfinite(bwd) and bwd > 0
    with pytest.raises(A.AppgaError):
        A.appga_gather_probe(ctx.handle, mat.handle, 48, 3)
    with pytest.raises(A.AppgaError):
        A.appga_gather_probe(ctx.handle, mat.handle, 64, 0)


def test_batched_slot_width_guard_at_the_limit(A, ctx):
    # The batched kernels stage col * Kp in 32 bits, so max(m, d) * Kp must stay
    # below 2^31.  A 4100^2 image (d = 16.81M) crossed by one horizontal ray:
    # K = 128 (Kp = 128, d * Kp = 2.15e9) is rejected on the host before any
    # device work; K = 64 (d * Kp = 1.08e9) runs and agrees with the
    # single-slice path, which has no such limit.
    n = 4100
    d = n * n
    col = (2050 * n + np.arange(n)).astype(np.int32)
    Amat = sp.csr_matrix((np.ones(n, np.float32), col, np.array([0, n], np.int32)), shape=(1, d))
    mat = A.Matrix(ctx, Amat, n, 1)
    try:
        g1 = torch.tensor([[2.0e4]], dtype=torch.float32, device=DEV)
        gam1 = torch.tensor([[50.0]], dtype=torch.float32, device=DEV)
        # a small step: one ray against a 13M-pixel initial disk makes the
        # EM step scale the ray's pixels by ~180 at beta = 1, which would
        # amplify the FP32 summation-order difference between the two paths
        p = A.default_params(max_iters=2, omega=1.0, beta=1e-3)
        # a full-size output even for the rejected call (8.6 GB)
        fbuf = torch.empty((128, d), dtype=torch.float32, device=DEV)
        with pytest.raises(A.AppgaError) as ei:
            A.appga_reconstruct_batched(ctx.handle, mat.handle, 128, g1.expand(128, 1).contiguous(),
                                        gam1.expand(128, 1).contiguous(), None, p, fbuf)
        assert ei.value.status == A.APPGA_EINVAL
        K = 64
        f = fbuf[:K]
        st = A.appga_reconstruct_batched(ctx.handle, mat.handle, K, g1.expand(K, 1).contiguous(),
                                         gam1.expand(K, 1).contiguous(), None, p, f)
        assert all(s.iters == 2 for s in st)
        one = torch.empty(d, dtype=torch.float32, device=DEV)
        A.appga_reconstruct(ctx.handle, mat.handle, g1[0], gam1[0], None, p, one)
        ref = one.cpu().numpy().astype(np.float64)
        for i in (0, K - 1):
            got = f[i].cpu().numpy()
            assert np.all(np.isfinite(got))
            assert rel(got, ref) <= 2e-6
            assert rel(got.reshape(n, n)[2050], ref.reshape(n, n)[2050]) <= 1e-5
        # the ray's row moved, the pixels far from it and from the disk edge did not
        ray = ref.reshape(n, n)[2050]
        far = ref.reshape(n, n)[1000, 2040:2060]
        assert np.ptp(far) == 0.0 and abs(ray[2050] - far[0]) > 1e-3 * far[0]
        del f, fbuf
    finally:
        mat.close()
