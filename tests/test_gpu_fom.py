"""GPU figures of merit (Sec. 4.1) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

from oracle import figures_of_merit as F

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


@pytest.mark.parametrize("n", [64, 256, 400])
def test_fom_matches_oracle(A, ctx, n):
    rng = np.random.default_rng(n)
    d = n * n
    t = rng.uniform(0.5, 4.0, d).astype(np.float32)
    f = (t * rng.uniform(0.8, 1.2, d) + rng.normal(0, 0.05, d)).astype(np.float32)
    h = F.disk_roi(n, n / 6, -n / 8, n / 20)
    b = F.disk_roi(n, -n / 5, n / 7, n / 20)
    t[h] *= 4.0  # a hot region
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(DEV)
    got = A.appga_figures_of_merit(ctx.handle, d, dev(f), dev(t), dev(h.astype(np.uint8)),
                                   dev(b.astype(np.uint8)), float(t.max()))
    f64, t64 = f.astype(np.float64), t.astype(np.float64)
    assert got.mse == pytest.approx(F.mse(f64, t64), rel=1e-12)
    assert got.psnr == pytest.approx(F.psnr(f64, t64, float(t.max())), abs=1e-10)
    assert got.rc == pytest.approx(F.relative_contrast(f64, h, b), rel=1e-12)
    assert got.rc_true == pytest.approx(F.relative_contrast(t64, h, b), rel=1e-12)
    assert got.nrc == pytest.approx(F.nrc(f64, t64, h, b), rel=1e-12)
    assert (got.n_roi_h, got.n_roi_b) == (int(h.sum()), int(b.sum()))
    out = torch.empty(n, dtype=torch.float32, device=DEV)
    A.appga_central_line_profile(ctx.handle, n, dev(f), out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), F.central_line_profile(f, n).astype(np.float32))


def test_fom_without_regions_and_identical_images(A, ctx):
    t = torch.rand(4096, device=DEV) + 0.5
    got = A.appga_figures_of_merit(ctx.handle, 4096, t, t, None, None, 2.0)
    assert got.mse == 0.0 and got.psnr == float("inf")
    assert np.isnan(got.rc) and np.isnan(got.nrc)


def test_fom_rejects_bad_arguments(A, ctx):
    t = torch.ones(16, device=DEV)
    m = torch.ones(16, dtype=torch.uint8, device=DEV)
    for args in ((0, t, t, None, None, 1.0), (16, t, t, m, None, 1.0), (16, t, t, None, None, 0.0)):
        with pytest.raises(A.AppgaError) as ei:
            A.appga_figures_of_merit(ctx.handle, *args)
        assert ei.value.status == A.APPGA_EINVAL
