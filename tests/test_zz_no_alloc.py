"""appga_objective_noalloc: the objective evaluation for callers that cannot
let the library allocate device memory (a process whose own pool owns all of
device memory, or a real-time loop that forbids allocation once running).
It must give the same Phi(f) as appga_objective, call after call, using only
the caller's buffers and the library's fixed scratch array.

This file is collected last on purpose: it runs after every other test in a
full run, and must also pass alone in a fresh process."""
import numpy as np
import pytest

from paper_2409_13344_gb300 import workload as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = "cuda:0"


@pytest.fixture(scope="module")
def lib():
    from paper_2409_13344_gb300 import build
    build.build()
    from paper_2409_13344_gb300 import appga
    if not torch.cuda.is_available():
        pytest.fail("the -m gpu tests need a CUDA device")
    return appga


@pytest.fixture(scope="module")
def ctx(lib):
    c = lib.Context(0)
    yield c
    c.close()


# 512 x 512 (360 x 731 bins) is the largest size the fixed scratch serves
@pytest.mark.parametrize("name,counts", [("64", 1e5), ("256", 1e6), ("512", 1e6)])
def test_noalloc_objective_matches_allocating_call_twice(lib, ctx, name, counts):
    geom = W.GEOMETRIES[name]
    A = W.system_matrix(name)
    sl = W.make_slice(A, geom, counts, W.seed_for(2))
    mat = lib.Matrix(ctx, A, geom.n, geom.n_angles)
    rng = np.random.default_rng(1)
    f = torch.from_numpy((sl.f_true * rng.uniform(0.9, 1.1, geom.d)).astype(np.float32)).to(DEV)
    g = torch.from_numpy(sl.g).to(DEV)
    gamma = torch.from_numpy(sl.gamma).to(DEV)
    p = lib.default_params()
    ref = lib.appga_objective(ctx.handle, mat.handle, f, g, gamma, p)
    out = torch.full((2,), float("nan"), dtype=torch.float64, device=DEV)
    lib.appga_objective_noalloc(ctx.handle, mat.handle, f, g, gamma, p, out[0:1])
    lib.appga_objective_noalloc(ctx.handle, mat.handle, f, g, gamma, p, out[1:2])
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    # same kernels, same reduction order: the values agree to the tests'
    # objective tolerance (in practice bit for bit)
    assert abs(got[0] - ref) <= 1e-12 * abs(ref)
    assert abs(got[1] - ref) <= 1e-12 * abs(ref)
    mat.close()


def test_noalloc_rejects_matrices_beyond_the_fixed_scratch(lib, ctx):
    # a 2048 x 2048 image (a few rays suffice) needs more scratch than the
    # fixed array holds: its stencil blocks alone leave more block partials
    # than fit
    n, m = 2048, 4
    row_ptr = np.array([0, 2, 3, 3, 4], np.int32)
    col = np.array([0, 5, 7, n * n - 1], np.int32)
    val = np.ones(4, np.float32)
    handle = lib.appga_matrix_create(ctx.handle, m, n * n, n, 4, row_ptr, col, val)
    f = torch.zeros(n * n, dtype=torch.float32, device=DEV)
    g = torch.ones(m, dtype=torch.float32, device=DEV)
    out = torch.zeros(1, dtype=torch.float64, device=DEV)
    with pytest.raises(lib.AppgaError) as ei:
        lib.appga_objective_noalloc(ctx.handle, handle, f, g, g, lib.default_params(), out)
    assert ei.value.status == lib.APPGA_EINVAL
    assert "scratch" in str(ei.value)
    lib.appga_matrix_destroy(handle)
