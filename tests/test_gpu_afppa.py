"""GPU AFPPA / FPPA for the non-smooth HOITV model (Sec. 4.4 extension of the
GN momentum) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

from oracle import afppa_oracle as AF
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


def setup(A, ctx, name, counts=1e5):
    if name not in _mats:
        geom = W.GEOMETRIES[name] if isinstance(name, str) else name
        Amat = W.system_matrix(name) if isinstance(name, str) else W.siddon_matrix(geom)
        _mats[name] = (geom, Amat, A.Matrix(ctx, Amat, geom.n, geom.n_angles))
    geom, Amat, mat = _mats[name]
    sl = W.make_slice(Amat, geom, counts, W.seed_for(6), phantom="lesions")
    return geom, Amat, mat, sl


def run(A, ctx, geom, mat, sl, **kw):
    d = geom.d
    f = torch.empty(d, dtype=torch.float32, device=DEV)
    b = torch.empty(2 * d, dtype=torch.float32, device=DEV)
    c = torch.empty(4 * d, dtype=torch.float32, device=DEV)
    st = A.appga_afppa_reconstruct(ctx.handle, mat.handle, torch.from_numpy(sl.g).to(DEV),
                                   torch.from_numpy(sl.gamma).to(DEV), None,
                                   A.default_params(**kw), f, b, c)
    return f.cpu().numpy(), b.cpu().numpy(), c.cpu().numpy(), st


def oracle(geom, Amat, sl, **kw):
    prob = O.Problem(Amat, sl.g, sl.gamma, geom.n)
    return AF.afppa(prob, O.Params(**kw), n_angles=geom.n_angles)


def rel(a, b):
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


CASES = [dict(momentum=1, mname="none", omega=0.5),
         dict(momentum=0, mname="gn", omega=0.5),
         dict(momentum=0, mname="gn", omega=0.25),
         dict(momentum=2, mname="nesterov", omega=0.5)]


@pytest.mark.parametrize("case", CASES, ids=["fppa", "gn0.5", "gn0.25", "nesterov"])
@pytest.mark.parametrize("name", ["64", W.Geometry(40, 48, 59)], ids=["64", "ragged40"])
def test_afppa_matches_oracle(A, ctx, case, name):
    geom, Amat, mat, sl = setup(A, ctx, name)
    kw = dict(lambda1=0.05, lambda2=0.02, beta=0.3, max_iters=30, omega=case["omega"])
    f, b, c, st = run(A, ctx, geom, mat, sl, momentum=case["momentum"], **kw)
    ref = oracle(geom, Amat, sl, momentum=case["mname"], **kw)
    assert st.iters == 30
    assert rel(f, ref.f) <= 1e-5, rel(f, ref.f)
    assert rel(b, ref.b) <= 1e-5 and rel(c, ref.c) <= 1e-5, (rel(b, ref.b), rel(c, ref.c))
    assert st.re == pytest.approx(ref.re[-1], rel=1e-3)
    assert st.rho1 == pytest.approx(ref.rho1[-1], rel=1e-6)
    assert st.rho2 == pytest.approx(ref.rho2[-1], rel=1e-6)
    d = geom.d
    assert np.hypot(b[:d], b[d:]).max() <= 0.05 * (1 + 1e-6)
    assert np.sqrt(sum(c[q * d:(q + 1) * d] ** 2 for q in range(4))).max() <= 0.02 * (1 + 1e-6)


def test_unregularised_fppa_equals_the_unregularised_ppga(A, ctx):
    # lam1 = lam2 = 0: zero duals, so every FPPA map is the momentum-free,
    # unregularised APPGA map: the same kernels give the same image bit for bit
    geom, Amat, mat, sl = setup(A, ctx, "64")
    kw = dict(lambda1=0.0, lambda2=0.0, momentum=1, max_iters=20)
    f, b, c, _ = run(A, ctx, geom, mat, sl, **kw)
    g = torch.empty(geom.d, dtype=torch.float32, device=DEV)
    A.appga_reconstruct(ctx.handle, mat.handle, torch.from_numpy(sl.g).to(DEV),
                        torch.from_numpy(sl.gamma).to(DEV), None, A.default_params(**kw), g)
    np.testing.assert_array_equal(f, g.cpu().numpy())
    assert not b.any() and not c.any()


def test_afppa_full_size_256(A, ctx):
    geom, Amat, mat, sl = setup(A, ctx, "256", counts=1e6)
    kw = dict(lambda1=0.05, lambda2=0.02, beta=0.3, max_iters=20, omega=0.5)
    f, b, c, st = run(A, ctx, geom, mat, sl, momentum=0, **kw)
    ref = oracle(geom, Amat, sl, momentum="gn", **kw)
    assert rel(f, ref.f) <= 1e-5 and rel(b, ref.b) <= 1e-5 and rel(c, ref.c) <= 1e-5


def test_afppa_rejects_a_stopping_tolerance(A, ctx):
    geom, Amat, mat, sl = setup(A, ctx, "64")
    with pytest.raises(A.AppgaError) as ei:
        run(A, ctx, geom, mat, sl, rel_obj_tol=1e-6)
    assert ei.value.status == A.APPGA_EINVAL
