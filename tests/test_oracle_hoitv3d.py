"""Pins of the 3-D SHOITV oracle and of APPGA on a volume (CPU, FP64).

The paper gives HOITV in 2-D (Sec. 2.1); the 3-D operators are the
Kronecker generalisation stated in ``oracle/hoitv3d_oracle.py``.  Each
check below fixes the oracle by something other than its own formulas:

* a voxel-by-voxel evaluation of the twelve components from the definition
  of D (brute force on tiny volumes);
* one slice reduces to the independently pinned 2-D oracle;
* permuting the axes of a cube leaves the regulariser unchanged;
* constant volumes give zero; a ramp along z gives hand-derived fields;
* the gradient matches central finite differences;
* the volume iteration with one slice is the 2-D iteration, and without
  regulariser and momentum it is MLEM slice by slice.
"""
import itertools

import numpy as np
import pytest

from oracle import appga_oracle as O
from oracle import hoitv3d_oracle as H
from paper_2409_13344_gb300 import workload as W


def _D(x):  # (D x)_i = x_i - x_{i-1} for i >= 1, 0 for i = 0
    n = len(x)
    return np.array([0.0] + [x[i] - x[i - 1] for i in range(1, n)])


def _Dt(y):  # (D^T y)_i = y_i [i >= 1] - y_{i+1} [i <= n-2]
    n = len(y)
    out = np.zeros(n)
    for i in range(n):
        if i >= 1:
            out[i] += y[i]
        if i + 1 <= n - 1:
            out[i] -= y[i + 1]
    return out


def _along(V, axis, op):
    return np.apply_along_axis(op, axis, V)


def _fields_by_loops(V):
    """The twelve component fields of a volume V[z, r, c], built from 1-D
    applications of D and D^T along each axis (axis 0 = z, 1 = r, 2 = c)."""
    Z, R, C = 0, 1, 2
    D = lambda V, ax: _along(V, ax, _D)
    Dt = lambda V, ax: _along(V, ax, _Dt)
    first = [D(V, C), D(V, R), D(V, Z)]
    second = [-Dt(D(V, C), C), -Dt(D(V, C), R), -Dt(D(V, R), R), -D(Dt(V, C), R),
              -Dt(D(V, Z), Z), -Dt(D(V, C), Z), -D(Dt(V, C), Z), -Dt(D(V, R), Z), -D(Dt(V, R), Z)]
    return [u.reshape(-1) for u in first + second]


@pytest.mark.parametrize("nz,n", [(1, 4), (2, 3), (3, 4), (4, 2), (5, 5)])
def test_components_match_voxelwise_definition(nz, n):
    rng = np.random.default_rng(10 * nz + n)
    V = rng.standard_normal((nz, n, n))
    u = H.b_matrix3(nz, n) @ V.reshape(-1)
    dv = V.size
    ref = _fields_by_loops(V)
    for q in range(12):
        np.testing.assert_allclose(u[q * dv:(q + 1) * dv], ref[q], rtol=0, atol=1e-12)


def test_single_slice_reduces_to_2d():
    n = 9
    rng = np.random.default_rng(4)
    F = rng.uniform(0.0, 3.0, n * n)
    B2d = O.b_matrix(n)
    reg = H.Regulariser3D(1, n)
    for lam1, lam2, eps in ((0.1, 0.05, 1e-3), (0.3, 0.7, 2.0)):
        a = reg.value(F, lam1, lam2, eps)
        b = O.phi_tilde(B2d @ F, n * n, lam1, lam2, eps)
        assert abs(a - b) <= 1e-13 * abs(b)
        ga = reg.grad(F, lam1, lam2, eps)
        gb = B2d.T @ O.grad_phi_tilde(B2d @ F, n * n, lam1, lam2, eps)
        np.testing.assert_allclose(ga, gb, rtol=0, atol=1e-13 * np.max(np.abs(gb)))


def test_axis_permutations_leave_regulariser_unchanged():
    n = 5
    rng = np.random.default_rng(8)
    V = rng.uniform(0.0, 2.0, (n, n, n))
    reg = H.Regulariser3D(n, n)
    base = reg.value(V, 0.2, 0.4, 0.05)
    g0 = reg.grad(V, 0.2, 0.4, 0.05).reshape(n, n, n)
    for perm in itertools.permutations(range(3)):
        Vp = np.ascontiguousarray(np.transpose(V, perm))
        assert abs(reg.value(Vp, 0.2, 0.4, 0.05) - base) <= 1e-12 * abs(base)
        gp = reg.grad(Vp, 0.2, 0.4, 0.05).reshape(n, n, n)
        np.testing.assert_allclose(gp, np.transpose(g0, perm), rtol=0, atol=1e-12)


def test_constant_volume_is_zero():
    u = H.b_matrix3(3, 6) @ np.full(3 * 36, 2.5)
    assert np.max(np.abs(u)) == 0.0


def test_z_ramp_special_case():
    # V[z, r, c] = z: hand-derived from the definition of D along each axis.
    nz, n = 5, 4
    z = np.arange(nz, dtype=float)
    V = np.broadcast_to(z[:, None, None], (nz, n, n)).copy()
    u = (H.b_matrix3(nz, n) @ V.reshape(-1)).reshape(12, nz, n, n)
    zge1 = (z >= 1).astype(float)[:, None, None] * np.ones((nz, n, n))
    zero = np.zeros((nz, n, n))
    end_c = np.zeros((n, n)); end_c[:, 0] = 1.0; end_c[:, -1] = -1.0    # [c=0] - [c=n-1]
    end_r = np.zeros((n, n)); end_r[0, :] = 1.0; end_r[-1, :] = -1.0    # [r=0] - [r=n-1]
    end_z = np.zeros((nz, n, n)); end_z[0] = 1.0; end_z[-1] = -1.0      # [z=0] - [z=nz-1]
    expected = [zero, zero, zge1,                    # Dc, Dr, Dz
                zero, zero, zero, zero,              # the four in-slice blocks
                end_z,                               # -Dz^T Dz
                zero, zge1 * end_c[None],            # -Dz^T Dc, -Dz Dc^T
                zero, zge1 * end_r[None]]            # -Dz^T Dr, -Dz Dr^T
    for q in range(12):
        np.testing.assert_array_equal(u[q], expected[q])


@pytest.mark.parametrize("eps", [1e-3, 0.5])
def test_regulariser_gradient_fd(eps):
    nz, n = 3, 4
    rng = np.random.default_rng(2)
    V = rng.uniform(0.5, 2.0, nz * n * n)
    reg = H.Regulariser3D(nz, n)
    gr = reg.grad(V, 0.3, 0.2, eps)
    h = 1e-6
    for j in range(0, V.size, 5):
        e = np.zeros(V.size); e[j] = h
        fd = (reg.value(V + e, 0.3, 0.2, eps) - reg.value(V - e, 0.3, 0.2, eps)) / (2 * h)
        assert gr[j] == pytest.approx(fd, rel=1e-6, abs=1e-7)


def test_group_norm_bounds():
    # ||B1||^2 <= 12 and ||B2||^2 <= 144 in 3-D (4 per first-order axis
    # difference; every second-order block has norm at most 4).
    nz, n = 4, 5
    s1 = np.linalg.norm(H.b1_matrix3(nz, n).toarray(), 2) ** 2
    s2 = np.linalg.norm(H.b2_matrix3(nz, n).toarray(), 2) ** 2
    assert s1 <= 12.0 + 1e-9 and s2 <= 144.0 + 1e-9
    assert s1 > 8.0


def _slices(nz, counts=1e5):
    geom = W.GEOMETRIES["64"]
    A = W.system_matrix("64")
    sls = [W.make_slice(A, geom, counts * (1 + z), W.seed_for(1, z)) for z in range(nz)]
    return geom, A, sls


def test_volume_with_one_slice_is_the_2d_iteration():
    geom, A, sls = _slices(1)
    p = O.Params(max_iters=12, omega=0.5)
    vol = H.VolumeProblem(A, sls[0].g[None], sls[0].gamma[None], geom.n)
    rv = H.appga_volume(vol, p, n_angles=geom.n_angles)
    r2 = O.appga(O.Problem(A, sls[0].g, sls[0].gamma, geom.n), p, n_angles=geom.n_angles)
    np.testing.assert_allclose(rv.f[0], r2.f, rtol=0, atol=1e-12 * np.max(r2.f))
    np.testing.assert_allclose(rv.phi, r2.phi, rtol=1e-13)


def test_volume_without_regulariser_or_momentum_is_slicewise_mlem():
    geom, A, sls = _slices(3)
    vol = H.VolumeProblem(A, np.stack([s.g for s in sls]), np.stack([s.gamma for s in sls]), geom.n)
    p = O.Params(lambda1=0.0, lambda2=0.0, beta=1.0, momentum="none", max_iters=3)
    res = H.appga_volume(vol, p, n_angles=geom.n_angles, track_phi=False)
    for z, s in enumerate(sls):
        prob = O.Problem(A, s.g, s.gamma, geom.n)
        ref = O.initial_image(s.g, s.gamma, geom.n, geom.n_angles)
        for _ in range(3):
            ref = O.mlem_step(prob, ref)
        assert np.max(np.abs(res.f[z] - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_volume_objective_decreases_and_stops():
    geom, A, sls = _slices(3)
    vol = H.VolumeProblem(A, np.stack([s.g for s in sls]), np.stack([s.gamma for s in sls]), geom.n)
    p = O.Params(max_iters=200, beta=0.5, omega=1.0, rel_obj_tol=1e-6)
    res = H.appga_volume(vol, p, n_angles=geom.n_angles)
    assert res.iters < 200
    last = abs(res.phi[-1] - res.phi[-2]) / abs(res.phi[-2])
    prev = abs(res.phi[-2] - res.phi[-3]) / abs(res.phi[-3])
    assert last <= 1e-6 < prev
    assert res.phi[-1] < res.phi[0]


def test_rectangular_boxes_match_voxelwise_definition():
    # the same twelve fields on a non-square box (used for sampled checks)
    rng = np.random.default_rng(12)
    V = rng.standard_normal((3, 4, 6))
    u = H.b_matrix3(3, 4, 6) @ V.reshape(-1)
    ref = _fields_by_loops(V)
    for q in range(12):
        np.testing.assert_allclose(u[q * V.size:(q + 1) * V.size], ref[q], rtol=0, atol=1e-12)
