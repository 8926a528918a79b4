"""Host-side matrix setup of the library, checked on the CPU.

``tests/host/csr_host_check.cpp`` is compiled against the library's own
host source (``csrc/csr_host.cpp`` and the internal header) and run on
seeded matrices.  What it computes is checked against definitions and
independent implementations:

* the transposed CSR that the back-projection streams (A^T w of Sec. 2.2,
  formed without atomics) equals A^T entry by entry, built here by brute
  force, and SciPy's CSC form of the Siddon matrix; each transposed row lists
  its rays in ascending order;
* rows padded to a multiple of 4 entries keep every entry in place and only
  add zero values on the row's last column, so every product is unchanged;
* the FP32 -> BF16 rounding of A's values is round-to-nearest-even, as
  PyTorch's conversion;
* the 8 x 8 tiled pixel order maps the n x n pixels one to one into
  tiled_size(n) entries, each 8 x 8 block onto one aligned run of 64, blocks
  and pixels within a block in raster order;
* the sliced layout of the solver loop's projections, decoded here from its
  documented word format and position rule, holds every padded row's
  entries in order and zero values everywhere else;
* the quarter-turn fold: the symmetry check accepts the Siddon matrices and
  rejects every matrix that breaks the symmetry by one column, one value bit,
  a repeated column or an odd size; the turn is NumPy's rot90 of the image;
  the orbit order lists each pixel once, in orbits of four turned pixels; and
  the two identities the folded loop rests on hold on the matrix, A f over
  the partner rows from the first half of A and the turned image, and A^T w
  from the folded transpose's two sums.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2409_13344_gb300", "csrc")
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
ROW_PAD = 4
SIDES = (1, 5, 8, 9, 16, 63, 64, 100)


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("g++ or the CUDA headers are missing")
    exe = str(tmp_path_factory.mktemp("host") / "csr_host_check")
    subprocess.run([gxx, "-O1", "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                    "-I", CUDA_INC, os.path.join(ROOT, "tests", "host", "csr_host_check.cpp"),
                    os.path.join(CSRC, "csr_host.cpp"), "-o", exe], check=True)
    return exe


def _run(exe, tmp_path, m, d, row_ptr, col, val, bf_in, fold=None):
    inp, out = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
    with open(inp, "wb") as f:
        np.array([m, d, len(col), len(bf_in)], np.int32).tofile(f)
        np.asarray(row_ptr, np.int32).tofile(f)
        np.asarray(col, np.int32).tofile(f)
        np.asarray(val, np.float32).tofile(f)
        np.asarray(bf_in, np.float32).tofile(f)
        np.array([len(SIDES)] + list(SIDES), np.int32).tofile(f)
        if fold is not None:
            np.array(fold, np.int32).tofile(f)
    subprocess.run([exe, inp, out], check=True)
    raw = open(out, "rb").read()
    pos = 0

    def take(dtype, n):
        nonlocal pos
        a = np.frombuffer(raw, dtype=dtype, count=n, offset=pos)
        pos += a.nbytes
        return a

    res = {}
    for key in ("at", "pa", "pt"):
        rows, nnz = take(np.int32, 2)
        res[key] = (take(np.int32, rows + 1), take(np.int32, nnz), take(np.float32, nnz))
    res["bf"] = take(np.uint16, len(bf_in))
    res["status"] = int(take(np.int32, 1)[0])
    res["tiled"] = {}
    for n in SIDES:
        size = int(take(np.int64, 1)[0])
        res["tiled"][n] = (size, take(np.int32, n * n).reshape(n, n))
    for key in ("sell_a", "sell_t"):
        ok = int(take(np.int32, 1)[0])
        if not ok:
            res[key] = None
            continue
        slices, npk = take(np.int32, 2)
        res[key] = (take(np.int32, slices + 1), take(np.uint64, npk), take(np.float32, 4 * npk))
    if fold is not None:
        res["sym"] = int(take(np.int32, 1)[0])
        res["orbit"] = take(np.int32, d)
        res["turn"] = take(np.int32, d)
        if res["sym"]:
            res["partner"] = take(np.int32, m // 2)
            rows, nnz = take(np.int32, 2)
            res["fold_t"] = (take(np.int32, rows + 1), take(np.int32, nnz),
                             take(np.float32, nnz))
    assert pos == len(raw)
    return res


def _random_csr(rng, m, d):
    """Rows of varied length (a share of them empty), columns unsorted within
    a row and occasionally repeated, positive values."""
    lens = rng.integers(0, 23, m)
    lens[rng.random(m) < 0.15] = 0
    row_ptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    col = rng.integers(0, d, int(row_ptr[-1])).astype(np.int32)
    val = rng.uniform(0.01, 2.0, int(row_ptr[-1])).astype(np.float32)
    return row_ptr, col, val


def _brute_transpose(m, d, row_ptr, col, val):
    rows = [[] for _ in range(d)]
    for i in range(m):
        for p in range(row_ptr[i], row_ptr[i + 1]):
            rows[col[p]].append((i, val[p]))
    t_ptr = np.concatenate([[0], np.cumsum([len(r) for r in rows])])
    t_col = np.array([i for r in rows for i, _ in r], np.int32)
    t_val = np.array([v for r in rows for _, v in r], np.float32)
    return t_ptr, t_col, t_val


def _check_padding(src, padded):
    s_ptr, s_col, s_val = src
    p_ptr, p_col, p_val = padded
    for i in range(len(s_ptr) - 1):
        n, pn = s_ptr[i + 1] - s_ptr[i], p_ptr[i + 1] - p_ptr[i]
        assert pn % ROW_PAD == 0 and n <= pn < n + ROW_PAD
        a, b = s_ptr[i], p_ptr[i]
        np.testing.assert_array_equal(p_col[b:b + n], s_col[a:a + n])
        np.testing.assert_array_equal(p_val[b:b + n], s_val[a:a + n])
        assert np.all(p_val[b + n:b + pn] == 0.0)
        if pn > n:
            assert np.all(p_col[b + n:b + pn] == s_col[a + n - 1])


def test_transpose_and_padding_random(harness, tmp_path):
    rng = np.random.default_rng(20240913)
    m, d = 300, 211
    row_ptr, col, val = _random_csr(rng, m, d)
    res = _run(harness, tmp_path, m, d, row_ptr, col, val, [])
    assert res["status"] == 0
    t_ptr, t_col, t_val = res["at"]
    e_ptr, e_col, e_val = _brute_transpose(m, d, row_ptr, col, val)
    np.testing.assert_array_equal(t_ptr, e_ptr)
    np.testing.assert_array_equal(t_col, e_col)
    np.testing.assert_array_equal(t_val, e_val)
    _check_padding((row_ptr, col, val), res["pa"])
    _check_padding(res["at"], res["pt"])
    # padded forms give the same products bit for bit (the added terms are +0)
    x = rng.uniform(0.0, 3.0, d).astype(np.float64)
    w = rng.uniform(-1.0, 1.0, m).astype(np.float64)
    A = sp.csr_matrix((val.astype(np.float64), col, row_ptr), shape=(m, d))
    pa_ptr, pa_col, pa_val = res["pa"]
    Ap = sp.csr_matrix((pa_val.astype(np.float64), pa_col, pa_ptr), shape=(m, d))
    pt_ptr, pt_col, pt_val = res["pt"]
    Atp = sp.csr_matrix((pt_val.astype(np.float64), pt_col, pt_ptr), shape=(d, m))
    for i in range(m):
        a = sum(float(val[p]) * x[col[p]] for p in range(row_ptr[i], row_ptr[i + 1]))
        b = sum(float(pa_val[p]) * x[pa_col[p]] for p in range(pa_ptr[i], pa_ptr[i + 1]))
        assert a == b
    np.testing.assert_allclose(Ap @ x, A @ x, rtol=1e-14, atol=0)
    np.testing.assert_allclose(Atp @ w, A.T @ w, rtol=1e-12, atol=1e-12)


def test_transpose_of_siddon_matrix_matches_scipy(harness, tmp_path):
    from paper_2409_13344_gb300 import workload as W
    A = W.system_matrix("64").tocsr()
    A.sort_indices()
    m, d = A.shape
    res = _run(harness, tmp_path, m, d, A.indptr, A.indices, A.data.astype(np.float32), [])
    assert res["status"] == 0
    C = A.tocsc()
    C.sort_indices()
    t_ptr, t_col, t_val = res["at"]
    np.testing.assert_array_equal(t_ptr, C.indptr)
    np.testing.assert_array_equal(t_col, C.indices)
    np.testing.assert_array_equal(t_val, C.data.astype(np.float32))
    _check_padding((A.indptr, A.indices, A.data.astype(np.float32)), res["pa"])


def test_bf16_rounding_is_nearest_even(harness, tmp_path):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(7)
    vals = [rng.standard_normal(4000) * 10.0 ** rng.integers(-30, 30, 4000)]
    # exact ties (low half 0x8000) with even and odd kept parts, neighbours of
    # ties, carries into the exponent, subnormals, the largest finite float
    hi = rng.integers(0x0001, 0x7f7f, 500, dtype=np.uint32)
    for low in (0x8000, 0x7fff, 0x8001, 0xffff, 0x0000, 0x0001):
        vals.append(((hi << 16) | low).view(np.float32))
    vals.append(np.array([0.0, -0.0, 1e-45, -1e-45, 1e-40, 3.4028235e38, -3.4028235e38,
                          np.float32(1.0) + np.float32(2.0 ** -8), 1.0 + 3 * 2.0 ** -8,
                          np.inf, -np.inf], np.float32))
    x = np.concatenate([np.asarray(v, np.float32) for v in vals])
    x = x[np.isfinite(x) | np.isinf(x)]
    res = _run(harness, tmp_path, 0, 1, [0], [], [], x)
    ref = torch.from_numpy(x.copy()).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    np.testing.assert_array_equal(res["bf"], ref)


def test_tiled_pixel_order(harness, tmp_path):
    res = _run(harness, tmp_path, 0, 1, [0], [], [], [])
    for n in SIDES:
        size, idx = res["tiled"][n]
        nb = -(-n // 8)
        assert size == nb * nb * 64
        flat = idx.reshape(-1)
        assert flat.min() >= 0 and flat.max() < size
        assert len(np.unique(flat)) == n * n  # one to one
        chunks = idx // 64
        prev_chunk = -1
        for br in range(nb):
            for bc in range(nb):
                blk = idx[8 * br:8 * br + 8, 8 * bc:8 * bc + 8]
                cb = chunks[8 * br:8 * br + 8, 8 * bc:8 * bc + 8]
                assert np.all(cb == cb.flat[0])  # the block sits in one aligned run of 64
                assert cb.flat[0] > prev_chunk   # blocks in raster order
                prev_chunk = cb.flat[0]
                assert np.all(np.diff(blk.reshape(-1)) > 0)  # raster order inside the block
                # a full block fills its run exactly
                if blk.shape == (8, 8):
                    np.testing.assert_array_equal(np.sort(blk.reshape(-1) % 64), np.arange(64))


SELL_LANES = 4   # lanes per row of the sliced layout (APPGA_SELL_LANES)
SELL_ROWS = 32 // SELL_LANES


def _decode_word(w):
    """Columns of one 64-bit pack word: base in bits 0-19, then three signed
    14-bit offsets from it."""
    w = int(w)
    base = w & 0xFFFFF
    out = [base]
    for i in range(3):
        o = (w >> (20 + 14 * i)) & 0x3FFF
        if o >= 0x2000:
            o -= 0x4000
        out.append(base + o)
    return out


def _check_sell(padded, sell):
    row_ptr, col, val = padded
    off, words, vals = sell
    rows = len(row_ptr) - 1
    assert len(off) == (rows + SELL_ROWS - 1) // SELL_ROWS + 1 and off[0] == 0
    assert np.all(np.diff(off) % 32 == 0)
    seen = np.zeros(len(words), bool)
    for r in range(rows):
        s, rr = divmod(r, SELL_ROWS)
        npk = (row_ptr[r + 1] - row_ptr[r]) // 4
        # the slice runs for as many steps as its longest row needs
        assert (off[s + 1] - off[s]) // 32 >= (npk + SELL_LANES - 1) // SELL_LANES
        for k in range(npk):
            pos = off[s] + (k // SELL_LANES) * 32 + rr * SELL_LANES + k % SELL_LANES
            e = row_ptr[r] + 4 * k
            assert _decode_word(words[pos]) == list(col[e:e + 4])
            np.testing.assert_array_equal(vals[4 * pos:4 * pos + 4], val[e:e + 4])
            seen[pos] = True
    assert np.all(vals.reshape(-1, 4)[~seen] == 0.0)


def test_sliced_layout_of_random_and_siddon_matrices(harness, tmp_path):
    from paper_2409_13344_gb300 import workload as W
    rng = np.random.default_rng(11)
    cases = [(37, 53) + _random_csr(rng, 37, 53), (8, 8) + _random_csr(rng, 8, 8)]
    A = W.siddon_matrix(W.Geometry(16, 10, 8))
    cases.append((A.shape[0], A.shape[1], A.indptr, A.indices, A.data))
    for m, d, row_ptr, col, val in cases:
        res = _run(harness, tmp_path, m, d, row_ptr, col, val, np.zeros(0, np.float32))
        _check_sell(res["pa"], res["sell_a"])
        _check_sell(res["pt"], res["sell_t"])


def test_sliced_layout_refuses_columns_beyond_the_word(harness, tmp_path):
    # one row with columns 0 and 9000 in one pack: the offset does not fit 14 bits
    res = _run(harness, tmp_path, 1, 9001, [0, 2], [0, 9000], [1.0, 2.0],
               np.zeros(0, np.float32))
    assert res["sell_a"] is None


def _fold_run(harness, tmp_path, A, n, na):
    m, d = A.shape
    return _run(harness, tmp_path, m, d, A.indptr, A.indices, A.data.astype(np.float32), [],
                fold=(n, na))


@pytest.mark.parametrize("name", ["64", "128"])
def test_quarter_turn_fold_of_siddon_matrix(harness, tmp_path, name):
    from paper_2409_13344_gb300 import workload as W
    geom = W.GEOMETRIES[name]
    A = W.system_matrix(name).tocsr()
    n, na, nb = geom.n, geom.n_angles, geom.n_bins
    m, d = A.shape
    res = _fold_run(harness, tmp_path, A, n, na)
    assert res["sym"] == 1
    # the turn: the pixel that rot90 (a quarter turn of the image array)
    # moves pixel j to
    idx = np.arange(d).reshape(n, n)
    turned = np.rot90(idx)               # turned[p] = the pixel that lands on p
    to = np.empty(d, np.int64)
    to[turned.reshape(-1)] = np.arange(d)
    np.testing.assert_array_equal(res["turn"], to)
    # orbit order: every pixel once, each group of four is j, turn(j), ...
    orb = res["orbit"]
    assert sorted(orb.tolist()) == list(range(d))
    grp = orb.reshape(-1, 4)
    for r in range(4):
        np.testing.assert_array_equal(to[grp[:, r]], grp[:, (r + 1) % 4])
    # partner rows: angle a + NPA/2, bin nb-1-b
    half = m // 2
    i = np.arange(half)
    np.testing.assert_array_equal(res["partner"], (i // nb + na // 2) * nb + nb - 1 - i % nb)
    # identity of the folded forward projection: (A f)_partner(i) equals row
    # i of A times the turned image, (f o turn)_j = f_turn(j)
    rng = np.random.default_rng(11)
    f = rng.uniform(0.0, 2.0, d)
    A64 = A.astype(np.float64)
    A1 = A64[:half]
    y = A64 @ f
    np.testing.assert_allclose(y[res["partner"]], A1 @ f[to], rtol=1e-12, atol=1e-12)
    # identity of the folded back-projection: (A^T w)_q = s1(q) + s2(turn^-1 q)
    # with s1, s2 the folded transpose's sums over w and w o partner
    w = rng.uniform(-1.0, 1.0, m)
    t_ptr, t_col, t_val = res["fold_t"]
    FT = sp.csr_matrix((t_val.astype(np.float64), t_col, t_ptr), shape=(d, half))
    s1 = FT @ w[:half]
    s2 = FT @ w[res["partner"]]
    bp = np.empty(d)
    for r in range(4):
        bp[grp[:, r]] = s1.reshape(-1, 4)[:, r] + s2.reshape(-1, 4)[:, (r + 3) % 4]
    np.testing.assert_allclose(bp, A64.T @ w, rtol=1e-12, atol=1e-12)
    # each folded transposed row: the rays of the first half through its pixel
    At1 = A1.T.tocsr()
    for k in (0, 1, 2, 3, d // 2 + 5, d - 1):
        p = orb[k]
        np.testing.assert_array_equal(t_col[t_ptr[k]:t_ptr[k + 1]],
                                      At1.indices[At1.indptr[p]:At1.indptr[p + 1]])


def test_quarter_turn_check_rejects_broken_symmetry(harness, tmp_path):
    from paper_2409_13344_gb300 import workload as W
    geom = W.GEOMETRIES["64"]
    A = W.system_matrix("64").tocsr()
    n, na, nb = geom.n, geom.n_angles, geom.n_bins
    m = A.shape[0]
    rng = np.random.default_rng(5)
    p = int(rng.integers(0, A.nnz))
    # one value one bit up
    B = A.copy()
    B.data = B.data.copy()
    B.data[p] = np.nextafter(B.data[p], np.float32(np.inf))
    assert _fold_run(harness, tmp_path, B, n, na)["sym"] == 0
    # one entry moved to a column its row does not have
    B = A.copy()
    B.indices = B.indices.copy()
    row = int(np.searchsorted(B.indptr, p, side="right") - 1)
    have = set(B.indices[B.indptr[row]:B.indptr[row + 1]].tolist())
    B.indices[p] = next(x for x in range(n * n) if x not in have)
    assert _fold_run(harness, tmp_path, B, n, na)["sym"] == 0
    # a repeated column, added to a row and, turned, to its partner row
    i = int(np.argmax(np.diff(A.indptr)[:m // 2] > 3))
    k = (i // nb + na // 2) * nb + nb - 1 - i % nb
    ci, vi = int(A.indices[A.indptr[i]]), A.data[A.indptr[i]]
    coo = A.tocoo()
    rows = np.concatenate([coo.row, [i, k]])
    cols = np.concatenate([coo.col, [ci, (n - 1 - ci % n) * n + ci // n]])
    vals = np.concatenate([coo.data, [vi, vi]]).astype(np.float32)
    order = np.argsort(rows, kind="stable")
    D = sp.csr_matrix((vals[order], cols[order],
                       np.concatenate([[0], np.cumsum(np.bincount(rows, minlength=m))])),
                      shape=A.shape)
    assert D.nnz == A.nnz + 2
    assert _fold_run(harness, tmp_path, D, n, na)["sym"] == 0
    # odd numbers of angles and an odd image side have no fold
    A5 = W.siddon_matrix(W.Geometry(8, 5, 11))
    assert _fold_run(harness, tmp_path, A5, 8, 5)["sym"] == 0
    A9 = W.siddon_matrix(W.Geometry(9, 4, 13))
    assert _fold_run(harness, tmp_path, A9, 9, 4)["sym"] == 0
    # another even side and even number of angles has it
    A10 = W.siddon_matrix(W.Geometry(10, 6, 15))
    assert _fold_run(harness, tmp_path, A10, 10, 6)["sym"] == 1
