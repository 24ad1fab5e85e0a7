"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each check is chosen so that a plausible slip in the oracle (a dropped term, a
flipped sign, a swapped index or operand) fails at least one of them: closed
forms of stencil Laplacians, identity and permutation matrices, dense brute
force through numpy, scipy's CCS conversion, central finite differences, and
the paper's printed table values.  ``test_planted_mistakes_are_caught`` plants
such slips in a copy of the oracle source and checks that the pins notice.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- helpers

def grid_missing_2d(N):
    """Number of 5-point neighbours of each grid point that fall outside the N x N grid."""
    i, j = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    miss = (i == 0).astype(int) + (i == N - 1) + (j == 0) + (j == N - 1)
    return miss.reshape(-1)


def linear_2d_expected(N, a, b, c):
    """(A x)_ij for x_ij = a i + b j + c under the Dirichlet 5-point Laplacian (diag 4, off -1):
    the four differences x_ij - x_nbr cancel for a linear field, leaving the sum of the field's
    values at the neighbours that lie outside the grid."""
    out = np.zeros((N, N))
    i, j = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    for di, dj in ((-1, 0), (1, 0), (0, -1), (0, 1)):
        ii, jj = i + di, j + dj
        outside = (ii < 0) | (ii >= N) | (jj < 0) | (jj >= N)
        out += np.where(outside, a * ii + b * jj + c, 0.0)
    return out.reshape(-1)


def missing_3d(N):
    """Number of 27-point neighbours (excluding the centre) outside the N^3 grid."""
    idx = np.arange(N)
    inside1 = np.array([1 + (x > 0) + (x < N - 1) for x in idx])  # neighbours along one axis incl. self
    tot = inside1[:, None, None] * inside1[None, :, None] * inside1[None, None, :]
    return (27 - tot).reshape(-1)


def linear_3d_expected(N, a, b, c, d):
    i, j, k = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    out = np.zeros((N, N, N))
    for di in (-1, 0, 1):
        for dj in (-1, 0, 1):
            for dk in (-1, 0, 1):
                if di == dj == dk == 0:
                    continue
                ii, jj, kk = i + di, j + dj, k + dk
                outside = (ii < 0) | (ii >= N) | (jj < 0) | (jj >= N) | (kk < 0) | (kk >= N)
                out += np.where(outside, a * ii + b * jj + c * kk + d, 0.0)
    return out.reshape(-1)


def dense_ref(A: synth.CSR, X):
    """Dense product through numpy, and the bound sum_p |val[p] X[col[p], :]| over the stored
    nonzeros (duplicates count separately, as they are stored separately)."""
    D = A.to_dense()
    rows = np.repeat(np.arange(A.m), A.row_lengths())
    Xa = np.asarray(X, dtype=np.float64)
    prod = np.abs(A.vals.astype(np.float64)[:, None] * Xa.reshape(A.n, -1)[A.col_idx])
    R = np.zeros((A.m, prod.shape[1]))
    np.add.at(R, rows, prod)
    return D @ Xa, R.reshape((A.m,) + Xa.shape[1:])


# ------------------------------------------------------- generator pins

def test_stencil2d_counts_and_paper_mesh_2048():
    for N in (1, 2, 3, 7, 64):
        A = synth.stencil2d(N)
        assert A.nnz == 5 * N * N - 4 * N
        assert A.row_ptr[0] == 0 and A.row_ptr[-1] == A.nnz
    assert synth.stencil2d(64).nnz == 20224
    # Paper Table "tab:matrices" row 20: mesh_2048
    fields = None
    for line in open(os.path.join(GOLDEN, "mesh_2048.txt")):
        if line.startswith("mesh_2048"):
            fields = line.split()
    rows, nnz, maxr = int(fields[1]), int(fields[2]), int(fields[4])
    A = synth.stencil2d(2048)
    assert A.m == rows and A.nnz == nnz
    assert A.row_lengths().max() == maxr
    # the table prints nnz/row truncated to two decimals (20963328 / 4194304 = 4.998...)
    assert int(A.nnz / A.m * 100) / 100 == float(fields[3])


def test_stencil3d_counts():
    for N in (1, 2, 3, 5):
        A = synth.stencil3d(N)
        assert A.nnz == (3 * N - 2) ** 3
    assert (3 * 100 - 2) ** 3 == 26463592


def test_generators_structure():
    B = synth.banded(5000, hbw=100, per_row=20, seed=7)
    lens = B.row_lengths()
    assert (lens == 20).all()
    for i in (0, 1, 2500, 4999):
        cols = B.col_idx[B.row_ptr[i]:B.row_ptr[i + 1]]
        assert (np.diff(cols) > 0).all() and i in cols
        assert np.abs(cols - i).max() <= 100
        v = B.vals[B.row_ptr[i]:B.row_ptr[i + 1]]
        diag = v[cols == i][0]
        assert diag == pytest.approx(np.abs(v[cols != i]).sum() + 1.0, rel=1e-15)
    R = synth.rmat(12, ef=8, seed=3)
    assert R.nnz <= 8 * 4096 and R.nnz > 4096
    rows = np.repeat(np.arange(R.m), R.row_lengths())
    key = rows.astype(np.int64) * R.n + R.col_idx
    assert (np.diff(key) > 0).all()  # sorted and deduplicated
    # determinism
    R2 = synth.rmat(12, ef=8, seed=3)
    assert np.array_equal(R.col_idx, R2.col_idx) and np.array_equal(R.row_ptr, R2.row_ptr)
    u = synth.uniform(1000, -1, 1, seed=5)
    assert u.min() >= -1 and u.max() < 1 and abs(u.mean()) < 0.1


# ------------------------------------------------------------ SpMV pins

def check_spmv_closed_forms(spmv):
    """Closed-form pins of an SpMV callable spmv(m, rp, ci, v, x) -> (y, r)."""
    for N in (1, 2, 5, 16):
        A = synth.stencil2d(N)
        y, r = spmv(A.m, A.row_ptr, A.col_idx, A.vals, np.ones(A.n))
        assert np.array_equal(y, grid_missing_2d(N).astype(float)), "A*1 on the 2D Laplacian"
        assert np.array_equal(r, (4.0 + (4 - grid_missing_2d(N))).astype(float)), "sum |a x| on A*1"
        a, b, c = 0.75, -1.25, 0.5
        i, j = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
        x = (a * i + b * j + c).reshape(-1).astype(float)
        y, _ = spmv(A.m, A.row_ptr, A.col_idx, A.vals, x)
        assert np.allclose(y, linear_2d_expected(N, a, b, c), rtol=0, atol=1e-12), "2D linear field"
    for N in (2, 4):
        A = synth.stencil3d(N)
        y, _ = spmv(A.m, A.row_ptr, A.col_idx, A.vals, np.ones(A.n))
        assert np.array_equal(y, missing_3d(N).astype(float)), "A*1 on the 27-point stencil"
        i, j, k = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
        x = (0.5 * i - 0.25 * j + 2.0 * k + 1.0).reshape(-1)
        y, _ = spmv(A.m, A.row_ptr, A.col_idx, A.vals, x)
        assert np.allclose(y, linear_3d_expected(N, 0.5, -0.25, 2.0, 1.0), rtol=0, atol=1e-12), "3D linear"


def check_spmv_permutation(spmv):
    rng = np.random.default_rng(11)
    for m in (1, 7, 100):
        # identity
        rp = np.arange(m + 1, dtype=np.int32)
        ci = np.arange(m, dtype=np.int32)
        x = rng.uniform(-1, 1, m)
        y, _ = spmv(m, rp, ci, np.ones(m), x)
        assert np.array_equal(y, x), "identity"
        # permutation: row i holds a single 1 in column pi[i], so y_i = x[pi[i]]
        pi = rng.permutation(m).astype(np.int32)
        y, _ = spmv(m, rp, pi, np.ones(m), x)
        assert np.array_equal(y, x[pi]), "permutation"
        # scaled permutation
        s = rng.uniform(0.5, 2.0, m)
        y, _ = spmv(m, rp, pi, s, x)
        assert np.array_equal(y, s * x[pi])


def check_spmv_brute_force(spmv):
    cases = [
        synth.random_csr(1, 1, 1.0, 1),
        synth.random_csr(5, 9, 0.4, 2, empty_rows=0.3),
        synth.random_csr(40, 17, 0.3, 3),
        synth.random_csr(17, 40, 0.3, 4, empty_rows=0.2),
        synth.random_csr(64, 64, 0.1, 5, sorted_cols=False),
        synth.random_csr(30, 30, 0.2, 6, duplicates=True),
        synth.random_csr(20, 20, 0.0, 7),  # tau = 0
    ]
    # one full row among empty ones
    rp = np.zeros(9, np.int32)
    rp[4:] = 33
    cases.append(synth.CSR(8, 33, rp, np.arange(33, dtype=np.int32), np.linspace(-1, 1, 33)))
    rng = np.random.default_rng(12)
    for A in cases:
        x = rng.uniform(-1, 1, A.n)
        y, r = spmv(A.m, A.row_ptr, A.col_idx, A.vals, x)
        yd, rd = dense_ref(A, x)
        assert y.shape == (A.m,)
        assert np.all(np.abs(y - yd) <= 1e-14 * rd + 0.0), "dense brute force"
        assert np.allclose(r, rd, rtol=1e-14, atol=0)
        assert np.all(np.abs(y) <= r * (1 + 1e-15))
        empty = A.row_lengths() == 0
        assert np.all(y[empty] == 0.0) and np.all(r[empty] == 0.0)


def _oracle_spmv(m, rp, ci, v, x):
    return oracle.spmv(m, rp, ci, v, x)


def test_spmv_closed_forms():
    check_spmv_closed_forms(_oracle_spmv)


def test_spmv_identity_permutation():
    check_spmv_permutation(_oracle_spmv)


def test_spmv_dense_brute_force():
    check_spmv_brute_force(_oracle_spmv)


def test_spmv_threads_do_not_change_result():
    A = synth.banded(3000, hbw=50, per_row=12, seed=9)
    x = synth.uniform(A.n, seed=9)
    y1, r1 = oracle.spmv(A.m, A.row_ptr, A.col_idx, A.vals, x, threads=1)
    y4, r4 = oracle.spmv(A.m, A.row_ptr, A.col_idx, A.vals, x, threads=4)
    assert np.array_equal(y1, y4) and np.array_equal(r1, r4)


def test_spmv_f32_inputs_accumulate_in_f64():
    rng = np.random.default_rng(13)
    A = synth.random_csr(50, 70, 0.3, 14, empty_rows=0.1)
    v32 = A.vals.astype(np.float32)
    x32 = rng.uniform(-1, 1, A.n).astype(np.float32)
    y, r = oracle.spmv(A.m, A.row_ptr, A.col_idx, v32, x32)
    D = synth.CSR(A.m, A.n, A.row_ptr, A.col_idx, v32.astype(np.float64)).to_dense()
    yd = D @ x32.astype(np.float64)
    rd = np.abs(D) @ np.abs(x32.astype(np.float64))
    # float x float products are exact in double; only the double sums round
    assert np.all(np.abs(y - yd) <= 1e-14 * rd)
    assert y.dtype == np.float64


# ------------------------------------------------------------ SpMM pins

def test_spmm_dense_brute_force_and_columns():
    rng = np.random.default_rng(21)
    for (m, n, k, dens, seed) in ((9, 13, 1, 0.3, 1), (40, 25, 4, 0.2, 2), (25, 40, 8, 0.15, 3),
                                  (64, 64, 16, 0.1, 4), (10, 10, 3, 0.0, 5), (33, 31, 5, 0.25, 6)):
        A = synth.random_csr(m, n, dens, seed, empty_rows=0.2)
        wide = rng.uniform(-1, 1, (n, k + 3))
        X = wide[:, :k]  # leading dimension k + 3 > k
        Y, R = oracle.spmm(m, A.row_ptr, A.col_idx, A.vals, X)
        Yd, Rd = dense_ref(A, X)
        assert Y.shape == (m, k)
        assert np.all(np.abs(Y - Yd) <= 1e-14 * Rd)
        assert np.allclose(R, Rd, rtol=1e-14, atol=0)
        for c in range(k):  # column c of Y is the SpMV of column c of X
            yc, _ = oracle.spmv(m, A.row_ptr, A.col_idx, A.vals, np.ascontiguousarray(X[:, c]))
            assert np.array_equal(Y[:, c], yc)


def test_spmm_stencil_constant_columns():
    N = 8
    A = synth.stencil2d(N)
    X = np.stack([np.ones(A.n), 2 * np.ones(A.n), -np.ones(A.n)], axis=1)
    Y, _ = oracle.spmm(A.m, A.row_ptr, A.col_idx, A.vals, X)
    miss = grid_missing_2d(N).astype(float)
    assert np.array_equal(Y[:, 0], miss) and np.array_equal(Y[:, 1], 2 * miss) and np.array_equal(Y[:, 2], -miss)


# ------------------------------------------------------- transpose pins

def test_transpose_matches_scipy_and_is_involution():
    sp = pytest.importorskip("scipy.sparse")
    for (m, n, dens, seed) in ((1, 1, 1.0, 1), (13, 29, 0.3, 2), (29, 13, 0.3, 3), (64, 64, 0.05, 4), (7, 7, 0.0, 5)):
        A = synth.random_csr(m, n, dens, seed, empty_rows=0.2)
        marker = np.arange(A.nnz, dtype=np.float64) + 1.0  # identifies each nonzero
        S = sp.csr_matrix((marker, A.col_idx, A.row_ptr), shape=(m, n))
        C = S.tocsc()  # the dual CCS of A is the CRS of A^T (Sec. 3)
        rpT, ciT, perm = oracle.transpose(m, n, A.row_ptr, A.col_idx)
        assert np.array_equal(rpT, C.indptr) and np.array_equal(ciT, C.indices)
        assert np.array_equal(perm.astype(np.float64) + 1.0, C.data)
        rpTT, ciTT, permTT = oracle.transpose(n, m, rpT, ciT)
        assert np.array_equal(rpTT, A.row_ptr) and np.array_equal(ciTT, A.col_idx)
        assert np.array_equal(perm[permTT], np.arange(A.nnz))


def test_transpose_stability_with_duplicates_and_unsorted():
    A = synth.random_csr(30, 12, 0.3, 8, sorted_cols=False, duplicates=True)
    rpT, ciT, perm = oracle.transpose(A.m, A.n, A.row_ptr, A.col_idx)
    rows = np.repeat(np.arange(A.m), A.row_lengths())
    # brute force: column j of A, in order of storage
    for j in range(A.n):
        expect = [p for p in range(A.nnz) if A.col_idx[p] == j]
        got = perm[rpT[j]:rpT[j + 1]]
        assert list(got) == expect
        assert np.array_equal(ciT[rpT[j]:rpT[j + 1]], rows[expect])


def test_transpose_rejects_bad_column():
    rp = np.array([0, 2], np.int32)
    with pytest.raises(ValueError):
        oracle.transpose(1, 3, rp, np.array([0, 3], np.int32))


def test_adjoint_identity():
    rng = np.random.default_rng(31)
    A = synth.random_csr(50, 35, 0.2, 9)
    x, w = rng.uniform(-1, 1, A.n), rng.uniform(-1, 1, A.m)
    rpT, ciT, perm = oracle.transpose(A.m, A.n, A.row_ptr, A.col_idx)
    Ax, _ = oracle.spmv(A.m, A.row_ptr, A.col_idx, A.vals, x)
    ATw, _ = oracle.spmv(A.n, rpT, ciT, A.vals[perm], w)
    assert abs(Ax @ w - x @ ATw) <= 1e-13 * (np.abs(A.vals).sum() + 1)


# -------------------------------------------------------- backward pins

def _loss(A, vals, X, W):
    """L = <A X, W> computed densely in numpy (independent of the oracle)."""
    D = synth.CSR(A.m, A.n, A.row_ptr, A.col_idx, vals).to_dense()
    return float(np.sum((D @ X) * W))


@pytest.mark.parametrize("k", [1, 3, 8])
def test_backward_finite_differences(k):
    rng = np.random.default_rng(40 + k)
    A = synth.random_csr(23, 19, 0.25, 41 + k, empty_rows=0.1, duplicates=True)
    X = rng.uniform(-1, 1, (A.n, k))
    W = rng.uniform(-1, 1, (A.m, k))
    dX, dvals, RdX, Rdv = oracle.backward(A.m, A.n, A.row_ptr, A.col_idx, A.vals, X, W)
    h = 1e-6
    # L is bilinear in (vals, X): a central difference is exact up to rounding
    for _ in range(8):
        dv = rng.uniform(-1, 1, A.nnz)
        fd = (_loss(A, A.vals + h * dv, X, W) - _loss(A, A.vals - h * dv, X, W)) / (2 * h)
        assert fd == pytest.approx(dvals @ dv, rel=1e-7, abs=1e-9)
        dx = rng.uniform(-1, 1, X.shape)
        fd = (_loss(A, A.vals, X + h * dx, W) - _loss(A, A.vals, X - h * dx, W)) / (2 * h)
        assert fd == pytest.approx(np.sum(dX * dx), rel=1e-7, abs=1e-9)
    # dense brute force
    D = A.to_dense()
    assert np.allclose(dX, D.T @ W, rtol=1e-13, atol=1e-13)
    rows = np.repeat(np.arange(A.m), A.row_lengths())
    assert np.allclose(dvals, np.einsum("pc,pc->p", W[rows], X[A.col_idx]), rtol=1e-13, atol=1e-14)
    RdX_bf = np.zeros_like(RdX)
    np.add.at(RdX_bf, A.col_idx, np.abs(A.vals[:, None] * W[rows]))
    assert np.allclose(RdX, RdX_bf, rtol=1e-13)
    assert np.all(Rdv >= np.abs(dvals) - 1e-15)


def test_backward_f32_inputs():
    rng = np.random.default_rng(50)
    A = synth.random_csr(20, 30, 0.3, 51).astype(np.float32)
    X = rng.uniform(-1, 1, (A.n, 4)).astype(np.float32)
    W = rng.uniform(-1, 1, (A.m, 4)).astype(np.float32)
    dX, dvals, _, _ = oracle.backward(A.m, A.n, A.row_ptr, A.col_idx, A.vals, X, W)
    D = synth.CSR(A.m, A.n, A.row_ptr, A.col_idx, A.vals.astype(np.float64)).to_dense()
    assert np.allclose(dX, D.T @ W.astype(np.float64), rtol=1e-13, atol=1e-13)


# ---------------------------------------------------------- batch offsets

def test_batch_offsets_brute_force():
    rng = np.random.default_rng(60)
    ms = rng.integers(0, 1000, 37).astype(np.int32)
    ns = rng.integers(1, 1000, 37).astype(np.int32)
    nnz = rng.integers(0, 10**6, 37).astype(np.int64)
    k = 8
    off_rows, off_nnz, off_rp, off_x, off_y = oracle.batch_offsets(ms, ns, nnz, k)
    r = z = rp = xo = yo = 0
    for b in range(37):
        assert (off_rows[b], off_nnz[b], off_rp[b], off_x[b], off_y[b]) == (r, z, rp, xo, yo)
        r += int(ms[b]); z += int(nnz[b]); rp += int(ms[b]) + 1; xo += int(ns[b]) * k; yo += int(ms[b]) * k
    assert (off_rows[37], off_nnz[37], off_rp[37], off_x[37], off_y[37]) == (r, z, rp, xo, yo)


# ------------------------------------------------------------------ UCLD

def _ucld_rows(rows, line):
    rp = np.zeros(len(rows) + 1, np.int32)
    rp[1:] = np.cumsum([len(r) for r in rows])
    ci = np.array([c for r in rows for c in r], np.int32)
    return oracle.ucld(len(rows), rp, ci, line)


def test_ucld_paper_example():
    """The worked example and the extremes of Sec. 4.1 (tests/golden/ucld_example.txt)."""
    from fractions import Fraction
    for line in open(os.path.join(GOLDEN, "ucld_example.txt")):
        if line.startswith("#") or not line.strip():
            continue
        cols, L, num, den = line.split()
        cols = [int(c) for c in cols.split(",")]
        u, lines, rows = _ucld_rows([cols], int(L))
        assert Fraction(u).limit_denominator(1000) == Fraction(int(num), int(den))
        assert rows == 1
    # the example's two lines, and order does not matter
    assert _ucld_rows([[20, 0, 19]], 8)[:2] == (3 / 16, 2)


def test_ucld_closed_forms():
    # identity: one nonzero per row on its own line -> 1 / line
    n = 1000
    rp = np.arange(n + 1, dtype=np.int32)
    ci = np.arange(n, dtype=np.int32)
    for L in (4, 8, 16):
        u, lines, rows = oracle.ucld(n, rp, ci, L)
        assert u == pytest.approx(1.0 / L, rel=1e-15) and lines == n and rows == n
    # a dense aligned 64-column row -> 1; empty rows are skipped
    u, lines, rows = _ucld_rows([[], list(range(64)), []], 8)
    assert (u, lines, rows) == (1.0, 8, 1)
    # 2D 5-point stencil, interior row i on an N x N grid with 8-element lines: the
    # vertical neighbours i +- N sit on their own lines (N >= 8), and i-1, i, i+1 share
    # one line unless i is first or last in its line
    N = 64
    A = synth.stencil2d(N)
    u, lines, rows = oracle.ucld(A.m, A.row_ptr, A.col_idx, 8)
    want = 0.0
    for i in range(A.m):
        r, c = divmod(i, N)
        cols = [i] + ([i - N] if r > 0 else []) + ([i + N] if r < N - 1 else []) + \
               ([i - 1] if c > 0 else []) + ([i + 1] if c < N - 1 else [])
        lines_i = len({x // 8 for x in cols})
        want += len(cols) / (8 * lines_i)
    assert u == pytest.approx(want / A.m, rel=1e-13)


def test_ucld_brute_force():
    rng = np.random.default_rng(70)
    for trial in range(20):
        A = synth.random_csr(int(rng.integers(1, 60)), int(rng.integers(1, 200)), float(rng.uniform(0, 0.3)),
                             100 + trial, sorted_cols=bool(trial % 2), duplicates=bool(trial % 3 == 0),
                             empty_rows=0.2)
        for L in (1, 4, 8, 16):
            s, tot, rows = 0.0, 0, 0
            for i in range(A.m):
                cols = A.col_idx[A.row_ptr[i]:A.row_ptr[i + 1]]
                if cols.size == 0:
                    continue
                d = np.unique(cols // L).size
                s += cols.size / (L * d)
                tot += d
                rows += 1
            u, lines, nrows = oracle.ucld(A.m, A.row_ptr, A.col_idx, L)
            assert (lines, nrows) == (tot, rows)
            assert u == pytest.approx(s / rows if rows else 0.0, rel=1e-14, abs=0.0)


UCLD_MUTATIONS = [
    ("runs instead of distinct lines", "qsort(buf, (size_t)len, sizeof(int), cmp_int);", ";"),
    ("line factor dropped", "sum += (double)len / ((double)line * (double)distinct);",
     "sum += (double)len / ((double)distinct);"),
    ("empty rows counted", "if (len == 0) continue;", "if (len == 0) { rows += 1; continue; }"),
    ("element index instead of line", "buf[q] = cids[rptrs[i] + q] / line;", "buf[q] = cids[rptrs[i] + q];"),
]


@pytest.mark.parametrize("name,old,new", UCLD_MUTATIONS, ids=[m[0] for m in UCLD_MUTATIONS])
def test_ucld_planted_mistakes_are_caught(tmp_path, monkeypatch, name, old, new):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    assert old in src
    c = tmp_path / "mut.c"
    c.write_text(src.replace(old, new, 1))
    so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-ffp-contract=off", "-o", str(so), str(c), "-lm"])
    lib = ctypes.CDLL(str(so))
    P, i32 = ctypes.c_void_p, ctypes.c_int
    lib.orc_ucld.argtypes = [i32, P, P, i32, P, P, P]

    def mutant(m, rp, ci, line):
        rp = np.ascontiguousarray(rp, np.int32)
        ci = np.ascontiguousarray(ci, np.int32)
        u, tot, rows = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_longlong()
        lib.orc_ucld(int(m), rp.ctypes.data, ci.ctypes.data if ci.size else 0, int(line), ctypes.byref(u),
                     ctypes.byref(tot), ctypes.byref(rows))
        return u.value, tot.value, rows.value

    monkeypatch.setattr(oracle, "ucld", mutant)
    caught = 0
    for check in (test_ucld_paper_example, test_ucld_closed_forms, test_ucld_brute_force):
        try:
            check()
        except AssertionError:
            caught += 1
    assert caught >= 1, f"no pin caught the planted mistake: {name}"


# ------------------------------------------------------------------ RCM

def _csr_from_edges(n, edges):
    rows = [[] for _ in range(n)]
    for a, b in edges:
        rows[a].append(b)
    rp = np.zeros(n + 1, np.int32)
    rp[1:] = np.cumsum([len(r) for r in rows])
    ci = np.array([c for r in rows for c in sorted(r)], np.int32)
    return rp, ci


def _bandwidth(n, rp, ci):
    rows = np.repeat(np.arange(n), np.diff(rp))
    return int(np.abs(rows - ci).max()) if ci.size else 0


def _sym_degrees(n, rp, ci):
    nb = [set() for _ in range(n)]
    for i in range(n):
        for j in ci[rp[i]:rp[i + 1]]:
            if j != i:
                nb[i].add(int(j))
                nb[int(j)].add(i)
    return nb


def _check_cm_structure(n, rp, ci, perm, rcm=None):
    """The reverse of perm must be a Cuthill-McKee order: isolated nodes first in index order;
    each component starts at a node and continues breadth first, every later node's parent
    (its earliest placed neighbour) placed before it, parents in non-decreasing position, and
    the children of one parent sorted by (degree, index)."""
    rcm = oracle.rcm if rcm is None else rcm
    order = list(perm[::-1])
    assert sorted(order) == list(range(n))
    nb = _sym_degrees(n, rp, ci)
    deg = [len(x) for x in nb]
    pos = {v: i for i, v in enumerate(order)}
    iso = [v for v in order if deg[v] == 0]
    assert order[:len(iso)] == sorted(iso)
    last_parent = -1
    prev = None
    for i in range(len(iso), n):
        v = order[i]
        earlier = [pos[u] for u in nb[v] if pos[u] < i]
        if not earlier:  # a component's first node
            last_parent, prev = -1, None
            continue
        par = min(earlier)
        assert par >= last_parent, "parents out of breadth-first order"
        if par == last_parent:
            assert (deg[prev], prev) < (deg[v], v), "children not sorted by (degree, index)"
        last_parent, prev = par, v


def test_rcm_path_has_bandwidth_one():
    rng = np.random.default_rng(80)
    for n in (2, 3, 17, 200):
        lab = rng.permutation(n)
        rp, ci = _csr_from_edges(n, [(lab[i], lab[i + 1]) for i in range(n - 1)])
        perm = oracle.rcm(n, rp, ci)
        brp, bci, _ = oracle.permute(n, rp, ci, None, perm)
        # A has only one direction of each edge: B's pattern is a relabelled path, bandwidth 1
        assert _bandwidth(n, brp, bci) == 1
        _check_cm_structure(n, rp, ci, perm)


def test_rcm_grid_has_bandwidth_n():
    """Cuthill-McKee from a corner of an N x N grid numbers it by anti-diagonals: bandwidth N."""
    for N in (5, 12, 24):
        A = synth.stencil2d(N)
        lab = np.random.default_rng(N).permutation(A.m)
        brp, bci, _ = oracle.permute(A.m, A.row_ptr, A.col_idx, None, lab)
        perm = oracle.rcm(A.m, brp, bci)
        crp, cci, _ = oracle.permute(A.m, brp, bci, None, perm)
        assert _bandwidth(A.m, crp, cci) == N
        _check_cm_structure(A.m, brp, bci, perm)


def test_rcm_starts_at_a_pseudo_peripheral_node():
    """A spider: centre 0 with arms of 1, 5 and 3 nodes.  The smallest node of degree 1 is the
    1-arm's end, but the George-Liu search moves the start to the end of the 5-arm (the far
    end of a longest path), where the Cuthill-McKee order must begin."""
    arms = [[1], [2, 3, 4, 5, 6], [7, 8, 9]]
    edges = []
    for arm in arms:
        prev = 0
        for v in arm:
            edges.append((prev, v))
            prev = v
    n = 10
    rp, ci = _csr_from_edges(n, edges)
    perm = oracle.rcm(n, rp, ci)
    assert perm[-1] == 6
    _check_cm_structure(n, rp, ci, perm)


def test_rcm_components_and_isolated_nodes():
    rng = np.random.default_rng(81)
    n = 40
    edges = [(3, 5), (5, 9), (20, 21), (21, 22), (22, 20), (30, 31), (31, 3)]
    rp, ci = _csr_from_edges(n, edges)
    perm = oracle.rcm(n, rp, ci)
    touched = {a for e in edges for a in e}
    iso = sorted(set(range(n)) - touched)
    assert list(perm[-len(iso):]) == iso[::-1]  # reversed: isolated nodes last, descending
    _check_cm_structure(n, rp, ci, perm)
    for trial in range(6):
        A = synth.random_csr(80, 80, 0.04, 300 + trial, sorted_cols=bool(trial % 2), duplicates=True,
                             empty_rows=0.3)
        _check_cm_structure(A.m, A.row_ptr, A.col_idx, oracle.rcm(A.m, A.row_ptr, A.col_idx))


def test_rcm_bandwidth_against_scipy():
    """scipy's reverse_cuthill_mckee (its own start and tie rules) as an independent yardstick."""
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    for trial, (side, hbw) in enumerate(((30, 4), (60, 9), (40, 15))):
        n = side * side
        A = synth.banded(n, hbw=hbw, per_row=min(hbw, 6), seed=400 + trial)
        lab = np.random.default_rng(trial).permutation(n)
        brp, bci, _ = oracle.permute(n, A.row_ptr, A.col_idx, None, lab)
        M = sp.csr_matrix((np.ones(bci.size), bci, brp), shape=(n, n))
        S = (M + M.T).tocsr()
        q = csgraph.reverse_cuthill_mckee(S, symmetric_mode=True)
        ours = oracle.rcm(n, brp, bci)
        srp, sci, _ = oracle.permute(n, S.indptr, S.indices, None, ours)
        qrp, qci, _ = oracle.permute(n, S.indptr, S.indices, None, q)
        assert _bandwidth(n, srp, sci) <= 1.5 * _bandwidth(n, qrp, qci) + 2
        assert _bandwidth(n, srp, sci) < _bandwidth(n, *oracle.permute(n, S.indptr, S.indices, None, lab)[:2])


def test_permute_brute_force():
    rng = np.random.default_rng(82)
    for trial in range(8):
        A = synth.random_csr(60, 60, 0.08, 500 + trial, sorted_cols=bool(trial % 2), duplicates=bool(trial % 3 == 0),
                             empty_rows=0.2)
        perm = rng.permutation(A.m).astype(np.int32)
        brp, bci, bv = oracle.permute(A.m, A.row_ptr, A.col_idx, A.vals, perm)
        D = A.to_dense()
        B = synth.CSR(A.m, A.m, brp, bci, bv).to_dense()
        assert np.array_equal(B, D[perm][:, perm])
        for i in range(A.m):
            assert np.all(np.diff(bci[brp[i]:brp[i + 1]]) >= 0)


RCM_MUTATIONS = [
    ("children by index only", "qsort(nb, (size_t)k, sizeof(int), cmp_nodes);", "qsort(nb, (size_t)k, sizeof(int), cmp_int);"),
    ("not reversed", "for (int i = 0; i < n; ++i) perm[i] = order[n - 1 - i];", "for (int i = 0; i < n; ++i) perm[i] = order[i];"),
    ("no pseudo-peripheral search", "if (lx > levels) {", "if (0) {"),
    ("start by index, not degree", "qsort(byrank, (size_t)n, sizeof(int), cmp_nodes); /* nodes by (degree, index) */",
     "; /* nodes by index */"),
]


@pytest.mark.parametrize("name,old,new", RCM_MUTATIONS, ids=[m[0] for m in RCM_MUTATIONS])
def test_rcm_planted_mistakes_are_caught(tmp_path, monkeypatch, name, old, new):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    assert old in src
    c = tmp_path / "mut.c"
    c.write_text(src.replace(old, new, 1))
    so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-ffp-contract=off", "-o", str(so), str(c), "-lm"])
    lib = ctypes.CDLL(str(so))
    P, i32 = ctypes.c_void_p, ctypes.c_int
    lib.orc_rcm.argtypes = [i32, P, P, P]

    def mutant(n, rp, ci):
        rp = np.ascontiguousarray(rp, np.int32)
        ci = np.ascontiguousarray(ci, np.int32)
        perm = np.empty(n, np.int32)
        lib.orc_rcm(int(n), rp.ctypes.data, ci.ctypes.data if ci.size else 0, perm.ctypes.data)
        return perm

    monkeypatch.setattr(oracle, "rcm", mutant)
    caught = 0
    for check in (test_rcm_path_has_bandwidth_one, test_rcm_grid_has_bandwidth_n,
                  test_rcm_starts_at_a_pseudo_peripheral_node, test_rcm_components_and_isolated_nodes):
        try:
            check()
        except AssertionError:
            caught += 1
    assert caught >= 1, f"no pin caught the planted mistake: {name}"


# ------------------------------------------------------- degree relabelling

def _lower_full(n):
    rp = np.concatenate([[0], np.cumsum(np.arange(1, n + 1))]).astype(np.int32)
    ci = np.concatenate([np.arange(i + 1) for i in range(n)]).astype(np.int32)
    return rp, ci


def check_relabel_closed_forms(relabel):
    n = 9
    # full lower triangle: column j holds n - j entries, so the order is the identity
    _, ci = _lower_full(n)
    assert np.array_equal(relabel(n, ci), np.arange(n))
    # full upper triangle: column j holds j + 1 entries, so the hottest is the last column
    ci_up = np.concatenate([np.arange(i, n) for i in range(n)]).astype(np.int32)
    assert np.array_equal(relabel(n, ci_up), np.arange(n)[::-1])
    # a permutation matrix: every column once, all ties, so ties by column id give the identity
    perm = np.random.default_rng(3).permutation(n).astype(np.int32)
    assert np.array_equal(relabel(n, perm), np.arange(n))
    # a rectangular matrix with one hub column (5), two columns of two entries (1, 7) and empty
    # columns: 5 first, then 1 and 7 by id, then the once-used 2, then the empty 0, 3, 4, 6, 8, 9
    ci = np.array([5, 1, 5, 7, 5, 2, 1, 5, 7], np.int32)
    want = np.empty(10, np.int32)
    want[[5, 1, 7, 2, 0, 3, 4, 6, 8, 9]] = np.arange(10)
    assert np.array_equal(relabel(10, ci), want)
    # no entries at all: every column ties, identity
    assert np.array_equal(relabel(4, np.zeros(0, np.int32)), np.arange(4))


def check_relabel_brute_force(relabel):
    for trial in range(6):
        A = synth.random_csr(40 + trial, 57, 0.1, 600 + trial, sorted_cols=bool(trial % 2), duplicates=True)
        deg = np.bincount(A.col_idx, minlength=A.n)
        order = np.lexsort((np.arange(A.n), -deg))  # degree descending, then column id
        want = np.empty(A.n, np.int64)
        want[order] = np.arange(A.n)
        got = relabel(A.n, A.col_idx)
        assert np.array_equal(got, want), trial
        assert np.array_equal(np.sort(got), np.arange(A.n))


def check_relabel_product_unchanged(relabel):
    """A' x' = A x bitwise: each row keeps its terms in storage order, with the same values."""
    for A in (synth.rmat(9, ef=8, seed=610), synth.random_csr(70, 90, 0.07, 611, duplicates=True, empty_rows=0.2)):
        x = synth.uniform(A.n, seed=612)
        newid = relabel(A.n, A.col_idx)
        xp = np.empty_like(x)
        xp[newid] = x
        y, r = oracle.spmv(A.m, A.row_ptr, A.col_idx, A.vals, x)
        y2, r2 = oracle.spmv(A.m, A.row_ptr, newid[A.col_idx], A.vals, xp)
        assert np.array_equal(y, y2) and np.array_equal(r, r2)


def test_relabel_closed_forms():
    check_relabel_closed_forms(oracle.degree_relabel)


def test_relabel_brute_force():
    check_relabel_brute_force(oracle.degree_relabel)


def test_relabel_product_unchanged():
    check_relabel_product_unchanged(oracle.degree_relabel)


def test_relabel_power_law_puts_the_hub_columns_first():
    """On R-MAT (a, b, c, d = 0.57, 0.19, 0.19, 0.05) column 0 is the most likely at every level, so
    it is the hottest; the top 1 % of the relabelled columns hold far more than 1 % of the entries."""
    A = synth.rmat(14, ef=16, seed=613)
    newid = oracle.degree_relabel(A.n, A.col_idx)
    assert newid[0] == 0
    deg = np.bincount(newid[A.col_idx], minlength=A.n)
    assert np.all(np.diff(deg) <= 0)
    assert deg[: A.n // 100].sum() > 0.1 * A.nnz


RELABEL_MUTATIONS = [
    ("coldest first", "return g_rl_deg[ja] > g_rl_deg[jb] ? -1 : 1;", "return g_rl_deg[ja] < g_rl_deg[jb] ? -1 : 1;"),
    ("ties by descending id", "return (ja > jb) - (ja < jb);                                                   /* then",
     "return (jb > ja) - (jb < ja);                                                   /* then"),
    ("order not inverted", "for (int q = 0; q < n; ++q) newid[order[q]] = q;",
     "for (int q = 0; q < n; ++q) newid[q] = order[q];"),
    ("repeats counted once", "deg[cids[p]] += 1;", "deg[cids[p]] = 1;"),
]


@pytest.mark.parametrize("name,old,new", RELABEL_MUTATIONS, ids=[m[0] for m in RELABEL_MUTATIONS])
def test_relabel_planted_mistakes_are_caught(tmp_path, name, old, new):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    assert old in src
    c = tmp_path / "mut.c"
    c.write_text(src.replace(old, new, 1))
    so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-ffp-contract=off", "-o", str(so), str(c), "-lm"])
    lib = ctypes.CDLL(str(so))
    P, i32 = ctypes.c_void_p, ctypes.c_int
    lib.orc_degree_relabel.argtypes = [i32, i32, P, P]

    def mutant(n, ci):
        ci = np.ascontiguousarray(ci, np.int32)
        newid = np.empty(n, np.int32)
        lib.orc_degree_relabel(int(n), int(ci.size), ci.ctypes.data if ci.size else 0, newid.ctypes.data)
        return newid

    caught = 0
    for check in (check_relabel_closed_forms, check_relabel_brute_force):
        try:
            check(mutant)
        except AssertionError:
            caught += 1
    assert caught >= 1, f"no pin caught the planted mistake: {name}"


# ----------------------------------------------------------------- BCSR

def _bcsr_dense(m, n, a, b, bptr, bcol, bval):
    D = np.zeros((((m + a - 1) // a) * a, (max(int(bcol.max()) + 1 if bcol.size else 0, (n + b - 1) // b)) * b))
    for I in range(bptr.size - 1):
        for k in range(bptr[I], bptr[I + 1]):
            D[I * a:(I + 1) * a, bcol[k] * b:(bcol[k] + 1) * b] += bval[k * a * b:(k + 1) * a * b].reshape(a, b)
    return D


BLOCKS = [(8, 1), (1, 8), (2, 8), (4, 8), (8, 4), (8, 2), (8, 8), (3, 5), (1, 1)]


def test_bcsr_expands_back_to_a():
    rng = np.random.default_rng(90)
    for trial in range(10):
        m, n = int(rng.integers(1, 70)), int(rng.integers(1, 70))
        A = synth.random_csr(m, n, float(rng.uniform(0.01, 0.4)), 600 + trial, sorted_cols=bool(trial % 2),
                             duplicates=bool(trial % 3 == 0), empty_rows=0.2)
        D = A.to_dense()
        for a, b in BLOCKS:
            bptr, bcol, bval = oracle.bcsr(A.m, A.n, A.row_ptr, A.col_idx, A.vals, a, b)
            E = _bcsr_dense(A.m, A.n, a, b, bptr, bcol, bval)
            assert np.array_equal(E[:m, :n], D)
            assert not E[m:, :].any() and not E[:, n:].any()
            for I in range(bptr.size - 1):  # block columns strictly increasing: no repeated block
                assert np.all(np.diff(bcol[bptr[I]:bptr[I + 1]]) > 0)
            # every stored block holds at least one stored entry of A
            rows = np.repeat(np.arange(A.m), A.row_lengths())
            keys = set(zip(rows // a, A.col_idx // b))
            got = {(I, int(bcol[k])) for I in range(bptr.size - 1) for k in range(bptr[I], bptr[I + 1])}
            assert got == keys
            x = rng.uniform(-1, 1, A.n)
            y, r = oracle.bcsr_spmv(A.m, A.n, a, b, bptr, bcol, bval, x)
            assert np.allclose(y, D @ x, rtol=0, atol=1e-13)
            assert np.allclose(r, np.abs(E[:m, :n]) @ np.abs(x), rtol=1e-13, atol=1e-15)


def test_bcsr_closed_forms():
    n = 64
    I = synth.CSR(n, n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.ones(n))
    for a, b in BLOCKS:
        bptr, bcol, _ = oracle.bcsr(n, n, I.row_ptr, I.col_idx, I.vals, a, b)
        # identity: block (i // a, i // b) for every i, so the blocks are the distinct pairs
        assert bcol.size == len({(i // a, i // b) for i in range(n)})
    assert oracle.bcsr(n, n, I.row_ptr, I.col_idx, I.vals, 8, 8)[1].size == 8
    assert oracle.bcsr(n, n, I.row_ptr, I.col_idx, I.vals, 8, 1)[1].size == n
    # dense 13 x 21: every region is a block
    Dn = np.arange(1, 13 * 21 + 1, dtype=np.float64).reshape(13, 21)
    rp = np.arange(0, 13 * 21 + 1, 21, dtype=np.int32)
    ci = np.tile(np.arange(21, dtype=np.int32), 13)
    for a, b in BLOCKS:
        bptr, bcol, bval = oracle.bcsr(13, 21, rp, ci, Dn.reshape(-1), a, b)
        assert bcol.size == ((13 + a - 1) // a) * ((21 + b - 1) // b)
    # the dof-8 block stencil fills 8 x 8 blocks exactly: one block per node coupling
    N = 4
    B = synth.stencil3d_blocks(N, 8)
    bptr, bcol, bval = oracle.bcsr(B.m, B.n, B.row_ptr, B.col_idx, B.vals, 8, 8)
    assert bcol.size == (3 * N - 2) ** 3 and bval.size == B.nnz and np.all(bval != 0)


BCSR_MUTATIONS = [
    # every replacement stays in bounds
    ("column mirrored inside the block", "bval[k * a * b + (long long)(i - r0) * b + (cids[p] - J * b)] += val[p];",
     "bval[k * a * b + (long long)(i - r0) * b + (b - 1 - (cids[p] - J * b))] += val[p];"),
    ("repeats overwrite", "bval[k * a * b + (long long)(i - r0) * b + (cids[p] - J * b)] += val[p];",
     "bval[k * a * b + (long long)(i - r0) * b + (cids[p] - J * b)] = val[p];"),
    ("block columns not made unique", "if (q == 0 || buf[q] != buf[q - 1]) {", "if (1) {"),
    ("abs bound without abs", "t = t + fabs(pr);", "t = t + pr;"),
]


@pytest.mark.parametrize("name,old,new", BCSR_MUTATIONS, ids=[m[0] for m in BCSR_MUTATIONS])
def test_bcsr_planted_mistakes_are_caught(tmp_path, monkeypatch, name, old, new):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    assert old in src
    c = tmp_path / "mut.c"
    c.write_text(src.replace(old, new, 1))
    so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-ffp-contract=off", "-o", str(so), str(c), "-lm"])
    lib = ctypes.CDLL(str(so))
    P, i32, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong
    lib.orc_bcsr.argtypes = [i32, i32, P, P, P, i32, i32, P, P, P]
    lib.orc_bcsr.restype = ll
    lib.orc_bcsr_spmv.argtypes = [i32, i32, i32, i32, P, P, P, P, P, P]

    def bcsr(m, n, rp, ci, v, a, b):
        rp, ci, v = (np.ascontiguousarray(x, t) for x, t in ((rp, np.int32), (ci, np.int32), (v, np.float64)))
        nb = lib.orc_bcsr(m, n, rp.ctypes.data, ci.ctypes.data if ci.size else 0, v.ctypes.data if v.size else 0,
                          a, b, None, None, None)
        bptr, bcol, bval = np.empty((m + a - 1) // a + 1, np.int32), np.empty(nb, np.int32), np.empty(nb * a * b)
        lib.orc_bcsr(m, n, rp.ctypes.data, ci.ctypes.data if ci.size else 0, v.ctypes.data if v.size else 0, a, b,
                     bptr.ctypes.data, bcol.ctypes.data if nb else 0, bval.ctypes.data if nb else 0)
        return bptr, bcol, bval

    def bcsr_spmv(m, n, a, b, bptr, bcol, bval, x):
        y, r = np.empty(m), np.empty(m)
        x = np.ascontiguousarray(x, np.float64)
        lib.orc_bcsr_spmv(m, n, a, b, bptr.ctypes.data, bcol.ctypes.data if bcol.size else 0,
                          bval.ctypes.data if bval.size else 0, x.ctypes.data, y.ctypes.data, r.ctypes.data)
        return y, r

    monkeypatch.setattr(oracle, "bcsr", bcsr)
    monkeypatch.setattr(oracle, "bcsr_spmv", bcsr_spmv)
    caught = 0
    for check in (test_bcsr_expands_back_to_a, test_bcsr_closed_forms):
        try:
            check()
        except (AssertionError, ValueError, IndexError):
            caught += 1
    assert caught >= 1, f"no pin caught the planted mistake: {name}"


# ---------------------------------------------- planted mistakes (mutation)

MUTATIONS = [
    # (name, text in oracle.c, replacement); every replacement stays in bounds
    ("dropped last term", "for (int p = rptrs[i]; p < rptrs[i + 1]; ++p) {\n      double t = val[p] * x[cids[p]];",
     "for (int p = rptrs[i]; p + 1 < rptrs[i + 1]; ++p) {\n      double t = val[p] * x[cids[p]];"),
    ("dropped first term", "for (int p = rptrs[i]; p < rptrs[i + 1]; ++p) {\n      double t = val[p] * x[cids[p]];",
     "for (int p = rptrs[i] + 1; p < rptrs[i + 1]; ++p) {\n      double t = val[p] * x[cids[p]];"),
    ("wrong sign", "s = s + t;", "s = s - t;"),
    ("wrong x index", "double t = val[p] * x[cids[p]];", "double t = val[p] * x[cids[rptrs[i]]];"),
    ("wrong value index", "double t = val[p] * x[cids[p]];", "double t = val[rptrs[i]] * x[cids[p]];"),
    ("abs bound without abs", "a = a + fabs(t);", "a = a + t;"),
]


def _build_mutant(tmp_path, old, new):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    assert old in src
    mutated = src.replace(old, new, 1)
    c = tmp_path / "mut.c"
    c.write_text(mutated)
    so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-ffp-contract=off", "-o", str(so), str(c), "-lm"])
    lib = ctypes.CDLL(str(so))
    P, i32 = ctypes.c_void_p, ctypes.c_int
    lib.orc_spmv_f64.argtypes = [i32, P, P, P, P, P, P, i32]

    def spmv(m, rp, ci, v, x):
        rp = np.ascontiguousarray(rp, np.int32)
        ci = np.ascontiguousarray(ci, np.int32)
        v = np.ascontiguousarray(v, np.float64)
        x = np.ascontiguousarray(x, np.float64)
        y = np.empty(m)
        r = np.empty(m)
        lib.orc_spmv_f64(m, rp.ctypes.data, ci.ctypes.data if ci.size else 0, v.ctypes.data if v.size else 0,
                         x.ctypes.data, y.ctypes.data, r.ctypes.data, 1)
        return y, r

    return spmv


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistakes_are_caught(tmp_path, name, old, new):
    spmv = _build_mutant(tmp_path, old, new)
    caught = 0
    for check in (check_spmv_closed_forms, check_spmv_permutation, check_spmv_brute_force):
        try:
            check(spmv)
        except AssertionError:
            caught += 1
    assert caught >= 1, f"no pin caught the planted mistake: {name}"
