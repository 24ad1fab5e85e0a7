"""Transpose (bit-exact) and backward (dX = A^T dY, dvals) of the CUDA path against the
CPU oracle, plus central finite differences through the autograd Function."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 2e-5}
NP = {torch.float64: np.float64, torch.float32: np.float32}


@pytest.fixture(scope="module")
def gbs():
    import paper_1302_1078_gb300 as g

    g.lib()
    return g


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def within(got, ref, bound, dtype, what):
    g = got.detach().double().cpu().numpy().reshape(ref.shape)
    bad = np.abs(g - ref) > TOL[dtype] * bound
    assert not bad.any(), f"{what}: {bad.sum()} entries off, e.g. {g[bad][:3]} vs {ref[bad][:3]}"
    assert np.all(g[bound == 0] == 0), f"{what}: nonzero where the bound is 0"


CASES = {
    "random_rect": lambda: synth.random_csr(300, 170, 0.05, 1, empty_rows=0.2),
    "random_tall": lambda: synth.random_csr(170, 300, 0.05, 2, empty_rows=0.2),
    "dup_unsorted": lambda: synth.random_csr(200, 200, 0.05, 3, sorted_cols=False, duplicates=True),
    "stencil2d_37": lambda: synth.stencil2d(37),
    "banded_20k": lambda: synth.banded(20000, hbw=1000, per_row=30, seed=4),
    "rmat_14": lambda: synth.rmat(14, ef=16, seed=5, vals="u0.5_1.5"),
    "one_col": lambda: synth.CSR(5000, 1, np.arange(5001, dtype=np.int32), np.zeros(5000, np.int32),
                                 np.linspace(-1, 1, 5000)),
    "empty": lambda: synth.random_csr(50, 60, 0.0, 6),
}
_cache = {}


def case(name):
    if name not in _cache:
        _cache[name] = CASES[name]()
    return _cache[name]


@pytest.mark.parametrize("name", list(CASES))
def test_transpose_bit_exact(gbs, name):
    A = case(name)
    rpT, ciT, perm = oracle.transpose(A.m, A.n, A.row_ptr, A.col_idx)
    t = gbs.TransposePlan(dev(A.row_ptr), dev(A.col_idx), A.n)
    g_rpT, g_ciT, g_perm = (x.cpu().numpy() for x in t.arrays())
    assert np.array_equal(g_rpT, rpT)
    assert np.array_equal(g_ciT, ciT)
    assert np.array_equal(g_perm, perm)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("k", [1, 3, 8, 16])
@pytest.mark.parametrize("name", list(CASES))
def test_backward_matches_oracle(gbs, name, k, dtype):
    A = case(name)
    v = A.vals.astype(NP[dtype])
    X = synth.uniform(A.n * k, seed=11, stream=k).reshape(A.n, k).astype(NP[dtype])
    W = synth.uniform(A.m * k, seed=12, stream=k).reshape(A.m, k).astype(NP[dtype])
    dX_ref, dv_ref, RdX, Rdv = oracle.backward(A.m, A.n, A.row_ptr, A.col_idx, v, X, W)
    t = gbs.TransposePlan(dev(A.row_ptr), dev(A.col_idx), A.n)
    vd = dev(v)
    if k == 1:
        dX, dvals = t.backward(vd, dev(X[:, 0]), dev(W[:, 0]))
    else:
        dX, dvals = t.backward(vd, dev(X), dev(W))
    within(dX, dX_ref, RdX, dtype, f"dX {name} k={k}")
    within(dvals, dv_ref, Rdv, dtype, f"dvals {name} k={k}")
    # determinism
    dX2, dvals2 = t.backward(vd, dev(X) if k > 1 else dev(X[:, 0]), dev(W) if k > 1 else dev(W[:, 0]))
    assert torch.equal(dX, dX2) and torch.equal(dvals, dvals2)


def rows_chunk_edges():
    """Row lengths that put row boundaries, empty rows and long rows across the 128-nonzero chunks
    the dvals pass uses to find each nonzero's row."""
    rng = np.random.default_rng(41)
    lens = [0] * 300 + [1000] + [0] * 300 + [1] * 257 + [129, 127, 128, 0, 0, 255, 1] + [0] * 50 + [3] * 40 + [0]
    lens = np.array(lens, dtype=np.int64)
    rp = np.zeros(lens.size + 1, dtype=np.int32)
    rp[1:] = np.cumsum(lens)
    n = 1200
    ci = np.concatenate([np.sort(rng.choice(n, size=l, replace=False)) for l in lens]).astype(np.int32)
    return synth.CSR(lens.size, n, rp, ci, synth.normal(int(rp[-1]), seed=42))


CASES["chunk_edges"] = rows_chunk_edges

V = {"ROWS": 1, "MERGE": 2, "ROWS_TMA": 3, "MERGE_DIRECT": 4}
AT_CONFIGS = [
    # values read in place through the transpose permutation
    dict(variant=V["ROWS"], lanes=1, threads=256, tile_nnz=2048),
    dict(variant=V["ROWS"], lanes=2, threads=128, tile_nnz=64),
    dict(variant=V["ROWS"], lanes=8, threads=256, tile_nnz=512),
    dict(variant=V["ROWS"], lanes=32, threads=64, tile_nnz=96),
    dict(variant=V["MERGE_DIRECT"], threads=256, items=31),
    dict(variant=V["MERGE_DIRECT"], threads=64, items=7),
    dict(variant=V["MERGE_DIRECT"], threads=128, items=63),
    dict(variant=V["MERGE"], threads=256, items=11),
    dict(variant=V["MERGE"], threads=128, items=7),
    # values permuted into scratch first
    dict(variant=V["ROWS_TMA"], lanes=2, threads=64),
]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("k", [1, 8])
@pytest.mark.parametrize("ci", range(len(AT_CONFIGS)))
@pytest.mark.parametrize("name", ["random_rect", "dup_unsorted", "stencil2d_37", "rmat_14", "chunk_edges", "empty"])
def test_backward_dX_configs(gbs, name, ci, k, dtype):
    """Every dX route (values through perm, or permuted first) on every variant against the oracle."""
    A = case(name)
    cfg = AT_CONFIGS[ci]
    v = A.vals.astype(NP[dtype])
    X = synth.uniform(A.n * k, seed=13, stream=k).reshape(A.n, k).astype(NP[dtype])
    W = synth.uniform(A.m * k, seed=14, stream=k).reshape(A.m, k).astype(NP[dtype])
    dX_ref, dv_ref, RdX, Rdv = oracle.backward(A.m, A.n, A.row_ptr, A.col_idx, v, X, W)
    t = gbs.TransposePlan(dev(A.row_ptr), dev(A.col_idx), A.n)
    try:
        t.set_config(dtype, k, cfg)
    except gbs._capi.GbsError as e:
        # ROWS_TMA stages a whole row block: A^T of a power-law matrix can exceed it
        if e.status == gbs._capi.GBS_EUNSUPPORTED and cfg["variant"] == V["ROWS_TMA"]:
            pytest.skip(str(e))
        raise
    got = t.config(dtype, k)
    assert got["variant"] == cfg["variant"]
    Xa, Wa = (dev(X[:, 0]), dev(W[:, 0])) if k == 1 else (dev(X), dev(W))
    dX, dvals = t.backward(dev(v), Xa, Wa)
    within(dX, dX_ref, RdX, dtype, f"dX {name} k={k} {cfg}")
    within(dvals, dv_ref, Rdv, dtype, f"dvals {name} k={k}")
    dX2, _ = t.backward(dev(v), Xa, Wa, need_dvals=False)
    assert torch.equal(dX, dX2)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("k", [1, 8])
@pytest.mark.parametrize("name", ["banded_20k", "rmat_14", "chunk_edges"])
def test_backward_prepared_tuned(gbs, name, k, dtype):
    """dX through a tuned plan of A^T (either route) against the oracle; idempotent prepare."""
    A = case(name)
    v = A.vals.astype(NP[dtype])
    X = synth.uniform(A.n * k, seed=15, stream=k).reshape(A.n, k).astype(NP[dtype])
    W = synth.uniform(A.m * k, seed=16, stream=k).reshape(A.m, k).astype(NP[dtype])
    dX_ref, _, RdX, _ = oracle.backward(A.m, A.n, A.row_ptr, A.col_idx, v, X, W)
    t = gbs.TransposePlan(dev(A.row_ptr), dev(A.col_idx), A.n)
    t.prepare(dtype, k, tune=True)
    cfg = t.config(dtype, k)
    t.prepare(dtype, k, tune=True)
    assert t.config(dtype, k) == cfg
    Xa, Wa = (dev(X[:, 0]), dev(W[:, 0])) if k == 1 else (dev(X), dev(W))
    dX, dvals = t.backward(dev(v), Xa, Wa, need_dvals=False)
    assert dvals is None
    within(dX, dX_ref, RdX, dtype, f"dX {name} k={k} tuned {cfg}")


def test_backward_config_errors(gbs):
    A = case("random_rect")
    t = gbs.TransposePlan(dev(A.row_ptr), dev(A.col_idx), A.n)
    with pytest.raises(Exception):
        t.set_config(torch.float64, 1, dict(variant=V["ROWS"], lanes=3))
    with pytest.raises(Exception):
        t.set_config(torch.float64, 0, dict(variant=V["ROWS"]))
    # AUTO: the statistics-based configuration, values in place
    t.set_config(torch.float64, 1, dict(variant=0))
    assert t.config(torch.float64, 1)["variant"] in (V["ROWS"], V["MERGE"], V["MERGE_DIRECT"])


def test_autograd_gradcheck(gbs):
    A = synth.random_csr(12, 9, 0.3, 21, empty_rows=0.2)
    op = gbs.CsrOperator(dev(A.row_ptr), dev(A.col_idx), A.n)
    vals = dev(A.vals).requires_grad_(True)
    X = torch.rand(A.n, 3, dtype=torch.float64, device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda v, x: op(v, x), (vals, X), eps=1e-6, atol=1e-9, rtol=1e-7)
    x1 = torch.rand(A.n, dtype=torch.float64, device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda v, x: op(v, x), (vals, x1), eps=1e-6, atol=1e-9, rtol=1e-7)


def fd_checks(gbs, A, k, dtype=torch.float64, h=1e-6, ndir=8, ncoord=64, seed=0):
    """Central differences of L(vals, X) = <A X, W> against the autograd gradients.

    L is bilinear, so a central difference is exact up to rounding.  The differences are
    formed entry by entry ((Y+ - Y-) . W), so unchanged entries cancel exactly.  Each check
    allows 1e-7 * |g| plus the difference's own rounding bound, derived from the arithmetic:
    an entry Y_i summed over len_i products carries an error of about
    eps * sqrt(len_i + 1) * (sum_p |a_p x_p| + |Y_i|), and dividing by 2h magnifies it."""
    rng = np.random.default_rng(seed)
    eps = 2.0 ** -52
    op = gbs.CsrOperator(dev(A.row_ptr), dev(A.col_idx), A.n)
    v0 = dev(A.vals.astype(NP[dtype]))
    Xh = synth.uniform(A.n * k, seed=31, stream=k).reshape(A.n, k).astype(NP[dtype])
    X0 = dev(Xh[:, 0]) if k == 1 else dev(Xh)
    W = dev(synth.uniform(A.m * k, seed=32, stream=k).astype(NP[dtype]))
    W = W if k == 1 else W.reshape(A.m, k)
    lens = dev(np.sqrt(A.row_lengths().astype(np.float64) + 1.0))
    lens = lens if k == 1 else lens[:, None]
    R = op.forward_raw(v0.abs(), X0.abs())  # sum_p |a_p x_p| per entry
    vals = v0.clone().requires_grad_(True)
    X = X0.clone().requires_grad_(True)
    L = (op(vals, X) * W).sum()
    gv, gx = torch.autograd.grad(L, (vals, X))

    def fd(dv, dx):
        Yp = op.forward_raw(v0 + h * dv, X0 + h * dx)
        Ym = op.forward_raw(v0 - h * dv, X0 - h * dx)
        d = Yp - Ym
        changed = d != 0
        err = 2 * eps * float((lens * (R + Yp.abs()) * W.abs() * changed).sum()) / (2 * h)
        return float((d * W).sum()) / (2 * h), err

    def check(pair, g):
        val, err = pair
        assert abs(val - g) <= 1e-7 * abs(g) + err + 1e-12, (val, g, err)

    for _ in range(ndir):
        dv = dev(rng.uniform(-1, 1, A.nnz))
        dx = dev(rng.uniform(-1, 1, tuple(X0.shape)))
        zero_v, zero_x = torch.zeros_like(dv), torch.zeros_like(dx)
        check(fd(dv, zero_x), float((gv * dv).sum()))
        check(fd(zero_v, dx), float((gx * dx).sum()))
    for _ in range(ncoord):
        p = int(rng.integers(A.nnz))
        e = torch.zeros(A.nnz, dtype=dtype, device="cuda")
        e[p] = 1
        check(fd(e, torch.zeros_like(X0)), float(gv[p]))
        j = int(rng.integers(A.n))
        ex = torch.zeros_like(X0)
        if k == 1:
            ex[j] = 1
            g = float(gx[j])
        else:
            c = int(rng.integers(k))
            ex[j, c] = 1
            g = float(gx[j, c])
        check(fd(torch.zeros_like(v0), ex), g)
    return gv, gx


@pytest.mark.parametrize("k", [1, 8])
def test_finite_differences_small(gbs, k):
    fd_checks(gbs, case("rmat_14"), k, ndir=4, ncoord=16)


# ----------------------------------------- full size: R-MAT scale 20, edge factor 16

@pytest.fixture(scope="module")
def rmat20():
    return synth.rmat(20, ef=16, seed=synth.BASE_SEED + 3, vals="u0.5_1.5")


def test_full_transpose_rmat20(gbs, rmat20):
    A = rmat20
    rpT, ciT, perm = oracle.transpose(A.m, A.n, A.row_ptr, A.col_idx)
    t = gbs.TransposePlan(dev(A.row_ptr), dev(A.col_idx), A.n)
    g = [x.cpu().numpy() for x in t.arrays()]
    assert np.array_equal(g[0], rpT) and np.array_equal(g[1], ciT) and np.array_equal(g[2], perm)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("k", [1, 8])
def test_full_backward_rmat20(gbs, rmat20, k, dtype):
    A = rmat20
    v = A.vals.astype(NP[dtype])
    X = synth.uniform(A.n * k, seed=41, stream=k).reshape(A.n, k).astype(NP[dtype])
    W = synth.uniform(A.m * k, seed=42, stream=k).reshape(A.m, k).astype(NP[dtype])
    dX_ref, dv_ref, RdX, Rdv = oracle.backward(A.m, A.n, A.row_ptr, A.col_idx, v, X, W)
    op = gbs.CsrOperator(dev(A.row_ptr), dev(A.col_idx), A.n)
    vals = dev(v).requires_grad_(True)
    Xd = (dev(X[:, 0]) if k == 1 else dev(X)).requires_grad_(True)
    Wd = dev(W[:, 0]) if k == 1 else dev(W)
    Y = op(vals, Xd)
    Y_ref, R = oracle.spmm(A.m, A.row_ptr, A.col_idx, v, X)
    within(Y, Y_ref, R, dtype, "forward")
    gv, gx = torch.autograd.grad((Y * Wd).sum(), (vals, Xd))
    within(gx, dX_ref, RdX, dtype, "dX")
    within(gv, dv_ref, Rdv, dtype, "dvals")


@pytest.mark.parametrize("k", [1, 8])
def test_full_finite_differences_rmat20(gbs, rmat20, k):
    fd_checks(gbs, rmat20, k, ndir=8, ncoord=64, seed=k)
