"""Parity of the CUDA SpMV / SpMM path (through the C ABI) with the CPU oracle.

Bound (per output entry): |y_gpu - y_oracle| <= tol * sum_p |a_p x_p|, with
tol = 1e-12 for FP64 and 2e-5 for FP32 inputs; an entry whose bound is 0 must
be exactly 0.  Index-valued facts (closed forms with integer results,
permutations) must match bitwise.
"""
import ctypes

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


def dev_csr(A: synth.CSR, dtype=torch.float64):
    d = torch.device("cuda:0")
    return (torch.from_numpy(A.row_ptr).to(d), torch.from_numpy(A.col_idx).to(d),
            torch.from_numpy(A.vals.astype(NP[dtype])).to(d))


def assert_close(y_gpu, y_ref, r, dtype, what=""):
    y = y_gpu.double().cpu().numpy().reshape(y_ref.shape)
    err = np.abs(y - y_ref)
    tol = TOL[dtype]
    bad = err > tol * r
    if bad.any():
        i = np.argwhere(bad)[0]
        raise AssertionError(f"{what}: {bad.sum()} entries off; first {tuple(i)}: gpu {y[tuple(i)]!r} "
                             f"oracle {y_ref[tuple(i)]!r} bound {tol * r[tuple(i)]!r}")
    zero = r == 0
    assert np.all(y[zero] == 0.0), f"{what}: entries with zero bound are not exactly 0"


def spmv_ref(A, x, dtype):
    v = A.vals.astype(NP[dtype])
    return oracle.spmv(A.m, A.row_ptr, A.col_idx, v, x.astype(NP[dtype]))


def hub_matrix():
    """Empty rows around one 100k-nonzero row and a few short ones."""
    m, n = 64, 200000
    lens = np.zeros(m, np.int64)
    lens[5] = 100000
    lens[6:12] = 3
    lens[40] = 7000
    rp = np.zeros(m + 1, np.int64)
    np.cumsum(lens, out=rp[1:])
    rng = np.random.default_rng(5)
    ci = np.concatenate([np.sort(rng.choice(n, int(l), replace=False)) for l in lens if l > 0]).astype(np.int32)
    v = rng.uniform(-1, 1, ci.size)
    return synth.CSR(m, n, rp.astype(np.int32), ci, v, "hub")


MATRICES = {
    "stencil2d_64": lambda: synth.stencil2d(64),
    "stencil2d_37": lambda: synth.stencil2d(37),
    "stencil3d_21": lambda: synth.stencil3d(21),
    "banded_30k": lambda: synth.banded(30001, hbw=1000, per_row=50, seed=3),
    "rmat_14": lambda: synth.rmat(14, ef=16, seed=4),
    "random_rect": lambda: synth.random_csr(333, 1201, 0.02, 5, empty_rows=0.3),
    "random_dup_unsorted": lambda: synth.random_csr(257, 257, 0.05, 6, sorted_cols=False, duplicates=True),
    "empty_nnz": lambda: synth.random_csr(100, 50, 0.0, 7),
    "one_row": lambda: synth.random_csr(1, 5000, 0.5, 8),
    "hub": hub_matrix,
}

_cache = {}


def matrix(name):
    if name not in _cache:
        _cache[name] = MATRICES[name]()
    return _cache[name]


CONFIGS = [None,
           dict(variant=1, lanes=1), dict(variant=1, lanes=2), dict(variant=1, lanes=4), dict(variant=1, lanes=8),
           dict(variant=1, lanes=16), dict(variant=1, lanes=32),
           dict(variant=1, lanes=1, threads=64, tile_nnz=64), dict(variant=1, lanes=4, threads=128, tile_nnz=100),
           dict(variant=2, items=1), dict(variant=2, items=4), dict(variant=2, items=16, threads=64),
           dict(variant=2, items=7, threads=96),
           dict(variant=4, items=1), dict(variant=4, items=5), dict(variant=4, items=31),
           dict(variant=4, items=63, threads=128), dict(variant=4, items=9, threads=96),
           dict(variant=5), dict(variant=5, threads=64), dict(variant=5, threads=1024)]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("name", list(MATRICES))
def test_spmv_parity_all_variants(gbs, name, dtype):
    A = matrix(name)
    x = synth.uniform(A.n, seed=synth.BASE_SEED, stream=11)
    y_ref, r = spmv_ref(A, x, dtype)
    rp, ci, v = dev_csr(A, dtype)
    xd = torch.from_numpy(x.astype(NP[dtype])).cuda()
    for cfg in CONFIGS:
        y = torch.full((A.m,), float("nan"), dtype=dtype, device="cuda")
        gbs.spmv_csr(rp, ci, v, xd, y, config=cfg)
        assert_close(y, y_ref, r, dtype, f"{name} {cfg}")


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 8, 16, 33, 70])
@pytest.mark.parametrize("name", ["stencil2d_37", "banded_30k", "rmat_14", "random_rect", "hub", "empty_nnz"])
def test_spmm_parity(gbs, name, k, dtype):
    A = matrix(name)
    if name == "hub" and k > 16:
        pytest.skip("covered by smaller k")
    rng = np.random.default_rng(k)
    ld = k + 3  # row stride > k: exercises the narrow-access path
    Xw = synth.uniform(A.n * ld, seed=synth.BASE_SEED, stream=100 + k).reshape(A.n, ld).astype(NP[dtype])
    X = Xw[:, :k]
    Y_ref, R = oracle.spmm(A.m, A.row_ptr, A.col_idx, A.vals.astype(NP[dtype]), X)
    rp, ci, v = dev_csr(A, dtype)
    Xd_wide = torch.from_numpy(Xw).cuda()
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    for cfg in [None, dict(variant=1), dict(variant=1, threads=128, tile_nnz=500), dict(variant=2),
                dict(variant=2, items=3, threads=128), dict(variant=4), dict(variant=4, items=13, threads=128),
                dict(variant=5), dict(variant=5, threads=96)]:
        for XX in (Xd, Xd_wide[:, :k]):
            Y = torch.full((A.m, k), float("nan"), dtype=dtype, device="cuda")
            gbs.spmm_csr(rp, ci, v, XX, Y, config=cfg)
            assert_close(Y, Y_ref, R, dtype, f"{name} k={k} {cfg} ld={XX.stride(0)}")
    del rng


def test_stencil_closed_forms_bitwise(gbs):
    N = 50
    A = synth.stencil2d(N)
    rp, ci, v = dev_csr(A)
    i, j = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    miss = ((i == 0).astype(int) + (i == N - 1) + (j == 0) + (j == N - 1)).reshape(-1).astype(float)
    for cfg in CONFIGS:
        y = gbs.spmv_csr(rp, ci, v, torch.ones(A.n, dtype=torch.float64, device="cuda"), config=cfg)
        assert np.array_equal(y.cpu().numpy(), miss), cfg


def test_permutation_bitwise(gbs):
    rng = np.random.default_rng(3)
    m = 100003
    pi = rng.permutation(m).astype(np.int32)
    rp = torch.arange(m + 1, dtype=torch.int32, device="cuda")
    ci = torch.from_numpy(pi).cuda()
    v = torch.ones(m, dtype=torch.float64, device="cuda")
    x = torch.from_numpy(rng.uniform(-1, 1, m)).cuda()
    for cfg in CONFIGS:
        y = gbs.spmv_csr(rp, ci, v, x, config=cfg)
        assert torch.equal(y, x[ci.long()]), cfg


def test_determinism_bitwise(gbs):
    A = matrix("rmat_14")
    rp, ci, v = dev_csr(A)
    x = torch.from_numpy(synth.uniform(A.n, seed=1)).cuda()
    for cfg in CONFIGS:
        y1 = gbs.spmv_csr(rp, ci, v, x, config=cfg)
        y2 = gbs.spmv_csr(rp, ci, v, x, config=cfg)
        assert torch.equal(y1, y2), cfg


@pytest.mark.parametrize("k", [1, 8])
def test_plans_and_tuner(gbs, k):
    for name in ("stencil3d_21", "rmat_14", "hub"):
        A = matrix(name)
        rp, ci, v = dev_csr(A)
        plan = gbs.Plan(rp, ci, A.n, torch.float64, k, tune=True, check=True)
        st = plan.stats
        lens = A.row_lengths()
        assert st["max_row"] == lens.max() and st["empty_rows"] == int((lens == 0).sum())
        assert st["nnz"] == A.nnz and st["m"] == A.m
        if k == 1:
            x = synth.uniform(A.n, seed=2)
            y_ref, r = oracle.spmv(A.m, A.row_ptr, A.col_idx, A.vals, x)
            y = plan.spmv(v, torch.from_numpy(x).cuda())
            assert_close(y, y_ref, r, torch.float64, f"plan {name} {plan.config}")
        else:
            X = synth.uniform(A.n * k, seed=3).reshape(A.n, k)
            Y_ref, R = oracle.spmm(A.m, A.row_ptr, A.col_idx, A.vals, X)
            Y = plan.spmm(v, torch.from_numpy(X).cuda())
            assert_close(Y, Y_ref, R, torch.float64, f"plan {name} {plan.config}")
        # every other configuration through the same plan
        for cfg in (dict(variant=1, lanes=2), dict(variant=2, items=5)):
            plan.set_config(cfg)
            if k == 1:
                assert_close(plan.spmv(v, torch.from_numpy(x).cuda()), y_ref, r, torch.float64, f"{name} {cfg}")
            else:
                assert_close(plan.spmm(v, torch.from_numpy(X).cuda()), Y_ref, R, torch.float64, f"{name} {cfg}")


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
def test_untuned_plan_picks_the_kernel_from_row_lengths(gbs, dtype):
    """A plan without tuning chooses its kernel from the row-length statistics: row-wise with
    lanes from the mean row length for the stencil and banded matrices, merge-path for the
    power-law R-MAT.  The one-shot spmv_csr (no statistics, no synchronisation) is merge-path
    everywhere; both agree with the oracle."""
    from paper_1302_1078_gb300 import _capi

    want = {"stencil3d_21": {_capi.VARIANT_ROWS}, "banded_30k": {_capi.VARIANT_ROWS},
            "rmat_14": {_capi.VARIANT_MERGE, _capi.VARIANT_MERGE_DIRECT}}
    for name, variants in want.items():
        A = matrix(name)
        rp, ci, v = dev_csr(A, dtype)
        x = synth.uniform(A.n, seed=12)
        y_ref, r = spmv_ref(A, x, dtype)
        xd = torch.from_numpy(x.astype(NP[dtype])).cuda()
        plan = gbs.Plan(rp, ci, A.n, dtype, 1)
        cfg = plan.config
        assert cfg["variant"] in variants, (name, cfg)
        mean = A.nnz / A.m
        if cfg["variant"] == _capi.VARIANT_ROWS:
            per = 64 if dtype == torch.float64 else 16
            assert cfg["lanes"] == 1 or mean > per * (cfg["lanes"] // 2), (name, cfg)
        assert_close(plan.spmv(v, xd), y_ref, r, dtype, f"untuned plan {name} {cfg}")
        assert_close(gbs.spmv_csr(rp, ci, v, xd), y_ref, r, dtype, f"one-shot {name}")


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("k", [1, 3, 8, 16, 40])
@pytest.mark.parametrize("name", ["stencil2d_37", "banded_30k", "rmat_14", "random_dup_unsorted", "hub", "empty_nnz"])
def test_rows_direct_is_bitwise_rows(gbs, name, k, dtype):
    """ROWS_DIRECT reads each row straight from global memory instead of a staged tile, with the
    same per-lane order of products as ROWS whose lanes split the columns (k > 1) or with one lane
    per row (k == 1): the two give the same bits, for aligned and narrow X, in every column panel."""
    A = matrix(name)
    rp, ci, v = dev_csr(A, dtype)
    for ld in (k, k + 1):
        Xw = synth.uniform(A.n * ld, seed=41, stream=ld).reshape(A.n, ld).astype(NP[dtype])
        X = torch.from_numpy(Xw).cuda()[:, :k]
        if k == 1:
            xd = torch.from_numpy(np.ascontiguousarray(Xw[:, 0])).cuda()
            y0 = gbs.spmv_csr(rp, ci, v, xd, config=dict(variant=1, lanes=1, tile_nnz=512))
            for th in (64, 256):
                y1 = gbs.spmv_csr(rp, ci, v, xd, config=dict(variant=5, threads=th))
                assert torch.equal(y0, y1), (name, th)
        else:
            Y0 = gbs.spmm_csr(rp, ci, v, X, config=dict(variant=1, tile_nnz=512))
            for th in (64, 256):
                Y1 = gbs.spmm_csr(rp, ci, v, X, config=dict(variant=5, threads=th))
                assert torch.equal(Y0, Y1), (name, k, ld, th)


def test_stats_and_validation(gbs):
    from paper_1302_1078_gb300 import _capi

    A = matrix("random_rect")
    rp, ci, v = dev_csr(A)
    st = gbs.csr_stats(rp, A.n)
    lens = A.row_lengths()
    assert st["max_row"] == lens.max() and st["empty_rows"] == int((lens == 0).sum())
    assert st["rows_over_32"] == int((lens > 32).sum())
    assert abs(st["mean_row"] - lens.mean()) < 1e-12
    assert abs(st["cv_row"] - lens.std() / lens.mean()) < 1e-9
    gbs.validate_csr(rp, ci, A.n)
    bad = ci.clone()
    bad[3] = A.n  # one column id out of range (only validated, never multiplied)
    with pytest.raises(gbs.GbsError) as e:
        gbs.validate_csr(rp, bad, A.n)
    assert e.value.status == _capi.GBS_EINDEX
    rp_bad = rp.clone()
    rp_bad[0] = 1
    with pytest.raises(gbs.GbsError):
        gbs.validate_csr(rp_bad, ci, A.n)


def test_zero_rows_and_zero_columns(gbs):
    rp = torch.zeros(1, dtype=torch.int32, device="cuda")
    ci = torch.zeros(0, dtype=torch.int32, device="cuda")
    v = torch.zeros(0, dtype=torch.float64, device="cuda")
    y = gbs.spmv_csr(rp, ci, v, torch.zeros(10, dtype=torch.float64, device="cuda"))
    assert y.numel() == 0
    # n = 0: all rows empty
    rp = torch.zeros(6, dtype=torch.int32, device="cuda")
    y = gbs.spmv_csr(rp, ci, v, torch.zeros(0, dtype=torch.float64, device="cuda"))
    assert torch.equal(y, torch.zeros(5, dtype=torch.float64, device="cuda"))



def test_bounded_wait_times_out_and_context_stays_usable(gbs):
    """A device wait that nothing completes gives up at its limit and reports GBS_ETIMEOUT; the
    next products on the same context are still right (no fault, no hang)."""
    import time

    from paper_1302_1078_gb300 import _capi

    stream = torch.cuda.current_stream().cuda_stream
    assert gbs.lib().gbs_wait_probe(0, stream) == _capi.GBS_EINVAL
    t0 = time.perf_counter()
    assert gbs.lib().gbs_wait_probe(20_000_000, stream) == _capi.GBS_ETIMEOUT  # 20 ms
    dt = time.perf_counter() - t0
    assert 0.019 <= dt < 5.0, dt
    A = matrix("stencil3d_21")
    rp, ci, v = dev_csr(A)
    x = synth.uniform(A.n, seed=5)
    y_ref, r = oracle.spmv(A.m, A.row_ptr, A.col_idx, A.vals, x)
    plan = gbs.Plan(rp, ci, A.n, torch.float64, 1, config=dict(variant=_capi.VARIANT_ROWS_TMA, lanes=4, threads=128))
    y = plan.spmv(v, torch.from_numpy(x).cuda())
    assert_close(y, y_ref, r, torch.float64, "after the timed-out wait")
    st = ctypes.c_int(-1)
    gbs.lib().gbs_plan_status(plan._h, ctypes.byref(st), stream)
    assert st.value == 0


def test_checked_mode_refuses_a_bad_structure_before_the_product(gbs, monkeypatch):
    """GBSPMV_CHECKED=1 validates the CSR structure before every product and returns GBS_EINDEX
    without launching it; a plan built with check=True refuses the structure at creation."""
    from paper_1302_1078_gb300 import _capi

    A = matrix("random_rect")
    rp, ci, v = dev_csr(A)
    bad = ci.clone()
    bad[3] = A.n  # one column id out of range
    # x padded past n, so that even an unchecked product would read inside the allocation
    x = torch.zeros(A.n + 64, dtype=torch.float64, device="cuda")
    monkeypatch.setenv("GBSPMV_CHECKED", "1")
    with pytest.raises(gbs.GbsError) as e:
        gbs.spmv_csr(rp, bad, v, x, n=A.n)
    assert e.value.status == _capi.GBS_EINDEX
    y = gbs.spmv_csr(rp, ci, v, x, n=A.n)  # a valid structure passes in checked mode
    assert torch.equal(y, torch.zeros(A.m, dtype=torch.float64, device="cuda"))
    monkeypatch.delenv("GBSPMV_CHECKED")
    with pytest.raises(gbs.GbsError) as e:
        gbs.Plan(rp, bad, A.n, torch.float64, 1, check=True)
    assert e.value.status == _capi.GBS_EINDEX

# ------------------------------------------------- column relabelling (plans)

RELABEL_BASES = [dict(variant=4, items=11), dict(variant=4, items=7, threads=128), dict(variant=2, items=15),
                 dict(variant=1, lanes=2), dict(variant=3, lanes=4, threads=128)]


def _relabel_run(plan, v, X, k):
    return plan.spmv(v, X) if k == 1 else plan.spmm(v, X)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("k", [1, 3, 8])
@pytest.mark.parametrize("name", ["rmat_14", "hub", "random_rect", "random_dup_unsorted", "empty_nnz", "one_row"])
def test_relabelled_plan_is_bitwise_the_plain_plan(gbs, name, k, dtype):
    """Relabelling the columns hottest first changes neither the rows nor the order of any row's
    terms: every variant gives bitwise the result it gives without relabelling (including the
    MERGE_DIRECT walk whose cold gathers skip L1), within the bound of the oracle; the relabelling
    itself equals the oracle's bit for bit."""
    A = matrix(name)
    rp, ci, v = dev_csr(A, dtype)
    if k == 1:
        x = synth.uniform(A.n, seed=21).astype(NP[dtype])
        Y_ref, R = oracle.spmv(A.m, A.row_ptr, A.col_idx, A.vals.astype(NP[dtype]), x)
        X = torch.from_numpy(x).cuda()
    else:
        ld = k + 1  # a row stride > k: the scatter of X's rows reads narrow rows
        Xw = synth.uniform(A.n * ld, seed=22, stream=k).reshape(A.n, ld).astype(NP[dtype])
        Y_ref, R = oracle.spmm(A.m, A.row_ptr, A.col_idx, A.vals.astype(NP[dtype]), Xw[:, :k])
        X = torch.from_numpy(Xw).cuda()[:, :k]
    want_ids = oracle.degree_relabel(A.n, A.col_idx)
    for base in RELABEL_BASES:
        try:
            plan = gbs.Plan(rp, ci, A.n, dtype, k, config=base)
        except gbs.GbsError as e:
            # the pipelined variant refuses row blocks larger than its shared-memory tile (the
            # hub rows of these power-law matrices); the refusal comes before any product
            assert base["variant"] == 3 and e.status == -8, (base, e)
            continue
        y0 = _relabel_run(plan, v, X, k).clone()
        assert_close(y0, Y_ref, R, dtype, f"{name} {base}")
        for rl in (1, 8, 1024):
            plan.set_config(dict(base, relabel=rl))
            y1 = _relabel_run(plan, v, X, k)
            assert torch.equal(y0, y1), f"{name} k={k} {base} relabel={rl}: not bitwise the plain result"
            y2 = _relabel_run(plan, v, X, k)  # the relabelled copy of x is rebuilt on every call
            assert torch.equal(y1, y2)
        ids = plan.relabel_ids().cpu().numpy()
        assert np.array_equal(ids, want_ids), f"{name}: relabelling differs from the oracle's"


def test_relabel_is_plans_only(gbs):
    A = matrix("rmat_14")
    rp, ci, v = dev_csr(A)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    with pytest.raises(gbs.GbsError):
        gbs.spmv_csr(rp, ci, v, x, config=dict(variant=4, relabel=1))
    plan = gbs.Plan(rp, ci, A.n, torch.float64, 1, config=dict(variant=4))
    with pytest.raises(gbs.GbsError):
        plan.relabel_ids()  # this plan does not relabel


def test_relabelled_backward_is_bitwise_the_plain_one(gbs):
    """dX = A^T dY through a relabelled plan of A^T (its columns are A's rows) equals the plain
    plan's bit for bit."""
    A = matrix("rmat_14")
    rp, ci, v = dev_csr(A)
    t = gbs.TransposePlan(rp, ci, A.n)
    for k in (1, 8):
        X = torch.from_numpy(synth.uniform(A.n * k, seed=23).reshape(A.n, k) if k > 1 else
                             synth.uniform(A.n, seed=23)).cuda()
        dY = torch.from_numpy(synth.uniform(A.m * k, seed=24).reshape(A.m, k) if k > 1 else
                              synth.uniform(A.m, seed=24)).cuda()
        t.set_config(torch.float64, k, dict(variant=4, items=11))
        dX0, dv0 = t.backward(v, X, dY)
        for rl in (1, 8):
            t.set_config(torch.float64, k, dict(variant=4, items=11, relabel=rl))
            dX1, dv1 = t.backward(v, X, dY)
            assert torch.equal(dX0, dX1) and torch.equal(dv0, dv1), (k, rl)


# ------------------------------------------------ full-size configurations

FULL = {
    "stencil3d_100": lambda: synth.stencil3d(100),
    "banded_2M": lambda: synth.banded(2_000_000, hbw=1000, per_row=50, seed=synth.BASE_SEED + 1),
    "rmat_22": lambda: synth.rmat(22, ef=16, seed=synth.BASE_SEED + 1),
}


@pytest.mark.parametrize("name", list(FULL))
def test_full_size_spmv_tuned_plan(gbs, name):
    """The bench's matrices and launch path (tuned plan), every row checked."""
    A = FULL[name]()
    x = synth.uniform(A.n, seed=synth.BASE_SEED + 1, stream=1)
    y_ref, r = oracle.spmv(A.m, A.row_ptr, A.col_idx, A.vals, x, threads=oracle.max_threads())
    rp, ci, v = dev_csr(A)
    plan = gbs.Plan(rp, ci, A.n, torch.float64, 1, tune=True)
    y = plan.spmv(v, torch.from_numpy(x).cuda())
    assert_close(y, y_ref, r, torch.float64, f"{name} {plan.config}")
    y2 = gbs.spmv_csr(rp, ci, v, torch.from_numpy(x).cuda())
    assert_close(y2, y_ref, r, torch.float64, f"{name} auto")
    cfg = plan.config
    if cfg["relabel"]:
        # the tuner's relabelled configuration is bitwise its plain counterpart, and the
        # relabelling equals the oracle's
        ids = plan.relabel_ids().cpu().numpy()
        assert np.array_equal(ids, oracle.degree_relabel(A.n, A.col_idx))
        plan.set_config(dict(cfg, relabel=0))
        y3 = plan.spmv(v, torch.from_numpy(x).cuda())
        assert torch.equal(y, y3), f"{name} {cfg}: relabelled result differs from the plain one"



@pytest.mark.parametrize("k", [4, 8, 16])
@pytest.mark.parametrize("name", list(FULL))
def test_full_size_spmm_tuned_plan(gbs, name, k):
    """The SpMM benchmark's matrices, widths and launch path (tuned plan), every entry checked."""
    A = FULL[name]()
    X = synth.uniform(A.n * k, seed=synth.BASE_SEED + 2, stream=k).reshape(A.n, k)
    Y_ref, R = oracle.spmm(A.m, A.row_ptr, A.col_idx, A.vals, X, threads=oracle.max_threads())
    rp, ci, v = dev_csr(A)
    plan = gbs.Plan(rp, ci, A.n, torch.float64, k, tune=True)
    Y = torch.full((A.m, k), float("nan"), dtype=torch.float64, device="cuda")
    plan.spmm(v, torch.from_numpy(X).cuda(), Y)
    assert_close(Y, Y_ref, R, torch.float64, f"{name} k={k} {plan.config}")

# ------------------------------------------- pipelined ROWS (bulk-copy staging)

TMA_SHAPES = [dict(lanes=1, threads=64), dict(lanes=1, threads=128), dict(lanes=1, threads=256), dict(lanes=2, threads=64),
              dict(lanes=4, threads=192), dict(lanes=4, threads=256), dict(lanes=8, threads=128),
              dict(lanes=32, threads=256)]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("k", [1, 3, 8])
@pytest.mark.parametrize("name", ["stencil2d_64", "stencil3d_21", "banded_30k", "rmat_14", "random_rect",
                                  "random_dup_unsorted", "empty_nnz", "one_row"])
def test_rows_tma_variant(gbs, name, k, dtype):
    from paper_1302_1078_gb300 import _capi

    A = matrix(name)
    rp, ci, v = dev_csr(A, dtype)
    if k == 1:
        x = synth.uniform(A.n, seed=3, stream=k).astype(NP[dtype])
        Y_ref, R = oracle.spmv(A.m, A.row_ptr, A.col_idx, A.vals.astype(NP[dtype]), x)
        xd = torch.from_numpy(x).cuda()
    else:
        X = synth.uniform(A.n * k, seed=3, stream=k).reshape(A.n, k).astype(NP[dtype])
        Y_ref, R = oracle.spmm(A.m, A.row_ptr, A.col_idx, A.vals.astype(NP[dtype]), X)
        xd = torch.from_numpy(X).cuda()
    plan = gbs.Plan(rp, ci, A.n, dtype, k)
    for shape in TMA_SHAPES:
        cfg = dict(variant=_capi.VARIANT_ROWS_TMA, **shape)
        try:
            plan.set_config(cfg)
        except gbs.GbsError as e:
            # a row block larger than the shared-memory tile: the plan refuses the variant
            assert e.status == _capi.GBS_EUNSUPPORTED
            continue
        assert plan.config["variant"] == _capi.VARIANT_ROWS_TMA
        out = torch.full(Y_ref.shape if k > 1 else (A.m,), float("nan"), dtype=dtype, device="cuda")
        if k == 1:
            plan.spmv(v, xd, out)
        else:
            plan.spmm(v, xd, out)
        assert_close(out, Y_ref, R, dtype, f"{name} k={k} {shape}")
        # misaligned values (8 bytes off a 16-byte boundary): the plan falls back to ROWS
        buf = torch.empty(v.numel() + 4, dtype=dtype, device="cuda")
        vm = buf[1:1 + v.numel()]
        vm.copy_(v)
        out2 = torch.full_like(out, float("nan"))
        if k == 1:
            plan.spmv(vm, xd, out2)
        else:
            plan.spmm(vm, xd, out2)
        assert_close(out2, Y_ref, R, dtype, f"{name} k={k} {shape} misaligned")
    st = ctypes.c_int(-1)
    gbs.lib().gbs_plan_status(plan._h, ctypes.byref(st), torch.cuda.current_stream().cuda_stream)
    assert st.value == 0


def test_rows_tma_refuses_huge_blocks(gbs):
    from paper_1302_1078_gb300 import _capi

    A = matrix("hub")
    rp, ci, v = dev_csr(A)
    plan = gbs.Plan(rp, ci, A.n, torch.float64, 1)
    with pytest.raises(gbs.GbsError) as e:
        plan.set_config(dict(variant=_capi.VARIANT_ROWS_TMA, lanes=1, threads=256))
    assert e.value.status == _capi.GBS_EUNSUPPORTED


# ---------------------------------------- FP64 products on the FP32 pipe (emul)

@pytest.mark.parametrize("emul", [1, 2, 3])
@pytest.mark.parametrize("k", [1, 2, 8, 16])
@pytest.mark.parametrize("name", ["stencil3d_21", "banded_30k", "rmat_14", "random_rect", "one_row"])
def test_rows_tma_emulated_fp64(gbs, name, k, emul):
    from paper_1302_1078_gb300 import _capi

    A = matrix(name)
    rp, ci, v = dev_csr(A)
    X = synth.uniform(A.n * k, seed=13, stream=k).reshape(A.n, k)
    if k == 1:
        Y_ref, R = oracle.spmv(A.m, A.row_ptr, A.col_idx, A.vals, X[:, 0])
    else:
        Y_ref, R = oracle.spmm(A.m, A.row_ptr, A.col_idx, A.vals, X)
    plan = gbs.Plan(rp, ci, A.n, torch.float64, k)
    for shape in (dict(lanes=1, threads=128), dict(lanes=2, threads=256), dict(lanes=4, threads=128)):
        try:
            plan.set_config(dict(variant=_capi.VARIANT_ROWS_TMA, emul=emul, **shape))
        except gbs.GbsError as e:
            assert e.status == _capi.GBS_EUNSUPPORTED
            continue
        assert plan.config["emul"] == emul
        if k == 1:
            out = plan.spmv(v, torch.from_numpy(np.ascontiguousarray(X[:, 0])).cuda())
        else:
            out = plan.spmm(v, torch.from_numpy(X).cuda())
        assert_close(out, Y_ref, R, torch.float64, f"{name} k={k} emul={emul} {shape}")


def test_emulated_fp64_extreme_magnitudes(gbs):
    """Operands outside the FP32 exponent range (and zeros, subnormals) take the native pipe
    inside the emulated kernel; every entry still meets the FP64 bound."""
    from paper_1302_1078_gb300 import _capi

    rng = np.random.default_rng(17)
    m, n, per = 2000, 3000, 24
    rp = np.arange(0, m * per + 1, per, dtype=np.int32)
    ci = np.sort(rng.integers(0, n, (m, per)), axis=1).astype(np.int32).reshape(-1)
    # 2^38 and 2^-38 sit at the edges of the FP32-pipe range (products up to 2^76 and down to
    # 2^-76 on the FP32 pipe); 1e30, 2^39 and 2^-39 are just outside it
    vmags = np.array([1.0, 1e-200, 1e200, 0.0, 5e-324, 1e-31, 3e38, 1e-45, 7.5, 2.0**38, 2.0**-38, 1e30, 2.0**39,
                      2.0**-39], np.float64)
    xmags = np.array([1.0, 1e-200, 1e100, 0.0, 5e-324, 1e-31, 3e38, 1e-45, 7.5, 2.0**38, 2.0**-38, 1e30, 2.0**39,
                      2.0**-39], np.float64)  # products stay finite
    v = rng.uniform(-1, 1, m * per) * vmags[rng.integers(0, vmags.size, m * per)]
    x = rng.uniform(-1, 1, n) * xmags[rng.integers(0, xmags.size, n)]
    A = synth.CSR(m, n, rp, ci, v)
    y_ref, r = oracle.spmv(m, rp, ci, v, x)
    d_rp, d_ci, d_v = dev_csr(A)
    plan = gbs.Plan(d_rp, d_ci, n, torch.float64, 1)
    for emul in (0, 1, 2, 3):
        for lanes, threads in ((1, 128), (4, 128), (8, 256)):
            plan.set_config(dict(variant=_capi.VARIANT_ROWS_TMA, lanes=lanes, threads=threads, emul=emul))
            y = plan.spmv(d_v, torch.from_numpy(x).cuda())
            assert_close(y, y_ref, r, torch.float64, f"extreme magnitudes emul={emul} lanes={lanes}")


def test_tuner_with_emulation(gbs):
    A = matrix("banded_30k")
    rp, ci, v = dev_csr(A)
    x = synth.uniform(A.n, seed=23)
    y_ref, r = oracle.spmv(A.m, A.row_ptr, A.col_idx, A.vals, x)
    plan = gbs.Plan(rp, ci, A.n, torch.float64, 1, tune=True, emulate=True)
    y = plan.spmv(v, torch.from_numpy(x).cuda())
    assert_close(y, y_ref, r, torch.float64, f"tuned with emulation {plan.config}")


def test_merge_direct_misaligned_values(gbs):
    """MERGE_DIRECT with vals / col_idx off a 16-byte boundary takes its scalar path."""
    A = matrix("rmat_14")
    rp, ci, v = dev_csr(A)
    x = synth.uniform(A.n, seed=29)
    y_ref, r = oracle.spmv(A.m, A.row_ptr, A.col_idx, A.vals, x)
    vb = torch.empty(v.numel() + 2, dtype=torch.float64, device="cuda")
    cb = torch.empty(ci.numel() + 2, dtype=torch.int32, device="cuda")
    vm, cm = vb[1:1 + v.numel()], cb[1:1 + ci.numel()]
    vm.copy_(v)
    cm.copy_(ci)
    for items in (3, 31):
        y = gbs.spmv_csr(rp, cm, vm, torch.from_numpy(x).cuda(), config=dict(variant=4, items=items))
        assert_close(y, y_ref, r, torch.float64, f"misaligned direct items={items}")
    # vals 16-byte but not 32-byte aligned: two 128-bit loads per group instead of one 256-bit
    vb2 = torch.empty(v.numel() + 4, dtype=torch.float64, device="cuda")
    v16 = vb2[2:2 + v.numel()]
    v16.copy_(v)
    assert v16.data_ptr() % 32 == 16
    for items in (3, 15, 31):
        y = gbs.spmv_csr(rp, ci, v16, torch.from_numpy(x).cuda(), config=dict(variant=4, items=items))
        assert_close(y, y_ref, r, torch.float64, f"16-byte aligned direct items={items}")
        y32 = gbs.spmv_csr(rp, ci, v, torch.from_numpy(x).cuda(), config=dict(variant=4, items=items))
        assert torch.equal(y, y32), "the 128-bit and 256-bit load paths must agree bitwise"

