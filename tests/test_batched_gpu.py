"""Batched persistent launch (CUDA graph) against the per-matrix loop (bitwise) and the oracle."""
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


def make_batch(specs, k, dtype, seed=0):
    mats, Xs, Ys, host = [], [], [], []
    for i, sp in enumerate(specs):
        A = synth.batch_matrix(sp)
        rp = torch.from_numpy(A.row_ptr).cuda()
        ci = torch.from_numpy(A.col_idx).cuda()
        v = torch.from_numpy(A.vals.astype(NP[dtype])).cuda()
        Xh = synth.uniform(A.n * k, seed=seed + 17, stream=i).astype(NP[dtype])
        X = torch.from_numpy(Xh).cuda() if k == 1 else torch.from_numpy(Xh.reshape(A.n, k)).cuda()
        Y = torch.full((A.m,) if k == 1 else (A.m, k), float("nan"), dtype=dtype, device="cuda")
        mats.append((rp, ci, v, A.n))
        Xs.append(X)
        Ys.append(Y)
        host.append((A, Xh.reshape(A.n, k)))
    return mats, Xs, Ys, host


def check_vs_oracle(host, Ys, dtype, idx=None):
    for b in (range(len(host)) if idx is None else idx):
        A, Xh = host[b]
        Yr, R = oracle.spmm(A.m, A.row_ptr, A.col_idx, A.vals.astype(NP[dtype]), Xh)
        got = Ys[b].double().cpu().numpy().reshape(Yr.shape)
        assert np.all(np.abs(got - Yr) <= TOL[dtype] * R), f"matrix {b} ({A.name})"
        assert np.all(got[R == 0] == 0)


SMALL = synth.batch_specs(30, rows_lo=200, rows_hi=6000)


@pytest.mark.parametrize("tune", [False, True], ids=["heuristic", "tuned"])
@pytest.mark.parametrize("k,dtype", [(8, torch.float64), (1, torch.float64), (1, torch.float32), (4, torch.float32),
                                     (3, torch.float64)], ids=["k8f64", "k1f64", "k1f32", "k4f32", "k3f64"])
def test_batched_equals_looped_and_oracle(gbs, k, dtype, tune):
    mats, Xs, Ys, host = make_batch(SMALL, k, dtype)
    plan = gbs.BatchedPlan(mats, Xs, Ys, tune=tune, check=True)
    info = plan.info()
    ib = info["item_begin"]
    assert ib[0] == 0 and all(b >= a for a, b in zip(ib, ib[1:])) and ib[-1] == info["total_items"]
    variants = {c["variant"] for c in info["configs"]}
    assert variants <= {1, 2}
    plan.run()
    torch.cuda.synchronize()
    batched = [y.clone() for y in Ys]
    check_vs_oracle(host, batched, dtype)
    for y in Ys:
        y.fill_(float("nan"))
    plan.run_looped()
    torch.cuda.synchronize()
    for b in range(len(Ys)):
        assert torch.equal(Ys[b], batched[b]), f"batched != looped for matrix {b}"
    # graph replays are repeatable (merge completion counters reset themselves)
    for _ in range(3):
        plan.run()
    torch.cuda.synchronize()
    for b in range(len(Ys)):
        assert torch.equal(Ys[b], batched[b]), f"replay differs for matrix {b}"


def test_batched_forced_merge_and_new_operands(gbs):
    """The R-MAT members take the merge path (completion counters, in-kernel fix-up); then new X/Y."""
    import paper_1302_1078_gb300 as g

    mats, Xs, Ys, host = make_batch(SMALL[:12], 8, torch.float64, seed=5)
    plan = g.BatchedPlan(mats, Xs, Ys)
    plan.run()
    torch.cuda.synchronize()
    check_vs_oracle(host, Ys, torch.float64)
    # new operands
    X2 = [torch.rand_like(x) for x in Xs]
    Y2 = [torch.full_like(y, float("nan")) for y in Ys]
    plan.run(X2, Y2)
    torch.cuda.synchronize()
    host2 = [(A, X2[b].cpu().numpy()) for b, (A, _) in enumerate(host)]
    check_vs_oracle(host2, Y2, torch.float64)


@pytest.mark.parametrize("k,dtype", [(8, torch.float64), (1, torch.float64), (1, torch.float32)],
                         ids=["k8f64", "k1f64", "k1f32"])
def test_batched_explicit_configs(gbs, k, dtype):
    """Caller-given per-matrix configurations (ROWS / MERGE / library's choice): equal to the
    per-matrix loop bitwise and to the oracle; other variants are refused."""
    mats, Xs, Ys, host = make_batch(SMALL[:18], k, dtype, seed=9)
    cycle = [dict(variant=2, items=5), dict(variant=1, lanes=2, tile_nnz=96), None,
             dict(variant=2, items=63), dict(variant=1, lanes=1, tile_nnz=4096), dict(variant=0)]
    cfgs = [cycle[b % len(cycle)] for b in range(len(mats))]
    plan = gbs.BatchedPlan(mats, Xs, Ys, configs=cfgs)
    info = plan.info()
    for b, c in enumerate(cfgs):
        if c is not None and c["variant"] != 0:
            assert info["configs"][b]["variant"] == c["variant"]
            if c["variant"] == 1:
                assert info["configs"][b]["tile_nnz"] == c["tile_nnz"]
    plan.run()
    torch.cuda.synchronize()
    batched = [y.clone() for y in Ys]
    check_vs_oracle(host, batched, dtype)
    plan.run_looped()
    torch.cuda.synchronize()
    for b in range(len(Ys)):
        assert torch.equal(Ys[b], batched[b]), f"batched != looped for matrix {b}"
    for v in (3, 4, 5):  # ROWS_TMA, MERGE_DIRECT and ROWS_DIRECT are not batch item forms
        with pytest.raises(gbs._capi.GbsError):
            gbs.BatchedPlan(mats[:2], Xs[:2], Ys[:2], configs=[dict(variant=v), None])
    with pytest.raises(gbs._capi.GbsError):  # tile below 32 nonzeros
        gbs.BatchedPlan(mats[:2], Xs[:2], Ys[:2], configs=[dict(variant=1, tile_nnz=16), None])
    if k == 1:  # lanes per row must be a power of two (k > 1 uses the batch's column lanes)
        with pytest.raises(gbs._capi.GbsError):
            gbs.BatchedPlan(mats[:2], Xs[:2], Ys[:2], configs=[dict(variant=1, lanes=3), None])


def test_batch_offsets_match_oracle(gbs):
    mats, Xs, Ys, host = make_batch(SMALL[:20], 8, torch.float64)
    plan = gbs.BatchedPlan(mats, Xs, Ys)
    got = plan.offsets()
    ms = np.array([A.m for A, _ in host], np.int32)
    ns = np.array([A.n for A, _ in host], np.int32)
    nz = np.array([A.nnz for A, _ in host], np.int64)
    ref = oracle.batch_offsets(ms, ns, nz, 8)
    for g_, r_ in zip(got, ref):
        assert np.array_equal(g_, r_)


def test_full_batch_512_k8(gbs):
    """The batched configuration at full size: 512 matrices, rows log-uniform in 1k-200k,
    k = 8, FP64, tuned; batched equals looped bitwise, a sample of matrices checked against
    the oracle."""
    specs = synth.batch_specs(512)
    mats, Xs, Ys, host = make_batch(specs, 8, torch.float64, seed=3)
    plan = gbs.BatchedPlan(mats, Xs, Ys, tune=True)
    plan.run()
    torch.cuda.synchronize()
    batched = [y.clone() for y in Ys]
    plan.run_looped()
    torch.cuda.synchronize()
    for b in range(len(Ys)):
        assert torch.equal(Ys[b], batched[b]), f"batched != looped for matrix {b}"
    rng = np.random.default_rng(0)
    sample = sorted(set(rng.choice(len(specs), 24, replace=False).tolist()) | {0, 1, 2, 511})
    check_vs_oracle(host, batched, torch.float64, sample)


def _hub_matrix():
    """Empty rows around one 100k-nonzero row, a 7000-nonzero row and a few short ones."""
    m, n = 64, 200000
    lens = np.zeros(m, np.int64)
    lens[5] = 100000
    lens[6:12] = 3
    lens[40] = 7000
    rp = np.zeros(m + 1, np.int64)
    np.cumsum(lens, out=rp[1:])
    rng = np.random.default_rng(5)
    ci = np.concatenate([np.sort(rng.choice(n, int(l), replace=False)) for l in lens if l > 0]).astype(np.int32)
    return synth.CSR(m, n, rp.astype(np.int32), ci, rng.uniform(-1, 1, ci.size), "hub")


@pytest.mark.parametrize("k,dtype", [(1, torch.float64), (4, torch.float64), (1, torch.float32)],
                         ids=["k1f64", "k4f64", "k1f32"])
def test_batched_hub_row_equals_looped(gbs, k, dtype):
    """A row spanning about 56 merge tiles (256 threads x 7 items).  In the per-matrix loop the
    standalone fix-up hands such a run of carries to a warp (loaded 32 at a time, added in tile
    order); in the batched kernel the CTA that retires the matrix adds them one by one.  The two
    must give the same bits, and both the oracle's result within the bound."""
    mats, Xs, Ys, host = [], [], [], []
    for i, A in enumerate([_hub_matrix(), synth.rmat(12, ef=8, seed=3)]):
        rp = torch.from_numpy(A.row_ptr).cuda()
        ci = torch.from_numpy(A.col_idx).cuda()
        v = torch.from_numpy(A.vals.astype(NP[dtype])).cuda()
        Xh = synth.uniform(A.n * k, seed=23, stream=i).astype(NP[dtype])
        X = torch.from_numpy(Xh).cuda() if k == 1 else torch.from_numpy(Xh.reshape(A.n, k)).cuda()
        Ys.append(torch.full((A.m,) if k == 1 else (A.m, k), float("nan"), dtype=dtype, device="cuda"))
        mats.append((rp, ci, v, A.n))
        Xs.append(X)
        host.append((A, Xh.reshape(A.n, k)))
    plan = gbs.BatchedPlan(mats, Xs, Ys, configs=[dict(variant=2, items=7), dict(variant=2, items=7)])
    assert plan.info()["configs"][0]["variant"] == 2
    plan.run()
    torch.cuda.synchronize()
    batched = [y.clone() for y in Ys]
    check_vs_oracle(host, batched, dtype)
    plan.run_looped()
    torch.cuda.synchronize()
    for b in range(len(Ys)):
        assert torch.equal(Ys[b], batched[b]), f"batched != looped for matrix {b}"
