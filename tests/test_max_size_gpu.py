"""Products at the largest supported size, m + nnz = 2^31 - 4097 (the 32-bit index limit less the
kernels' headroom), against the oracle on every row.

The matrix has 4096 rows of about 524k nonzeros over 2^20 columns, so nonzero positions run up
to 2^31 - 8194: every grid-stride loop, tile pass and 4-element rounding of a nonzero range is
exercised within a few thousand of 2^31.  About 26 GB of host and device memory.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

LIMIT = 2**31 - 4097  # largest m + nnz the library accepts
M, N = 4096, 1 << 20
TOL = {torch.float64: 1e-12, torch.float32: 2e-5}


@pytest.fixture(scope="module")
def gbs():
    import paper_1302_1078_gb300 as g

    g.lib()
    return g


@pytest.fixture(scope="module")
def big():
    nnz = LIMIT - M
    base, extra = divmod(nnz, M)
    lens = np.full(M, base, np.int64)
    lens[:extra] += 1
    rp = np.zeros(M + 1, np.int64)
    np.cumsum(lens, out=rp[1:])
    assert rp[-1] == nnz and rp[-1] < 2**31
    rp = rp.astype(np.int32)
    # columns: 0, 1, ..., N - 1 repeated (distinct within a row: rows are shorter than N)
    ci = np.tile(np.arange(N, dtype=np.int32), nnz // N + 1)[:nnz]
    vals = np.tile(np.array([1.0, 0.5, 0.25, 2.0, 1.5, 0.75, 1.25], np.float32), nnz // 7 + 1)[:nnz]
    x = synth.uniform(N, seed=synth.BASE_SEED + 99).astype(np.float32)
    y, r = oracle.spmv(M, rp, ci, vals, x, threads=oracle.max_threads())
    d = torch.device("cuda:0")
    out = dict(nnz=nnz, rp=rp, ci=ci, vals=vals, x=x, y=y, r=r,
               rp_d=torch.from_numpy(rp).to(d), ci_d=torch.from_numpy(ci).to(d),
               v_d=torch.from_numpy(vals).to(d), x_d=torch.from_numpy(x).to(d))
    yield out
    out.clear()
    torch.cuda.empty_cache()


def check(y_gpu, y_ref, r, dtype, what):
    y = y_gpu.double().cpu().numpy()
    bad = np.abs(y - y_ref) > TOL[dtype] * r
    assert not bad.any(), f"{what}: {int(bad.sum())} rows off, first {int(np.argmax(bad))}"


@pytest.mark.parametrize("cfg", [dict(variant=1, lanes=32, threads=256), dict(variant=1, lanes=4, threads=128),
                                 dict(variant=2, threads=256), dict(variant=4, threads=256, items=11),
                                 dict(variant=4, threads=128, items=63)],
                         ids=["rows_l32", "rows_l4", "merge", "merge_direct_11", "merge_direct_63"])
def test_max_size_f32(gbs, big, cfg):
    plan = gbs.Plan(big["rp_d"], big["ci_d"], N, torch.float32, 1, config=cfg)
    y = torch.full((M,), float("nan"), dtype=torch.float32, device="cuda")
    plan.spmv(big["v_d"], big["x_d"], y)
    check(y, big["y"], big["r"], torch.float32, str(cfg))


def test_max_size_auto_and_rows_tma_refusal(gbs, big):
    from paper_1302_1078_gb300 import _capi

    y = gbs.spmv_csr(big["rp_d"], big["ci_d"], big["v_d"], big["x_d"], n=N)
    check(y, big["y"], big["r"], torch.float32, "spmv_csr")
    plan = gbs.Plan(big["rp_d"], big["ci_d"], N, torch.float32, 1)
    with pytest.raises(gbs.GbsError) as e:  # a row block of 524k nonzeros exceeds the bulk-copy tile
        plan.set_config(dict(variant=_capi.VARIANT_ROWS_TMA, lanes=32, threads=128))
    assert e.value.status == _capi.GBS_EUNSUPPORTED


def test_max_size_f64_direct(gbs, big):
    """Double values (17 GB), merge-direct with 256-bit value loads."""
    v64 = big["vals"].astype(np.float64)
    x64 = big["x"].astype(np.float64)
    y_ref, r = oracle.spmv(M, big["rp"], big["ci"], v64, x64, threads=oracle.max_threads())
    v_d = torch.from_numpy(v64).cuda()
    del v64
    plan = gbs.Plan(big["rp_d"], big["ci_d"], N, torch.float64, 1, config=dict(variant=4, threads=256, items=11))
    y = torch.full((M,), float("nan"), dtype=torch.float64, device="cuda")
    plan.spmv(v_d, torch.from_numpy(x64).cuda(), y)
    check(y, y_ref, r, torch.float64, "f64 merge_direct")
