"""spmv_csr_noalloc: the SpMV entry point for callers that must not allocate device memory
(for example a host application that owns every device allocation, or a latency-critical
loop where an allocation could block or fail).  Its scratch is a static array inside the
library.  The test calls it through the C ABI and compares it with spmv_csr on two calls in
a row (different matrices, so the second call runs over the first call's leftover scratch),
within the parity bound the other tests use.  It needs nothing from the other test files,
so it passes alone in a fresh process as well as after them."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 2e-5}
NP = {torch.float64: np.float64, torch.float32: np.float32}


def _noalloc(lib, A, v, x, y, dtype):
    code = 0 if dtype == torch.float64 else 1
    stream = torch.cuda.current_stream().cuda_stream
    return lib.spmv_csr_noalloc(A["m"], A["n"], A["nnz"], A["rp"].data_ptr(), A["ci"].data_ptr(), v.data_ptr(), code,
                                x.data_ptr(), y.data_ptr(), stream)


def _dev(M: synth.CSR):
    return dict(m=M.m, n=M.n, nnz=M.nnz, rp=torch.from_numpy(M.row_ptr).cuda(), ci=torch.from_numpy(M.col_idx).cuda())


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
def test_noalloc_matches_spmv_csr_on_two_calls(dtype):
    import paper_1302_1078_gb300 as gbs

    lib = gbs.lib()
    # the larger matrix first, then a smaller one: the second call reuses scratch the first left behind
    mats = [synth.rmat(15, ef=16, seed=7), synth.banded(20011, hbw=500, per_row=21, seed=8)]
    for i, M in enumerate(mats):
        A = _dev(M)
        v = torch.from_numpy(M.vals.astype(NP[dtype])).cuda()
        xh = synth.uniform(M.n, seed=9, stream=i).astype(NP[dtype])
        x = torch.from_numpy(xh).cuda()
        y = torch.full((M.m,), float("nan"), dtype=dtype, device="cuda")
        rc = _noalloc(lib, A, v, x, y, dtype)
        assert rc == 0, lib.gbs_last_error()
        y_ref = gbs.spmv_csr(A["rp"], A["ci"], v, x)
        torch.cuda.synchronize()
        _, r = oracle.spmv(M.m, M.row_ptr, M.col_idx, M.vals.astype(NP[dtype]), xh)
        got, ref = y.double().cpu().numpy(), y_ref.double().cpu().numpy()
        assert np.all(np.abs(got - ref) <= TOL[dtype] * r), f"call {i}: differs from spmv_csr"
        assert np.all(got[r == 0] == 0.0)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import paper_1302_1078_gb300 as gbs

    lib = gbs.lib()
    # m + nnz = 1.2e9 needs more scratch than the static array holds: rejected before any launch,
    # so the (never dereferenced) pointers may be anything non-NULL
    rc = lib.spmv_csr_noalloc(600_000_000, 600_000_000, 600_000_000, 16, 16, 16, 0, 16, 16, None)
    assert rc == -8  # GBS_EUNSUPPORTED
    assert b"static scratch" in lib.gbs_last_error()
