"""Register-blocked CRS (Sec. 4.5) on the GPU: the blocks equal the oracle's element by element,
and the product from the blocks meets the FP64 / FP32 bound against the oracle's SpMV."""
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


CASES = {
    "random_ragged": lambda: synth.random_csr(203, 117, 0.05, 1, empty_rows=0.2),
    "unsorted_dups": lambda: synth.random_csr(150, 150, 0.06, 2, sorted_cols=False, duplicates=True),
    "stencil2d_37": lambda: synth.stencil2d(37),
    "blocks_dof8": lambda: synth.stencil3d_blocks(5, 8),
    "banded_20k": lambda: synth.banded(20000, hbw=1000, per_row=30, seed=4),
    "rmat_12": lambda: synth.rmat(12, ef=8, seed=5, vals="u0.5_1.5"),
    "empty": lambda: synth.random_csr(50, 60, 0.0, 6),
}
_cache = {}


def case(name):
    if name not in _cache:
        _cache[name] = CASES[name]()
    return _cache[name]


SIZES = [(a, b) for a in (1, 2, 4, 8) for b in (1, 2, 4, 8)]


@pytest.mark.parametrize("ab", SIZES, ids=[f"{a}x{b}" for a, b in SIZES])
@pytest.mark.parametrize("name", list(CASES))
def test_bcsr_blocks_and_product(gbs, name, ab):
    a, b = ab
    A = case(name)
    bptr, bcol, bval = oracle.bcsr(A.m, A.n, A.row_ptr, A.col_idx, A.vals, a, b)
    x = synth.uniform(A.n, seed=31)
    y_ref, r = oracle.spmv(A.m, A.row_ptr, A.col_idx, A.vals, x)
    for dtype in (torch.float64, torch.float32):
        v = A.vals.astype(NP[dtype])
        B = gbs.BCSR(dev(A.row_ptr), dev(A.col_idx), dev(v), A.n, a, b)
        assert B.nblocks == bcol.size
        gp, gc, gv = (t.cpu().numpy() for t in B.arrays())
        assert np.array_equal(gp, bptr) and np.array_equal(gc, bcol)
        if dtype == torch.float64:
            assert np.array_equal(gv, bval)
        else:
            _, _, bval32 = oracle.bcsr(A.m, A.n, A.row_ptr, A.col_idx, v.astype(np.float64), a, b)
            assert np.allclose(gv.astype(np.float64), bval32, rtol=1e-6, atol=0)
        xd = dev(x.astype(NP[dtype]))
        y = B.spmv(xd)
        if dtype == torch.float32:
            y_ref32, r32 = oracle.spmv(A.m, A.row_ptr, A.col_idx, v, x.astype(np.float32))
            got, want, bound = y.double().cpu().numpy(), y_ref32, r32
        else:
            got, want, bound = y.cpu().numpy(), y_ref, r
        assert np.all(np.abs(got - want) <= TOL[dtype] * bound), f"{name} {a}x{b} {dtype}"
        assert np.all(got[bound == 0] == 0)
        assert torch.equal(B.spmv(xd), y)


def test_bcsr_rejects_other_sizes(gbs):
    A = case("random_ragged")
    with pytest.raises(gbs._capi.GbsError):
        gbs.BCSR(dev(A.row_ptr), dev(A.col_idx), dev(A.vals), A.n, 3, 8)
