"""UCLD (Sec. 4.1) on the GPU against the CPU oracle: line counts bit-exact, the mean within
the fixed-point resolution of the device sum (5e-10)."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gbs():
    import paper_1302_1078_gb300 as g

    g.lib()
    return g


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rows_csr(rows, n):
    rp = np.zeros(len(rows) + 1, np.int32)
    rp[1:] = np.cumsum([len(r) for r in rows])
    ci = np.array([c for r in rows for c in r], np.int32)
    return synth.CSR(len(rows), n, rp, ci, np.ones(ci.size))


CASES = {
    "paper_example": lambda: rows_csr([[0, 19, 20]], 32),
    "extremes": lambda: rows_csr([[0, 8, 16], list(range(8)), [], [5]], 64),
    "stencil2d_64": lambda: synth.stencil2d(64),
    "stencil3d_40": lambda: synth.stencil3d(40),
    "banded_50k": lambda: synth.banded(50000, hbw=1000, per_row=50, seed=7),
    "rmat_16": lambda: synth.rmat(16, ef=16, seed=8),
    "unsorted_dups": lambda: synth.random_csr(500, 3000, 0.02, 9, sorted_cols=False, duplicates=True, empty_rows=0.3),
    "long_rows": lambda: rows_csr([list(range(0, 40000, 3)), list(range(7, 9000)), [1]], 40000),
    "long_unsorted": lambda: rows_csr([list(range(2999, -1, -7)), [3, 1, 2, 1]], 3000),
    "empty": lambda: synth.random_csr(50, 60, 0.0, 6),
}


@pytest.mark.parametrize("line", [1, 4, 8, 16])
@pytest.mark.parametrize("name", list(CASES))
def test_ucld_matches_oracle(gbs, name, line):
    A = CASES[name]()
    u_ref, lines_ref, rows_ref = oracle.ucld(A.m, A.row_ptr, A.col_idx, line)
    got = gbs.ucld(dev(A.row_ptr), dev(A.col_idx), A.n, line)
    assert got["lines"] == lines_ref and got["nonempty_rows"] == rows_ref
    assert abs(got["ucld"] - u_ref) <= 5e-10
    # deterministic
    assert gbs.ucld(dev(A.row_ptr), dev(A.col_idx), A.n, line) == got


def test_ucld_paper_value_on_gpu(gbs):
    A = CASES["paper_example"]()
    got = gbs.ucld(dev(A.row_ptr), dev(A.col_idx), A.n, 8)
    assert abs(got["ucld"] - 3 / 16) <= 5e-10 and got["lines"] == 2
