"""Reverse Cuthill-McKee (Sec. 4.4) and the symmetric permutation on the GPU against the CPU
oracle: the orders and the permuted matrices are equal element by element."""
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


def from_edges(n, edges):
    rows = [[] for _ in range(n)]
    for a, b in edges:
        rows[a].append(b)
    rp = np.zeros(n + 1, np.int32)
    rp[1:] = np.cumsum([len(r) for r in rows])
    ci = np.array([c for r in rows for c in sorted(r)], np.int32)
    return synth.CSR(n, n, rp, ci, np.arange(ci.size, dtype=np.float64) + 0.5)


def relabelled(A, seed):
    lab = np.random.default_rng(seed).permutation(A.m).astype(np.int32)
    rp, ci, v = oracle.permute(A.m, A.row_ptr, A.col_idx, A.vals, lab)
    return synth.CSR(A.m, A.m, rp, ci, v)


def spider():
    edges, prev = [], 0
    for arm in ([1], [2, 3, 4, 5, 6], [7, 8, 9]):
        prev = 0
        for v in arm:
            edges.append((prev, v))
            prev = v
    return from_edges(10, edges)


CASES = {
    "path": lambda: from_edges(200, [(i, i + 1) for i in range(199)]),
    "path_relabelled": lambda: relabelled(from_edges(200, [(i, i + 1) for i in range(199)]), 1),
    "grid_relabelled": lambda: relabelled(synth.stencil2d(24), 2),
    "spider": spider,
    "components": lambda: from_edges(40, [(3, 5), (5, 9), (20, 21), (21, 22), (22, 20), (30, 31), (31, 3)]),
    "random_unsorted_dups": lambda: synth.random_csr(300, 300, 0.02, 11, sorted_cols=False, duplicates=True,
                                                     empty_rows=0.3),
    "banded_50k": lambda: synth.banded(50000, hbw=1000, per_row=50, seed=12),
    "stencil3d_20": lambda: synth.stencil3d(20),
    "rmat_14": lambda: synth.rmat(14, ef=16, seed=13, vals="u0.5_1.5"),
    "rmat_12_sparse": lambda: synth.rmat(12, ef=2, seed=14),
    "one": lambda: from_edges(1, []),
    "no_edges": lambda: from_edges(57, []),
}
_cache = {}


def case(name):
    if name not in _cache:
        _cache[name] = CASES[name]()
    return _cache[name]


@pytest.mark.parametrize("name", list(CASES))
def test_rcm_matches_oracle(gbs, name):
    A = case(name)
    want = oracle.rcm(A.m, A.row_ptr, A.col_idx)
    got = gbs.rcm(dev(A.row_ptr), dev(A.col_idx)).cpu().numpy()
    assert np.array_equal(got, want)
    # deterministic
    assert np.array_equal(gbs.rcm(dev(A.row_ptr), dev(A.col_idx)).cpu().numpy(), want)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("name", ["path_relabelled", "grid_relabelled", "random_unsorted_dups", "banded_50k",
                                  "rmat_14", "components", "one"])
def test_permute_matches_oracle(gbs, name, dtype):
    A = case(name)
    for perm in (oracle.rcm(A.m, A.row_ptr, A.col_idx),
                 np.random.default_rng(5).permutation(A.m).astype(np.int32)):
        v = A.vals.astype(np.float64 if dtype == torch.float64 else np.float32)
        rp, ci, bv = oracle.permute(A.m, A.row_ptr, A.col_idx, v.astype(np.float64), perm)
        grp, gci, gbv = gbs.permute_csr(dev(A.row_ptr), dev(A.col_idx), dev(v), dev(perm))
        assert np.array_equal(grp.cpu().numpy(), rp)
        assert np.array_equal(gci.cpu().numpy(), ci)
        assert np.array_equal(gbv.cpu().numpy().astype(np.float64), bv)
        # pattern only
        prp, pci, pv = gbs.permute_csr(dev(A.row_ptr), dev(A.col_idx), None, dev(perm))
        assert pv is None and torch.equal(prp, grp) and torch.equal(pci, gci)


def test_spmv_commutes_with_the_permutation(gbs):
    """(P A P^T)(P x) = P (A x): the reordered product on the GPU equals the permuted product."""
    A = case("rmat_14")
    perm = gbs.rcm(dev(A.row_ptr), dev(A.col_idx))
    brp, bci, bv = gbs.permute_csr(dev(A.row_ptr), dev(A.col_idx), dev(A.vals), perm)
    x = synth.uniform(A.n, seed=21)
    y, r = oracle.spmv(A.m, A.row_ptr, A.col_idx, A.vals, x)
    p = perm.cpu().numpy()
    yb = gbs.spmv_csr(brp, bci, bv, dev(x[p])).cpu().numpy()
    assert np.all(np.abs(yb - y[p]) <= 1e-12 * r[p])
