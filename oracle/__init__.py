"""CPU oracle for CSR SpMV / SpMM / transpose / backward (TEST INFRASTRUCTURE).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library never imports it, and
it shares no code with the GPU library.

The arithmetic lives in ``oracle.c`` (plain C, double precision, sequential
sums in stored order).  This module compiles that file with gcc on first use
and marshals numpy arrays into it.  Every function returns float64 results
together with the matching sums of absolute products, which scale the accuracy
bound a parallel result is held to.

Parity status of each entry point (the pins are in ``tests/test_oracle.py``):

* ``spmv``, ``spmm``: pinned by closed forms (stencil Laplacians applied to
  constant and linear fields), identity and permutation matrices, and dense
  brute force on tiny matrices.
* ``transpose``: pinned by the dual CCS of scipy.sparse, the involution
  (A^T)^T = A and brute-force stability checks.
* ``backward``: pinned by central finite differences of the bilinear loss
  <A X, W> and by dense brute force.
* ``batch_offsets``: pinned by brute-force running sums.
* ``rcm``, ``permute``: pinned by closed forms (a relabelled path has bandwidth 1, a
  relabelled N x N grid bandwidth N), components and isolated nodes, the breadth-first
  structure the ordering must have, and scipy's RCM as an independent bandwidth bound.
* ``bcsr``, ``bcsr_spmv``: pinned by dense brute force (the blocks expand back to A),
  closed-form block counts (identity, dense, block-diagonal) and the fill of a dense block.
* ``ucld``: pinned by the paper's worked example (Sec. 4.1, row 0 19 20 -> 3/16),
  its two extremes (1/line and 1) and brute force on tiny matrices.
* ``degree_relabel``: pinned by closed forms (full lower and upper triangles give the
  identity and the reversal, a permutation matrix ties everywhere and gives the
  identity), numpy's lexsort on random matrices with repeated entries, and the
  invariant that the relabelled product equals the original one bitwise.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` (gcc, no fused multiply-add, OpenMP if available)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        try:
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P, i32, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong
            lib.orc_spmv_f64.argtypes = [i32, P, P, P, P, P, P, i32]
            lib.orc_spmv_f32.argtypes = [i32, P, P, P, P, P, P, i32]
            lib.orc_spmm_f64.argtypes = [i32, i32, P, P, P, P, ll, P, ll, P, i32]
            lib.orc_spmm_f32.argtypes = [i32, i32, P, P, P, P, ll, P, ll, P, i32]
            lib.orc_transpose.argtypes = [i32, i32, P, P, P, P, P]
            lib.orc_transpose.restype = i32
            lib.orc_backward_f64.argtypes = [i32, i32, i32, P, P, P, P, ll, P, ll, P, ll, P, P, P]
            lib.orc_backward_f32.argtypes = [i32, i32, i32, P, P, P, P, ll, P, ll, P, ll, P, P, P]
            lib.orc_batch_offsets.argtypes = [i32, P, P, P, i32, P, P, P, P, P]
            lib.orc_ucld.argtypes = [i32, P, P, i32, P, P, P]
            lib.orc_rcm.argtypes = [i32, P, P, P]
            lib.orc_rcm.restype = i32
            lib.orc_permute.argtypes = [i32, P, P, P, P, P, P, P]
            lib.orc_permute.restype = i32
            lib.orc_bcsr.argtypes = [i32, i32, P, P, P, i32, i32, P, P, P]
            lib.orc_bcsr.restype = ll
            lib.orc_bcsr_spmv.argtypes = [i32, i32, i32, i32, P, P, P, P, P, P]
            lib.orc_degree_relabel.argtypes = [i32, i32, P, P]
            lib.orc_degree_relabel.restype = i32
            lib.orc_max_threads.restype = i32
            _lib = lib
    return _lib


def _c(a: np.ndarray, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a: np.ndarray) -> int:
    return a.ctypes.data if a.size else 0


def _float_kind(vals: np.ndarray) -> str:
    if vals.dtype == np.float64:
        return "f64"
    if vals.dtype == np.float32:
        return "f32"
    raise TypeError(f"values must be float64 or float32, got {vals.dtype}")


def max_threads() -> int:
    return int(_load().orc_max_threads())


def spmv(m, row_ptr, col_idx, vals, x, threads: int = 1):
    """Return (y, r): y_i = sum_p val[p] x[col[p]] and r_i = sum_p |val[p] x[col[p]]|."""
    lib = _load()
    kind = _float_kind(vals)
    dt = np.float64 if kind == "f64" else np.float32
    rp, ci = _c(row_ptr, np.int32), _c(col_idx, np.int32)
    v, xv = _c(vals, dt), _c(x, dt)
    y = np.empty(m, np.float64)
    r = np.empty(m, np.float64)
    fn = lib.orc_spmv_f64 if kind == "f64" else lib.orc_spmv_f32
    fn(int(m), _p(rp), _p(ci), _p(v), _p(xv), _p(y), _p(r), int(threads))
    return y, r


def spmm(m, row_ptr, col_idx, vals, X, threads: int = 1):
    """Return (Y, R) for Y = A X with X an n x k row-major array; Y and R are m x k float64."""
    lib = _load()
    kind = _float_kind(vals)
    dt = np.float64 if kind == "f64" else np.float32
    X = np.asarray(X)
    if X.ndim != 2:
        raise ValueError("X must be 2-D")
    k = X.shape[1]
    ldx = X.strides[0] // X.itemsize
    if X.dtype != dt or X.strides[1] != X.itemsize:
        X = _c(X, dt)
        ldx = k
    rp, ci, v = _c(row_ptr, np.int32), _c(col_idx, np.int32), _c(vals, dt)
    Y = np.empty((m, k), np.float64)
    R = np.empty((m, k), np.float64)
    fn = lib.orc_spmm_f64 if kind == "f64" else lib.orc_spmm_f32
    fn(int(m), int(k), _p(rp), _p(ci), _p(v), X.ctypes.data if X.size else 0, int(max(ldx, 1)),
       _p(Y), int(max(k, 1)), _p(R), int(threads))
    return Y, R


def transpose(m, n, row_ptr, col_idx):
    """Return (row_ptr_T[n+1], col_idx_T[nnz], perm[nnz]) of A^T by a stable counting sort."""
    lib = _load()
    rp, ci = _c(row_ptr, np.int32), _c(col_idx, np.int32)
    nnz = int(rp[m])
    rpT = np.empty(n + 1, np.int32)
    ciT = np.empty(nnz, np.int32)
    perm = np.empty(nnz, np.int32)
    rc = lib.orc_transpose(int(m), int(n), _p(rp), _p(ci), _p(rpT), _p(ciT), _p(perm))
    if rc != 0:
        raise ValueError("column index out of range")
    return rpT, ciT, perm


def backward(m, n, row_ptr, col_idx, vals, X, dY):
    """Gradients of <A X, W> with dY = W: returns (dX n x k, dvals nnz, RdX, Rdvals), float64."""
    lib = _load()
    kind = _float_kind(vals)
    dt = np.float64 if kind == "f64" else np.float32
    X = _c(X, dt)
    dY = _c(dY, dt)
    k = X.shape[1]
    rp, ci, v = _c(row_ptr, np.int32), _c(col_idx, np.int32), _c(vals, dt)
    nnz = int(rp[m])
    dX = np.empty((n, k), np.float64)
    RdX = np.empty((n, k), np.float64)
    dvals = np.empty(nnz, np.float64)
    Rdv = np.empty(nnz, np.float64)
    fn = lib.orc_backward_f64 if kind == "f64" else lib.orc_backward_f32
    fn(int(m), int(n), int(k), _p(rp), _p(ci), _p(v), _p(X), int(max(k, 1)), _p(dY), int(max(k, 1)),
       _p(dX), int(max(k, 1)), _p(dvals), _p(RdX), _p(Rdv))
    return dX, dvals, RdX, Rdv


def batch_offsets(ms, ns, nnzs, k):
    """Exclusive prefix sums (nmat+1 entries each) of rows, nonzeros, row_ptr entries,
    X entries (n*k) and Y entries (m*k), in input order."""
    lib = _load()
    ms, ns = _c(ms, np.int32), _c(ns, np.int32)
    nz = _c(nnzs, np.int64)
    b = ms.shape[0]
    outs = [np.empty(b + 1, np.int64) for _ in range(5)]
    lib.orc_batch_offsets(int(b), _p(ms), _p(ns), _p(nz), int(k), *[o.ctypes.data for o in outs])
    return tuple(outs)


def ucld(m, row_ptr, col_idx, line: int = 8):
    """(UCLD, sum over rows of distinct x lines, non-empty rows) for aligned lines of
    ``line`` elements (Sec. 4.1): the mean over non-empty rows of nnz_i / (line * lines_i)."""
    lib = _load()
    rp, ci = _c(row_ptr, np.int32), _c(col_idx, np.int32)
    u = ctypes.c_double()
    tot, rows = ctypes.c_longlong(), ctypes.c_longlong()
    lib.orc_ucld(int(m), _p(rp), _p(ci), int(line), ctypes.byref(u), ctypes.byref(tot), ctypes.byref(rows))
    return u.value, tot.value, rows.value


def rcm(n, row_ptr, col_idx):
    """Reverse Cuthill-McKee permutation (perm[i] = node placed at i) of the symmetric
    pattern of A + A^T for a square A (Sec. 4.4; tie-breaking rules in oracle.c)."""
    lib = _load()
    rp, ci = _c(row_ptr, np.int32), _c(col_idx, np.int32)
    perm = np.empty(max(int(n), 0), np.int32)
    if lib.orc_rcm(int(n), _p(rp), _p(ci), _p(perm)) != 0:
        raise MemoryError("orc_rcm")
    return perm


def permute(n, row_ptr, col_idx, vals, perm):
    """B = P A P^T: (row_ptr, col_idx, vals) of B, columns sorted within rows."""
    lib = _load()
    rp, ci, p = _c(row_ptr, np.int32), _c(col_idx, np.int32), _c(perm, np.int32)
    v = None if vals is None else _c(vals, np.float64)
    brp = np.empty(int(n) + 1, np.int32)
    bci = np.empty(ci.size, np.int32)
    bv = None if v is None else np.empty(ci.size, np.float64)
    rc = lib.orc_permute(int(n), _p(rp), _p(ci), None if v is None else _p(v), _p(p), _p(brp), _p(bci),
                         None if bv is None else _p(bv))
    if rc != 0:
        raise MemoryError("orc_permute")
    return brp, bci, bv


def bcsr(m, n, row_ptr, col_idx, vals, a: int, b: int):
    """Register-blocked CRS (Sec. 4.5) with aligned a x b dense blocks: (bptr, bcol, bval)."""
    lib = _load()
    rp, ci, v = _c(row_ptr, np.int32), _c(col_idx, np.int32), _c(vals, np.float64)
    mb = (int(m) + a - 1) // a
    nb = lib.orc_bcsr(int(m), int(n), _p(rp), _p(ci), _p(v), int(a), int(b), None, None, None)
    if nb < 0:
        raise MemoryError("orc_bcsr")
    bptr = np.empty(mb + 1, np.int32)
    bcol = np.empty(nb, np.int32)
    bval = np.empty(nb * a * b, np.float64)
    lib.orc_bcsr(int(m), int(n), _p(rp), _p(ci), _p(v), int(a), int(b), _p(bptr), _p(bcol), _p(bval))
    return bptr, bcol, bval


def bcsr_spmv(m, n, a, b, bptr, bcol, bval, x):
    """y <- A x from the blocks, with the sums of |products|."""
    lib = _load()
    bptr, bcol, bval, x = _c(bptr, np.int32), _c(bcol, np.int32), _c(bval, np.float64), _c(x, np.float64)
    y, r = np.empty(int(m)), np.empty(int(m))
    lib.orc_bcsr_spmv(int(m), int(n), int(a), int(b), _p(bptr), _p(bcol), _p(bval), _p(x), _p(y), _p(r))
    return y, r


def degree_relabel(n, col_idx):
    """newid[j] = rank of column j when the columns are ordered by stored entries, most first,
    ties by ascending column id (the relabelling of oracle.c's orc_degree_relabel)."""
    lib = _load()
    ci = _c(col_idx, np.int32)
    newid = np.empty(max(int(n), 0), np.int32)
    rc = lib.orc_degree_relabel(int(n), int(ci.size), _p(ci), _p(newid))
    if rc == -1:
        raise ValueError("column index out of range")
    if rc != 0:
        raise MemoryError("orc_degree_relabel")
    return newid
