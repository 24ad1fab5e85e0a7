"""Seeded synthetic CSR inputs shared by the oracle tests, the GPU tests and the bench.

This package builds inputs only.  It contains none of the multiplication
arithmetic, and neither the oracle nor the GPU library imports it.  The
generators are written in C (``synth.c``) and compiled on first use with gcc.

The matrices stand in for the paper's UFL test set (Sec. 4, Table
"tab:matrices"), which is not available here:

* ``stencil2d(N)``: 2D 5-point Laplacian.  ``stencil2d(2048)`` is the paper's
  ``mesh_2048`` (4,194,304 rows, 20,963,328 nonzeros, at most 5 per row).
* ``stencil3d(N)``: 3D 27-point stencil, the regular mesh class.
* ``banded(m, hbw, per_row)``: FEM-like rows with 20-60 nonzeros.
* ``rmat(scale, ef)``: power-law rows, like webbase-1M and scircuit.
* ``batch_specs(count)``: the recipe for a batch of uneven matrices.

Every generator is a pure function of its arguments and seed.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None

# Seed of configuration i is BASE_SEED + i.
BASE_SEED = 20130205


def build(force: bool = False) -> str:
    """Compile ``libsynth.so`` next to its source (gcc, portable flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            ll, i32, u64, f64 = ctypes.c_longlong, ctypes.c_int, ctypes.c_uint64, ctypes.c_double
            lib.syn_uniform_f64.argtypes = [ll, f64, f64, u64, u64, P]
            lib.syn_normal_f64.argtypes = [ll, u64, u64, P]
            lib.syn_stencil2d.argtypes = [i32, P, P, P]
            lib.syn_stencil2d.restype = ll
            lib.syn_stencil3d.argtypes = [i32, P, P, P]
            lib.syn_stencil3d.restype = ll
            lib.syn_banded_rowptr.argtypes = [i32, i32, i32, P]
            lib.syn_banded_rowptr.restype = ll
            lib.syn_banded_fill.argtypes = [i32, i32, u64, P, P, P]
            lib.syn_rmat.argtypes = [i32, i32, f64, f64, f64, u64, P, P]
            lib.syn_rmat.restype = ll
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


@dataclass
class CSR:
    """A CSR matrix on the host: m x n, row_ptr[m+1], col_idx[nnz] (int32), vals[nnz]."""

    m: int
    n: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    vals: np.ndarray
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])

    def astype(self, dtype) -> "CSR":
        return CSR(self.m, self.n, self.row_ptr, self.col_idx, self.vals.astype(dtype), self.name)

    def row_lengths(self) -> np.ndarray:
        return np.diff(self.row_ptr.astype(np.int64))

    def to_dense(self) -> np.ndarray:
        """Dense copy for tiny matrices (duplicates add up)."""
        d = np.zeros((self.m, self.n), dtype=np.float64)
        rows = np.repeat(np.arange(self.m), self.row_lengths())
        np.add.at(d, (rows, self.col_idx.astype(np.int64)), self.vals.astype(np.float64))
        return d


def uniform(count: int, lo: float = -1.0, hi: float = 1.0, seed: int = BASE_SEED, stream: int = 0) -> np.ndarray:
    """``count`` doubles uniform in [lo, hi) from stream ``stream`` of ``seed``."""
    out = np.empty(int(count), dtype=np.float64)
    if count:
        _load().syn_uniform_f64(int(count), float(lo), float(hi), int(seed) & (2**64 - 1), int(stream), _ptr(out))
    return out


def normal(count: int, seed: int = BASE_SEED, stream: int = 0) -> np.ndarray:
    out = np.empty(int(count), dtype=np.float64)
    if count:
        _load().syn_normal_f64(int(count), int(seed) & (2**64 - 1), int(stream), _ptr(out))
    return out


def stencil2d(N: int) -> CSR:
    """2D 5-point Laplacian on an N x N grid: diag 4, off -1, nnz = 5N^2 - 4N."""
    m = N * N
    nnz = 5 * N * N - 4 * N
    rp = np.empty(m + 1, np.int32)
    ci = np.empty(nnz, np.int32)
    v = np.empty(nnz, np.float64)
    got = _load().syn_stencil2d(N, _ptr(rp), _ptr(ci), _ptr(v))
    assert got == nnz
    return CSR(m, m, rp, ci, v, f"stencil2d_{N}")


def stencil3d(N: int) -> CSR:
    """3D 27-point stencil on N^3: diag 26, off -1, nnz = (3N-2)^3."""
    m = N ** 3
    nnz = (3 * N - 2) ** 3
    rp = np.empty(m + 1, np.int32)
    ci = np.empty(nnz, np.int32)
    v = np.empty(nnz, np.float64)
    got = _load().syn_stencil3d(N, _ptr(rp), _ptr(ci), _ptr(v))
    assert got == nnz
    return CSR(m, m, rp, ci, v, f"stencil3d_{N}")


def stencil3d_blocks(N: int, dof: int = 8, seed: int = BASE_SEED + 5) -> CSR:
    """Block-structured FEM-like matrix: the 27-point stencil on N^3 nodes with ``dof`` unknowns
    per node, every node-node coupling a dense dof x dof block (rows and columns of node u are
    u*dof .. u*dof+dof-1).  Off-diagonal values N(0,1), diagonal = sum of |row| + 1.
    nnz = dof^2 (3N-2)^3.  The register-blocking study's blocky case (aligned blocks fill)."""
    nodes = stencil3d(N)
    m = nodes.m * dof
    deg = np.diff(nodes.row_ptr).astype(np.int64)
    seg = (nodes.col_idx.astype(np.int64)[:, None] * dof + np.arange(dof)).reshape(-1)  # per node, contiguous
    row_len = np.repeat(deg * dof, dof)
    rp = np.zeros(m + 1, np.int64)
    rp[1:] = np.cumsum(row_len)
    # row r = u*dof + d takes node u's column segment
    u_of_row = np.repeat(np.arange(nodes.m), dof)
    starts = nodes.row_ptr[:-1].astype(np.int64)[u_of_row] * dof
    lens = row_len
    idx = np.repeat(starts - rp[:-1], lens) + np.arange(rp[-1])
    ci = seg[idx].astype(np.int32)
    v = normal(int(rp[-1]), seed=seed)
    rows = np.repeat(np.arange(m), lens)
    diag = ci == rows
    absum = np.add.reduceat(np.abs(np.where(diag, 0.0, v)), rp[:-1].astype(np.int64)) if m else np.zeros(0)
    v[diag] = absum + 1.0
    return CSR(m, m, rp.astype(np.int32), ci, v, f"stencil3d_{N}_dof{dof}")


def banded(m: int, hbw: int = 1000, per_row: int = 50, seed: int = BASE_SEED + 1) -> CSR:
    """Random banded FEM-like matrix: |i-j| <= hbw, ``per_row`` distinct columns per row
    (diagonal included), N(0,1) off-diagonals, diagonal = sum |off| + 1."""
    lib = _load()
    rp = np.empty(m + 1, np.int32)
    nnz = lib.syn_banded_rowptr(m, hbw, per_row, _ptr(rp))
    ci = np.empty(nnz, np.int32)
    v = np.empty(nnz, np.float64)
    lib.syn_banded_fill(m, hbw, int(seed), _ptr(rp), _ptr(ci), _ptr(v))
    return CSR(m, m, rp, ci, v, f"banded_{m}_hbw{hbw}_r{per_row}")


RMAT_ABC = (0.57, 0.19, 0.19)


def rmat(scale: int, ef: int = 16, seed: int = BASE_SEED + 1, vals: str = "one",
         abc=RMAT_ABC, val_seed_stream: int = 1) -> CSR:
    """R-MAT graph with 2^scale vertices and ef * 2^scale generated directed edges,
    duplicates removed, self loops kept, not symmetrised.

    ``vals``: ``"one"`` (all 1.0) or ``"u0.5_1.5"`` (uniform in [0.5, 1.5))."""
    m = 1 << scale
    rp = np.empty(m + 1, np.int32)
    ci = np.empty(ef * m, np.int32)
    a, b, c = abc
    nnz = _load().syn_rmat(scale, ef, a, b, c, int(seed), _ptr(rp), _ptr(ci))
    ci = ci[:nnz].copy()
    if vals == "one":
        v = np.ones(nnz, np.float64)
    elif vals == "u0.5_1.5":
        v = uniform(nnz, 0.5, 1.5, seed=seed, stream=val_seed_stream)
    else:
        raise ValueError(vals)
    return CSR(m, m, rp, ci, v, f"rmat_s{scale}_ef{ef}")


def random_csr(m: int, n: int, density: float, seed: int, empty_rows: float = 0.0,
               sorted_cols: bool = True, duplicates: bool = False) -> CSR:
    """Small random CSR for brute-force tests: Bernoulli(density) pattern, some rows
    forced empty, optional unsorted or duplicated columns; values uniform[-1,1)."""
    rng = np.random.default_rng(seed)
    mask = rng.random((m, n)) < density
    if empty_rows > 0:
        mask[rng.random(m) < empty_rows, :] = False
    rows, cols = np.nonzero(mask)
    if duplicates and rows.size:
        pick = rng.random(rows.size) < 0.3
        rows = np.concatenate([rows, rows[pick]])
        cols = np.concatenate([cols, cols[pick]])
        order = np.argsort(rows, kind="stable")
        rows, cols = rows[order], cols[order]
    if not sorted_cols and rows.size:
        key = rows * (n + 1) + rng.permutation(rows.size) % (n + 1)
        order = np.argsort(key, kind="stable")
        rows, cols = rows[order], cols[order]
    counts = np.bincount(rows, minlength=m) if rows.size else np.zeros(m, np.int64)
    rp = np.zeros(m + 1, np.int64)
    np.cumsum(counts, out=rp[1:])
    v = rng.uniform(-1.0, 1.0, rows.size)
    return CSR(m, n, rp.astype(np.int32), cols.astype(np.int32), v, f"random_{m}x{n}")


@dataclass
class BatchSpec:
    kind: str  # "stencil2d" | "banded" | "rmat"
    rows: int
    avg: int
    seed: int


def batch_specs(count: int = 512, seed: int = BASE_SEED + 4, rows_lo: int = 1000, rows_hi: int = 200000,
                avg_lo: int = 4, avg_hi: int = 64) -> list[BatchSpec]:
    """Recipe for a batch of uneven matrices: rows log-uniform in [rows_lo, rows_hi],
    integer average nonzeros per row uniform in [avg_lo, avg_hi], structure kinds taken
    round-robin (stencil2d, banded, rmat).  Stencils keep their 5 per row; the side of a
    stencil is round(sqrt(rows)); an R-MAT uses scale round(log2(rows)) and edge factor avg."""
    u = uniform(2 * count, 0.0, 1.0, seed=seed, stream=0)
    kinds = ("stencil2d", "banded", "rmat")
    specs = []
    for i in range(count):
        rows = int(round(math.exp(math.log(rows_lo) + u[2 * i] * (math.log(rows_hi) - math.log(rows_lo)))))
        avg = avg_lo + int(u[2 * i + 1] * (avg_hi - avg_lo + 1))
        avg = min(avg, avg_hi)
        specs.append(BatchSpec(kinds[i % 3], rows, avg, seed * 1000003 + i))
    return specs


def batch_matrix(spec: BatchSpec) -> CSR:
    """Materialise one batch member."""
    if spec.kind == "stencil2d":
        return stencil2d(max(2, int(round(math.sqrt(spec.rows)))))
    if spec.kind == "banded":
        return banded(spec.rows, hbw=1000, per_row=spec.avg, seed=spec.seed)
    if spec.kind == "rmat":
        scale = max(1, int(round(math.log2(spec.rows))))
        return rmat(scale, ef=spec.avg, seed=spec.seed, vals="one")
    raise ValueError(spec.kind)
