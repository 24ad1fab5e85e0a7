"""gbspmv: CSR SpMV / SpMM on GB300 (sm_103a) behind a C ABI.

Thin Python binding over ``libgbspmv.so`` (see ``include/gbspmv.h``).  PyTorch
supplies device memory and the current CUDA stream; every step of every
product runs in the library's CUDA kernels.  The functions here only check
and marshal arguments.  If the library cannot be loaded, every call raises:
there is no CPU fallback.

    y = spmv_csr(row_ptr, col_idx, vals, x)           # y <- A x      (paper Sec. 3)
    Y = spmm_csr(row_ptr, col_idx, vals, X)           # Y <- A X, X row major n x k (Sec. 5)
    plan = Plan(row_ptr, col_idx, n, dtype, k, tune=True); plan.spmv(vals, x, y)
"""
from __future__ import annotations

import ctypes

import torch

from . import _capi
from ._capi import GbsError, gbs_config, gbs_stats  # noqa: F401

__all__ = [
    "spmv_csr", "spmm_csr", "Plan", "csr_stats", "validate_csr", "default_config", "GbsError", "lib",
    "TransposePlan", "CsrOperator", "SpMMFunction", "spmm_autograd", "BatchedPlan",
]


def lib():
    """The loaded C library (built on first use if needed)."""
    return _capi.load()


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float64:
        return _capi.GBS_F64
    if t.dtype == torch.float32:
        return _capi.GBS_F32
    raise TypeError(f"values must be float64 or float32, got {t.dtype}")


def _ptr(t) -> int:
    if t is None:
        return 0
    return t.data_ptr() if t.numel() else 0


def _stream(device: torch.device, stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return int(stream.cuda_stream)


def _need_cuda(*ts):
    dev = None
    for t in ts:
        if t is None:
            continue
        if not t.is_cuda:
            raise ValueError("gbspmv operates on CUDA tensors only")
        if dev is None:
            dev = t.device
        elif t.device != dev:
            raise ValueError("all tensors must be on the same device")
    return dev


def _check_index(row_ptr: torch.Tensor, col_idx: torch.Tensor):
    if row_ptr.dtype != torch.int32 or col_idx.dtype != torch.int32:
        raise TypeError("row_ptr and col_idx must be int32")
    if row_ptr.dim() != 1 or col_idx.dim() != 1 or not row_ptr.is_contiguous() or not col_idx.is_contiguous():
        raise ValueError("row_ptr and col_idx must be contiguous 1-D tensors")


def _check_vals(vals: torch.Tensor, nnz: int):
    """The kernels read vals as nnz contiguous entries."""
    if vals.dim() != 1 or vals.numel() != nnz or not vals.is_contiguous():
        raise ValueError(f"vals must be a contiguous 1-D tensor of nnz = {nnz} entries")


def _check_vector(t: torch.Tensor, size: int, dtype, what: str, exact: bool):
    if t.dtype != dtype or t.dim() != 1 or not t.is_contiguous() or (t.numel() != size if exact else t.numel() < size):
        need = f"{size}" if exact else f"at least {size}"
        raise ValueError(f"{what} must be a contiguous 1-D {dtype} tensor of {need} entries")


def _check_block(t: torch.Tensor, rows: int, k: int, dtype, what: str, exact: bool):
    """A row-major rows x k block; its row stride may exceed k."""
    if (t.dtype != dtype or t.dim() != 2 or t.shape[1] != k or t.stride(1) != 1 or
            (t.shape[0] != rows if exact else t.shape[0] < rows)):
        need = f"{rows}" if exact else f"at least {rows}"
        raise ValueError(f"{what} must be a row-major 2-D {dtype} tensor of {need} rows and {k} columns")


def _config(cfg) -> gbs_config | None:
    if cfg is None:
        return None
    if isinstance(cfg, gbs_config):
        return cfg
    c = gbs_config()
    for k, v in dict(cfg).items():
        setattr(c, k, int(v))
    return c


def spmv_csr(row_ptr, col_idx, vals, x, y=None, *, n: int | None = None, config=None, stream=None):
    """y <- A x for the CSR matrix (row_ptr, col_idx, vals).  Returns y."""
    _check_index(row_ptr, col_idx)
    _check_vals(vals, col_idx.numel())
    n = x.numel() if n is None else n
    _check_vector(x, n, vals.dtype, "x", exact=False)
    dev = _need_cuda(row_ptr, col_idx, vals, x, y)
    dt = _dtype_code(vals)
    m = row_ptr.numel() - 1
    if y is None:
        y = torch.empty(m, dtype=vals.dtype, device=dev)
    elif y.dtype != vals.dtype or y.numel() != m or not y.is_contiguous():
        raise ValueError("y must be contiguous with m entries of the values' dtype")
    L = lib()
    c = _config(config)
    s = _stream(dev, stream)
    if c is None:
        rc = L.spmv_csr(m, n, col_idx.numel(), _ptr(row_ptr), _ptr(col_idx), _ptr(vals), dt, _ptr(x), _ptr(y), s)
    else:
        rc = L.spmv_csr_cfg(m, n, col_idx.numel(), _ptr(row_ptr), _ptr(col_idx), _ptr(vals), dt, _ptr(x), _ptr(y),
                            ctypes.byref(c), s)
    _capi.check(rc, "spmv_csr")
    return y


def spmm_csr(row_ptr, col_idx, vals, X, Y=None, *, config=None, stream=None):
    """Y <- A X with X an n x k row-major tensor (a row stride >= k is allowed).  Returns Y."""
    _check_index(row_ptr, col_idx)
    _check_vals(vals, col_idx.numel())
    dev = _need_cuda(row_ptr, col_idx, vals, X, Y)
    dt = _dtype_code(vals)
    if X.dtype != vals.dtype or X.dim() != 2 or X.stride(1) != 1:
        raise ValueError("X must be 2-D, row major, of the values' dtype")
    m = row_ptr.numel() - 1
    n, k = X.shape
    if Y is None:
        Y = torch.empty((m, k), dtype=vals.dtype, device=dev)
    elif Y.dtype != vals.dtype or Y.dim() != 2 or Y.shape != (m, k) or Y.stride(1) != 1:
        raise ValueError("Y must be m x k, row major, of the values' dtype")
    L = lib()
    c = _config(config)
    s = _stream(dev, stream)
    ldx, ldy = max(X.stride(0), k), max(Y.stride(0), k)
    args = (m, n, col_idx.numel(), _ptr(row_ptr), _ptr(col_idx), _ptr(vals), dt, k, _ptr(X), ldx, _ptr(Y), ldy)
    rc = L.spmm_csr(*args, s) if c is None else L.spmm_csr_cfg(*args, ctypes.byref(c), s)
    _capi.check(rc, "spmm_csr")
    return Y


def csr_stats(row_ptr, n: int, nnz: int | None = None, stream=None) -> dict:
    """Row-length statistics computed on the device."""
    dev = _need_cuda(row_ptr)
    m = row_ptr.numel() - 1
    nnz = int(row_ptr[-1].item()) if nnz is None else nnz
    st = gbs_stats()
    _capi.check(lib().gbs_csr_stats(m, n, nnz, _ptr(row_ptr), ctypes.byref(st), _stream(dev, stream)), "gbs_csr_stats")
    return st.as_dict()


def ucld(row_ptr, col_idx, n: int, line_elems: int = 8, stream=None) -> dict:
    """Useful cacheline density (Sec. 4.1) for aligned x lines of ``line_elems`` elements:
    {"ucld": mean over non-empty rows of nnz_i / (line_elems * lines_i), "lines": sum of lines_i,
    "nonempty_rows": ...}, computed on the device."""
    _check_index(row_ptr, col_idx)
    dev = _need_cuda(row_ptr, col_idx)
    m = row_ptr.numel() - 1
    u = ctypes.c_double()
    tot, rows = ctypes.c_longlong(), ctypes.c_longlong()
    _capi.check(lib().gbs_ucld(m, int(n), col_idx.numel(), _ptr(row_ptr), _ptr(col_idx), int(line_elems),
                               ctypes.byref(u), ctypes.byref(tot), ctypes.byref(rows), _stream(dev, stream)),
                "gbs_ucld")
    return {"ucld": u.value, "lines": tot.value, "nonempty_rows": rows.value}


def rcm(row_ptr, col_idx, stream=None):
    """Reverse Cuthill-McKee permutation (int32 device tensor, perm[i] = node placed at i) of the
    symmetric pattern of the square matrix (row_ptr, col_idx) (Sec. 4.4), computed on the device."""
    _check_index(row_ptr, col_idx)
    dev = _need_cuda(row_ptr, col_idx)
    n = row_ptr.numel() - 1
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    _capi.check(lib().gbs_rcm(n, col_idx.numel(), _ptr(row_ptr), _ptr(col_idx), _ptr(perm), _stream(dev, stream)),
                "gbs_rcm")
    return perm


def permute_csr(row_ptr, col_idx, vals, perm, stream=None):
    """B = P A P^T: (row_ptr, col_idx, vals) of B with columns sorted in every row; vals may be None."""
    _check_index(row_ptr, col_idx)
    dev = _need_cuda(row_ptr, col_idx, perm, vals)
    n, nnz = row_ptr.numel() - 1, col_idx.numel()
    brp = torch.empty(n + 1, dtype=torch.int32, device=dev)
    bci = torch.empty(nnz, dtype=torch.int32, device=dev)
    bv = None if vals is None else torch.empty_like(vals)
    dt = 0 if vals is None else _dtype_code(vals)
    _capi.check(lib().gbs_permute_csr(n, nnz, _ptr(row_ptr), _ptr(col_idx), _ptr(vals), dt, _ptr(perm), _ptr(brp),
                                      _ptr(bci), _ptr(bv), _stream(dev, stream)), "gbs_permute_csr")
    return brp, bci, bv


class BCSR:
    """Register-blocked CRS (Sec. 4.5) of (row_ptr, col_idx, vals) with aligned a x b dense blocks,
    converted on the device; spmv(x) multiplies from the blocks."""

    def __init__(self, row_ptr, col_idx, vals, n: int, a: int, b: int, stream=None):
        _check_index(row_ptr, col_idx)
        dev = _need_cuda(row_ptr, col_idx, vals)
        self.m, self.n, self.a, self.b = row_ptr.numel() - 1, int(n), int(a), int(b)
        self.dtype, self.device = vals.dtype, dev
        self._h = ctypes.c_void_p()
        _capi.check(lib().gbs_bcsr_create(ctypes.byref(self._h), self.m, self.n, col_idx.numel(), _ptr(row_ptr),
                                          _ptr(col_idx), _ptr(vals), _dtype_code(vals), self.a, self.b,
                                          _stream(dev, stream)), "gbs_bcsr_create")
        mb, nb = ctypes.c_int(), ctypes.c_longlong()
        _capi.check(lib().gbs_bcsr_info(self._h, ctypes.byref(mb), ctypes.byref(nb), None, None), "gbs_bcsr_info")
        self.block_rows, self.nblocks = mb.value, nb.value

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                lib().gbs_bcsr_destroy(h)
            except Exception:
                pass
            self._h = None

    def arrays(self):
        """Copies of (bptr, bcol, bval) as device tensors."""
        bp, bc, bv = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        _capi.check(lib().gbs_bcsr_arrays(self._h, ctypes.byref(bp), ctypes.byref(bc), ctypes.byref(bv)),
                    "gbs_bcsr_arrays")
        es = 8 if self.dtype == torch.float64 else 4
        out = []
        for ptr, count, dt, size in ((bp, self.block_rows + 1, torch.int32, 4), (bc, self.nblocks, torch.int32, 4),
                                     (bv, self.nblocks * self.a * self.b, self.dtype, es)):
            t = torch.empty(count, dtype=dt, device=self.device)
            if count and ptr.value:
                torch.cuda.synchronize(self.device)
                _cudart_copy(t, ptr.value, count * size)
            out.append(t)
        return tuple(out)

    def spmv(self, x, y=None, stream=None):
        _need_cuda(x, y)
        if y is None:
            y = torch.empty(self.m, dtype=self.dtype, device=self.device)
        _capi.check(lib().spmv_bcsr(self._h, _ptr(x), _ptr(y), _stream(self.device, stream)), "spmv_bcsr")
        return y


def _cudart_copy(dst, src_ptr: int, nbytes: int) -> None:
    """Device-to-device copy from a raw pointer into a tensor (through a zero-copy view)."""
    import numpy as np  # noqa: F401

    class _Arr:
        def __init__(self, ptr, n, dt):
            self.__cuda_array_interface__ = {"shape": (n,), "typestr": dt, "data": (ptr, False), "version": 3}

    typestr = {torch.int32: "<i4", torch.float64: "<f8", torch.float32: "<f4"}[dst.dtype]
    src = torch.as_tensor(_Arr(src_ptr, dst.numel(), typestr), device=dst.device)
    dst.copy_(src)


def validate_csr(row_ptr, col_idx, n: int, stream=None) -> None:
    """Raise GbsError(GBS_EINDEX) if the CSR structure is malformed."""
    dev = _need_cuda(row_ptr, col_idx)
    m = row_ptr.numel() - 1
    _capi.check(lib().gbs_validate_csr(m, n, col_idx.numel(), _ptr(row_ptr), _ptr(col_idx), _stream(dev, stream)),
                "gbs_validate_csr")


def default_config(stats: dict, dtype: torch.dtype, k: int = 1) -> dict:
    st = gbs_stats()
    for key, v in stats.items():
        setattr(st, key, v)
    c = gbs_config()
    dt = _capi.GBS_F64 if dtype == torch.float64 else _capi.GBS_F32
    _capi.check(lib().gbs_default_config(ctypes.byref(st), dt, int(k), ctypes.byref(c)), "gbs_default_config")
    return c.as_dict()


class Plan:
    """A fixed CSR structure with its chosen (optionally autotuned) configuration.

    The plan keeps references to row_ptr and col_idx; executing it allocates nothing."""

    def __init__(self, row_ptr, col_idx, n: int, dtype=torch.float64, k: int = 1, *, tune: bool = False,
                 check: bool = False, emulate: bool = False, config=None, stream=None):
        _check_index(row_ptr, col_idx)
        dev = _need_cuda(row_ptr, col_idx)
        self.row_ptr, self.col_idx = row_ptr, col_idx
        self.m, self.n, self.nnz, self.k = row_ptr.numel() - 1, int(n), col_idx.numel(), int(k)
        self.dtype = dtype
        self.device = dev
        self._h = ctypes.c_void_p()
        flags = (_capi.PLAN_TUNE if tune else 0) | (_capi.PLAN_CHECK if check else 0) | \
            (_capi.PLAN_EMULATE if emulate else 0)
        dt = _capi.GBS_F64 if dtype == torch.float64 else _capi.GBS_F32
        _capi.check(lib().gbs_plan_create(ctypes.byref(self._h), self.m, self.n, self.nnz, _ptr(row_ptr),
                                          _ptr(col_idx), dt, self.k, flags, _stream(dev, stream)), "gbs_plan_create")
        if config is not None:
            self.set_config(config)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                lib().gbs_plan_destroy(h)
            except Exception:
                pass
            self._h = None

    @property
    def config(self) -> dict:
        c = gbs_config()
        _capi.check(lib().gbs_plan_get_config(self._h, ctypes.byref(c)), "gbs_plan_get_config")
        return c.as_dict()

    def set_config(self, cfg) -> None:
        _capi.check(lib().gbs_plan_set_config(self._h, ctypes.byref(_config(cfg))), "gbs_plan_set_config")

    @property
    def stats(self) -> dict:
        st = gbs_stats()
        _capi.check(lib().gbs_plan_get_stats(self._h, ctypes.byref(st)), "gbs_plan_get_stats")
        return st.as_dict()

    def relabel_ids(self, stream=None):
        """newid (int32, n entries, on the device) of a plan whose configuration relabels its
        columns: the rank of each column by stored entries, most first, ties by column id."""
        out = torch.empty(self.n, dtype=torch.int32, device=self.device)
        _capi.check(lib().gbs_plan_relabel_ids(self._h, _ptr(out), _stream(self.device, stream)),
                    "gbs_plan_relabel_ids")
        return out

    def spmv(self, vals, x, y=None, stream=None):
        _need_cuda(vals, x, y)
        if y is None:
            y = torch.empty(self.m, dtype=self.dtype, device=self.device)
        if vals.dtype != self.dtype or x.dtype != self.dtype or y.dtype != self.dtype:
            raise TypeError("dtype differs from the plan's")
        _check_vals(vals, self.nnz)
        _check_vector(x, self.n, self.dtype, "x", exact=False)
        _check_vector(y, self.m, self.dtype, "y", exact=True)
        _capi.check(lib().spmv_csr_plan(self._h, _ptr(vals), _ptr(x), _ptr(y), _stream(self.device, stream)),
                    "spmv_csr_plan")
        return y

    def spmm(self, vals, X, Y=None, stream=None):
        _need_cuda(vals, X, Y)
        if vals.dtype != self.dtype:
            raise TypeError("dtype differs from the plan's")
        _check_vals(vals, self.nnz)
        _check_block(X, self.n, self.k, self.dtype, "X", exact=False)
        if Y is None:
            Y = torch.empty((self.m, self.k), dtype=self.dtype, device=self.device)
        _check_block(Y, self.m, self.k, self.dtype, "Y", exact=True)
        _capi.check(lib().spmm_csr_plan(self._h, _ptr(vals), _ptr(X), max(X.stride(0), self.k), _ptr(Y),
                                        max(Y.stride(0), self.k), _stream(self.device, stream)), "spmm_csr_plan")
        return Y


# --------------------------------------------------------- transpose + backward

class TransposePlan:
    """CSR of A^T built on the device (stable, bit-exact) plus the backward kernels."""

    def __init__(self, row_ptr, col_idx, n: int, stream=None):
        _check_index(row_ptr, col_idx)
        dev = _need_cuda(row_ptr, col_idx)
        self.row_ptr, self.col_idx = row_ptr, col_idx
        self.m, self.n, self.nnz = row_ptr.numel() - 1, int(n), col_idx.numel()
        self.device = dev
        self._h = ctypes.c_void_p()
        _capi.check(lib().gbs_transpose_plan(ctypes.byref(self._h), self.m, self.n, self.nnz, _ptr(row_ptr),
                                             _ptr(col_idx), _stream(dev, stream)), "gbs_transpose_plan")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                lib().gbs_tplan_destroy(h)
            except Exception:
                pass
            self._h = None

    def arrays(self, stream=None):
        """(row_ptr_T [n+1], col_idx_T [nnz], perm [nnz]) as new int32 device tensors."""
        rpT = torch.empty(self.n + 1, dtype=torch.int32, device=self.device)
        ciT = torch.empty(self.nnz, dtype=torch.int32, device=self.device)
        perm = torch.empty(self.nnz, dtype=torch.int32, device=self.device)
        _capi.check(lib().gbs_tplan_export(self._h, _ptr(rpT), _ptr(ciT), _ptr(perm), _stream(self.device, stream)),
                    "gbs_tplan_export")
        return rpT, ciT, perm

    def prepare(self, dtype, k: int, tune: bool = True, stream=None):
        """Make a (tuned) plan of A^T for dtype and k; later backward calls use it for dX."""
        dt = _capi.GBS_F64 if dtype == torch.float64 else _capi.GBS_F32
        _capi.check(lib().gbs_tplan_prepare(self._h, dt, int(k), _capi.PLAN_TUNE if tune else 0,
                                            _stream(self.device, stream)), "gbs_tplan_prepare")

    def set_config(self, dtype, k: int, cfg, stream=None) -> None:
        """Configuration of dX = A^T dY for dtype and k.  ROWS, MERGE and MERGE_DIRECT read A's
        values in place through the transpose permutation; ROWS_TMA permutes them first."""
        dt = _capi.GBS_F64 if dtype == torch.float64 else _capi.GBS_F32
        _capi.check(lib().gbs_tplan_set_config(self._h, dt, int(k), ctypes.byref(_config(cfg)),
                                               _stream(self.device, stream)), "gbs_tplan_set_config")

    def config(self, dtype, k: int) -> dict:
        """The configuration dX uses for dtype and k (prepared, or picked from A^T's row statistics)."""
        dt = _capi.GBS_F64 if dtype == torch.float64 else _capi.GBS_F32
        c = gbs_config()
        _capi.check(lib().gbs_tplan_get_config(self._h, dt, int(k), ctypes.byref(c)), "gbs_tplan_get_config")
        return c.as_dict()

    def backward(self, vals, X, dY, need_dX: bool = True, need_dvals: bool = True, stream=None):
        """(dX, dvals) of Y = A X for upstream dY; X and dY are 1-D (SpMV) or 2-D row major."""
        _need_cuda(vals, X, dY)
        dt = _dtype_code(vals)
        _check_vals(vals, self.nnz)
        if X.dim() != dY.dim() or X.dim() not in (1, 2) or X.shape[0] != self.n or dY.shape[0] != self.m or \
                (X.dim() == 2 and X.shape[1] != dY.shape[1]):
            raise ValueError(f"X must be n = {self.n} by k and dY m = {self.m} by k (both 1-D for k = 1)")
        vec = X.dim() == 1
        k = 1 if vec else X.shape[1]
        if X.dtype != vals.dtype or dY.dtype != vals.dtype:
            raise TypeError("X and dY must have the values' dtype")
        if vec:
            X2, dY2 = X.contiguous(), dY.contiguous()
            ldx = lddy = 1
        else:
            X2 = X if X.stride(1) == 1 else X.contiguous()
            dY2 = dY if dY.stride(1) == 1 else dY.contiguous()
            ldx, lddy = max(X2.stride(0), k), max(dY2.stride(0), k)
        dX = None
        if need_dX:
            dX = torch.empty(self.n if vec else (self.n, k), dtype=vals.dtype, device=self.device)
        dvals = torch.empty(self.nnz, dtype=vals.dtype, device=self.device) if need_dvals else None
        _capi.check(lib().spmv_csr_backward(self._h, _ptr(self.row_ptr), _ptr(self.col_idx), _ptr(vals), dt, k,
                                            _ptr(X2), ldx, _ptr(dY2), lddy, _ptr(dX), k, _ptr(dvals),
                                            _stream(self.device, stream)), "spmv_csr_backward")
        return dX, dvals


class CsrOperator:
    """A fixed sparsity pattern A (m x n) whose product with X is differentiable in both the
    stored values and X:  Y = op(vals, X).  Forward runs through plans (one per k), backward
    through a TransposePlan built on first use (the one-time transpose)."""

    def __init__(self, row_ptr, col_idx, n: int, tune: bool = False):
        _check_index(row_ptr, col_idx)
        self.row_ptr, self.col_idx, self.n = row_ptr, col_idx, int(n)
        self.m = row_ptr.numel() - 1
        self.tune = tune
        self._plans = {}
        self._tplan = None
        self._prepared = set()

    def plan(self, dtype, k):
        key = (dtype, k)
        if key not in self._plans:
            self._plans[key] = Plan(self.row_ptr, self.col_idx, self.n, dtype, k, tune=self.tune)
        return self._plans[key]

    @property
    def tplan(self) -> TransposePlan:
        if self._tplan is None:
            self._tplan = TransposePlan(self.row_ptr, self.col_idx, self.n)
        return self._tplan

    def forward_raw(self, vals, X):
        if X.dim() == 1:
            return self.plan(vals.dtype, 1).spmv(vals, X.contiguous())
        Xc = X if X.stride(1) == 1 else X.contiguous()
        return self.plan(vals.dtype, X.shape[1]).spmm(vals, Xc)

    def __call__(self, vals, X):
        return SpMMFunction.apply(vals, X, self)


class SpMMFunction(torch.autograd.Function):
    """Y = A X (or y = A x) with gradients for the stored values and for X."""

    @staticmethod
    def forward(ctx, vals, X, op: CsrOperator):
        ctx.op = op
        ctx.save_for_backward(vals, X)
        return op.forward_raw(vals, X)

    @staticmethod
    def backward(ctx, dY):
        vals, X = ctx.saved_tensors
        need_v, need_x = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        op = ctx.op
        k = 1 if X.dim() == 1 else X.shape[1]
        if need_x and op.tune and (vals.dtype, k) not in op._prepared:
            op.tplan.prepare(vals.dtype, k, tune=True)
            op._prepared.add((vals.dtype, k))
        dX, dvals = op.tplan.backward(vals, X, dY, need_dX=need_x, need_dvals=need_v)
        return dvals, dX, None


def spmm_autograd(row_ptr, col_idx, vals, X, n: int | None = None):
    """One-shot differentiable product (builds a CsrOperator; reuse one for repeated calls)."""
    n = X.shape[0] if n is None else n
    return CsrOperator(row_ptr, col_idx, n)(vals, X)


# ---------------------------------------------------------------------- batched

class BatchedPlan:
    """Many products Y_b = A_b X_b in one persistent launch replayed from a CUDA graph.

    ``mats``: list of (row_ptr, col_idx, vals, n); ``X``/``Y``: lists of dense operands
    (1-D for k == 1, else n x k / m x k row major).  Keeps references to every tensor."""

    def __init__(self, mats, X, Y, *, tune: bool = False, check: bool = False, configs=None, stream=None):
        if not (len(mats) == len(X) == len(Y)) or not mats:
            raise ValueError("mats, X and Y must be non-empty lists of equal length")
        self.nmat = len(mats)
        self.dtype = mats[0][2].dtype
        self.k = 1 if X[0].dim() == 1 else X[0].shape[1]
        dev = _need_cuda(*[t for mat in mats for t in mat[:3]], *X, *Y)
        self.device = dev
        self._keep = (list(mats), list(X), list(Y))
        arr = (_capi.gbs_batch_item * self.nmat)()
        for b, ((rp, ci, v, n), x, y) in enumerate(zip(mats, X, Y)):
            _check_index(rp, ci)
            if v.dtype != self.dtype or x.dtype != self.dtype or y.dtype != self.dtype:
                raise TypeError("all values and operands must share one dtype")
            kk = 1 if x.dim() == 1 else x.shape[1]
            if kk != self.k:
                raise ValueError("every X must have the same k")
            it = arr[b]
            it.m, it.n, it.nnz = rp.numel() - 1, int(n), ci.numel()
            it.row_ptr, it.col_idx, it.vals = _ptr(rp), _ptr(ci), _ptr(v)
            it.X, it.Y = _ptr(x), _ptr(y)
            it.ldx = max(x.stride(0), self.k) if x.dim() == 2 else 1
            it.ldy = max(y.stride(0), self.k) if y.dim() == 2 else 1
        self._items = arr
        self._h = ctypes.c_void_p()
        flags = (_capi.PLAN_TUNE if tune else 0) | (_capi.PLAN_CHECK if check else 0)
        if configs is None:
            _capi.check(lib().spmv_csr_batched_plan(ctypes.byref(self._h), self.nmat, arr, _dtype_code(mats[0][2]),
                                                    self.k, flags, _stream(dev, stream)), "spmv_csr_batched_plan")
        else:
            # per-matrix configurations (dicts or gbs_config; None / variant 0 = the library's choice)
            if len(configs) != self.nmat:
                raise ValueError("configs must have one entry per matrix")
            cfgs = (gbs_config * self.nmat)()
            for b, c in enumerate(configs):
                if c is not None:
                    cfgs[b] = _config(c)
            _capi.check(lib().spmv_csr_batched_plan_cfg(ctypes.byref(self._h), self.nmat, arr,
                                                        _dtype_code(mats[0][2]), self.k, flags, cfgs,
                                                        _stream(dev, stream)), "spmv_csr_batched_plan_cfg")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                lib().spmv_csr_batched_destroy(h)
            except Exception:
                pass
            self._h = None

    def run(self, X=None, Y=None, stream=None):
        """Replay the graph (optionally with new X / Y lists of the same shapes)."""
        xp = yp = None
        if X is not None:
            xp = (ctypes.c_void_p * self.nmat)(*[_ptr(t) for t in X])
            self._keep = (self._keep[0], list(X), self._keep[2])
        if Y is not None:
            yp = (ctypes.c_void_p * self.nmat)(*[_ptr(t) for t in Y])
            self._keep = (self._keep[0], self._keep[1], list(Y))
        _capi.check(lib().spmv_csr_batched(self._h, xp, yp, _stream(self.device, stream)), "spmv_csr_batched")

    def run_looped(self, stream=None):
        """The same products as one launch per matrix (the baseline)."""
        _capi.check(lib().spmv_csr_batched_looped(self._h, _stream(self.device, stream)), "spmv_csr_batched_looped")

    def info(self) -> dict:
        cfgs = (gbs_config * self.nmat)()
        ib = (ctypes.c_int * (self.nmat + 1))()
        grid, total = ctypes.c_int(), ctypes.c_int()
        _capi.check(lib().spmv_csr_batched_info(self._h, cfgs, ib, ctypes.byref(grid), ctypes.byref(total)),
                    "spmv_csr_batched_info")
        return {"configs": [c.as_dict() for c in cfgs], "item_begin": list(ib), "grid": grid.value,
                "total_items": total.value}

    def offsets(self):
        """(rows, nonzeros, row_ptr entries, X entries, Y entries) offsets, each nmat + 1 int64."""
        import numpy as np

        outs = [np.zeros(self.nmat + 1, np.int64) for _ in range(5)]
        ptrs = [o.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)) for o in outs]
        _capi.check(lib().spmv_csr_batched_offsets(self._h, *ptrs), "spmv_csr_batched_offsets")
        return tuple(outs)
