"""The C-ABI library builds, loads without a GPU, and exports every function that
include/*.h declares; argument errors are reported before any CUDA call."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**([A-Za-z_][A-Za-z0-9_]*)\s*\(", text, re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1302_1078_gb300 import _capi

    return _capi.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("spmv_csr", "spmm_csr", "gbs_plan_create", "spmv_csr_plan", "gbs_validate_csr"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1302_1078_gb300 import _capi

    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"
    # and the Python binding declares a signature for each of them
    unbound = [n for n in declared_functions() if n not in _capi.SIGNATURES]
    assert not unbound, f"no ctypes signature for: {unbound}"


def test_status_strings(lib):
    assert lib.gbs_status_string(0) == b"ok"
    assert lib.gbs_status_string(-1) == b"invalid argument"
    assert lib.gbs_version() >= 100


def test_argument_errors_need_no_gpu(lib):
    from paper_1302_1078_gb300 import _capi

    # negative sizes, bad dtype, ld < k: rejected on the host before any CUDA call
    assert lib.spmv_csr(-1, 4, 0, None, None, None, 0, None, None, None) == _capi.GBS_EINVAL
    assert lib.spmv_csr(4, 4, 0, 16, None, None, 7, None, None, None) == _capi.GBS_EDTYPE
    assert lib.spmm_csr(4, 4, 0, 16, None, None, 0, 8, 16, 4, 16, 8, None) == _capi.GBS_EINVAL
    assert lib.spmm_csr(4, 4, 0, 16, None, None, 0, 0, 16, 4, 16, 4, None) == _capi.GBS_EINVAL
    assert lib.spmv_csr(4, 4, 10, 16, None, None, 0, 16, 16, None) == _capi.GBS_EINVAL  # NULL col_idx with nnz > 0
    assert b"NULL" in lib.gbs_last_error()
    assert lib.gbs_plan_create(None, 1, 1, 0, None, None, 0, 1, 0, None) == _capi.GBS_EINVAL
    cfg = _capi.gbs_config(variant=1, lanes=3, threads=256, tile_nnz=2048, items=0)
    assert lib.spmv_csr_cfg(4, 4, 0, 16, None, None, 0, 16, 16, ctypes.byref(cfg), None) == _capi.GBS_EINVAL
    assert lib.gbs_ucld(4, 4, 0, 16, None, 0, None, None, None, None) == _capi.GBS_EINVAL  # line_elems < 1
    assert lib.gbs_ucld(-1, 4, 0, None, None, 8, None, None, None, None) == _capi.GBS_EINVAL
    assert lib.gbs_tplan_set_config(None, 0, 1, None, None) == _capi.GBS_EINVAL
    # reordering and register blocking: argument checks on the host
    assert lib.gbs_rcm(-1, 0, None, None, None, None) == _capi.GBS_EINVAL
    assert lib.gbs_rcm(4, 0, 16, None, None, None) == _capi.GBS_EINVAL  # perm is NULL
    assert lib.gbs_permute_csr(4, 0, 16, None, None, 0, None, None, None, None, None) == _capi.GBS_EINVAL
    assert lib.gbs_permute_csr(4, 0, 16, None, 16, 9, 16, 16, None, 16, None) == _capi.GBS_EDTYPE
    h = ctypes.c_void_p()
    assert lib.gbs_bcsr_create(ctypes.byref(h), 4, 4, 0, 16, None, 16, 0, 3, 8, None) == _capi.GBS_EUNSUPPORTED
    assert lib.gbs_bcsr_create(ctypes.byref(h), 4, 4, 0, 16, None, 16, 7, 8, 8, None) == _capi.GBS_EDTYPE
    assert lib.gbs_bcsr_create(None, 4, 4, 0, 16, None, 16, 0, 8, 8, None) == _capi.GBS_EINVAL
    assert lib.spmv_bcsr(None, None, None, None) == _capi.GBS_EINVAL
    assert lib.gbs_bcsr_destroy(None) == _capi.GBS_OK
    assert lib.spmv_csr_batched_plan_cfg(None, 1, None, 0, 1, 0, None, None) == _capi.GBS_EINVAL
    # size limit m + nnz <= 2^31 - 4097: one past it is refused on the host, for every kind of call
    big = 2**31 - 4096
    assert lib.spmv_csr(1, 4, big - 1, 16, 16, 16, 0, 16, 16, None) == _capi.GBS_EUNSUPPORTED
    assert b"2^31 - 4097" in lib.gbs_last_error()
    assert lib.gbs_plan_create(ctypes.byref(h), 1, 4, big - 1, 16, 16, 0, 1, 0, None) == _capi.GBS_EUNSUPPORTED
    assert lib.gbs_transpose_plan(ctypes.byref(h), 1, 4, big - 1, 16, 16, None) == _capi.GBS_EUNSUPPORTED
    assert lib.gbs_ucld(1, 4, big - 1, 16, 16, 8, None, None, None, None) == _capi.GBS_EUNSUPPORTED


@pytest.mark.parametrize("entry", ["spmv_csr", "spmv_csr_noalloc"])
def test_misaligned_pointers_are_refused_on_the_host(lib, entry):
    """A pointer off its element size is refused with GBS_EALIGN before any CUDA call (the
    pointers are never dereferenced, so no GPU is needed): vals, x, y at an odd byte offset
    for FP64 and FP32, and row_ptr / col_idx off 4 bytes."""
    from paper_1302_1078_gb300 import _capi

    f = getattr(lib, entry)
    ok = 4096
    for dt in (_capi.GBS_F64, _capi.GBS_F32):
        for bad in range(5):
            args = [ok, ok, ok, ok, ok]  # row_ptr, col_idx, vals, x, y
            args[bad] = ok + 2
            rp, ci, v, x, y = args
            assert f(8, 8, 16, rp, ci, v, dt, x, y, None) == _capi.GBS_EALIGN, (dt, bad)
            assert b"aligned" in lib.gbs_last_error()
    # FP64 arrays 4 bytes off: aligned for FP32 but not for FP64
    assert f(8, 8, 16, ok, ok, ok + 4, _capi.GBS_F64, ok, ok, None) == _capi.GBS_EALIGN


def test_default_config_host_only(lib):
    from paper_1302_1078_gb300 import _capi

    st = _capi.gbs_stats(m=1000, n=1000, nnz=27000, max_row=27, empty_rows=0, mean_row=27.0, cv_row=0.05)
    c = _capi.gbs_config()
    assert lib.gbs_default_config(ctypes.byref(st), 0, 1, ctypes.byref(c)) == 0
    assert c.variant == _capi.VARIANT_ROWS and c.lanes == 1
    st2 = _capi.gbs_stats(m=1000, n=1000, nnz=16000, max_row=5000, empty_rows=300, mean_row=16.0, cv_row=8.0)
    assert lib.gbs_default_config(ctypes.byref(st2), 0, 1, ctypes.byref(c)) == 0
    assert c.variant == _capi.VARIANT_MERGE


def test_binding_checks_operands_before_any_call():
    """The Python binding refuses operands the kernels would read out of bounds, before it
    touches the library or a device (so this runs on the CPU)."""
    import torch

    import paper_1302_1078_gb300 as gbs

    rp = torch.tensor([0, 2, 3], dtype=torch.int32)
    ci = torch.tensor([0, 1, 1], dtype=torch.int32)
    x = torch.zeros(2, dtype=torch.float64)
    with pytest.raises(ValueError, match="vals"):
        gbs.spmv_csr(rp, ci, torch.zeros(2, dtype=torch.float64), x)  # nnz = 3
    with pytest.raises(ValueError, match="vals"):
        gbs.spmv_csr(rp, ci, torch.zeros(6, dtype=torch.float64)[::2], x)  # not contiguous
    with pytest.raises(ValueError, match="x must"):
        gbs.spmv_csr(rp, ci, torch.zeros(3, dtype=torch.float64), x, n=4)  # x shorter than n
    with pytest.raises(ValueError, match="x must"):
        gbs.spmv_csr(rp, ci, torch.zeros(3, dtype=torch.float64), x.float())  # dtype
    with pytest.raises(ValueError, match="vals"):
        gbs.spmm_csr(rp, ci, torch.zeros(4, dtype=torch.float64), torch.zeros(2, 3, dtype=torch.float64))
    with pytest.raises(ValueError, match="CUDA"):  # well-formed host tensors: refused as not on a GPU
        gbs.spmv_csr(rp, ci, torch.zeros(3, dtype=torch.float64), x)

