"""The C-ABI library loads, exports every function include/bpdc.h declares,
and rejects malformed arguments before touching a GPU."""
import ctypes

import numpy as np
import pytest
import scipy.sparse as sp

import paper_2510_08695_gb300 as pkg
from paper_2510_08695_gb300 import _bpdc, build


@pytest.fixture(scope="module")
def lib():
    build.build()
    return pkg.load()


def test_every_declared_symbol_is_exported(lib):
    syms = pkg.declared_symbols()
    assert len(syms) >= 12
    for s in syms:
        assert hasattr(lib, s), s
    assert pkg.version().startswith("bpdc")


def test_checked_build_exports_every_declared_symbol(lib):
    """libbpdc_checked.so (the bounds-checked debugging build) exports the same
    C-ABI; only it implements bpdc_check_status."""
    chk = ctypes.CDLL(build.LIB_CHECKED)
    for s in pkg.declared_symbols():
        assert hasattr(chk, s), s
    site, index = ctypes.c_int32(), ctypes.c_int64()
    assert lib.bpdc_check_status(0, ctypes.byref(site), ctypes.byref(index)) == _bpdc.ERR_UNSUPPORTED
    assert chk.bpdc_check_status(0, None, None) == _bpdc.ERR_INVALID_ARG


def test_default_options(lib):
    o = _bpdc._Opts()
    lib.bpdc_opts_default(ctypes.byref(o))
    assert o.variant == 0 and abs(o.ms_scale - 0.625) < 1e-7 and o.max_iter == 50
    assert o.dc_enable == 1 and o.dc_prior == 0 and o.tie_seed == 0x2510086950


def _create(lib, H, L, D, priors, opts=None):
    h, kh = _bpdc._csr(H)
    l, kl = _bpdc._csr(L)
    d, kd = _bpdc._csr(D)
    pr = np.ascontiguousarray(priors, dtype=np.float64)
    o = opts or _bpdc.Options()
    oc = o._c()
    out = ctypes.c_void_p()
    rc = lib.bpdc_graph_create(ctypes.byref(h), ctypes.byref(l), ctypes.byref(d),
                               pr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(oc), 0,
                               ctypes.byref(out))
    return rc, out


def _small():
    H = sp.csr_matrix(np.array([[1, 1, 0], [0, 1, 1]], np.uint8))
    L = sp.csr_matrix(np.array([[1, 1, 1]], np.uint8))
    D = sp.csr_matrix(np.array([[1, 0, 1]], np.uint8))
    return H, L, D, np.full(3, 0.1)


def test_argument_validation(lib):
    H, L, D, p = _small()
    # priors outside (0, 1/2]
    for bad in (0.0, 0.6, np.nan, -0.1):
        pr = p.copy()
        pr[1] = bad
        rc, _ = _create(lib, H, L, D, pr)
        assert rc == _bpdc.ERR_INVALID_ARG, bad
    # column counts differ
    rc, _ = _create(lib, H, sp.csr_matrix(np.ones((1, 4), np.uint8)), D, p)
    assert rc == _bpdc.ERR_DIM_MISMATCH
    # options out of range
    for o in (_bpdc.Options(ms_scale=0.0), _bpdc.Options(ms_scale=1.5), _bpdc.Options(max_iter=-1),
              _bpdc.Options(max_iter=70000), _bpdc.Options(dc_enable=2), _bpdc.Options(tie_rel=-1.0)):
        rc, _ = _create(lib, H, L, D, p, o)
        assert rc == _bpdc.ERR_INVALID_ARG, o
    rc, _ = _create(lib, H, L, D, p, _bpdc.Options(variant=2))
    assert rc == _bpdc.ERR_INVALID_ARG
    # malformed CSR: duplicate column, column out of range, bad row_ptr
    ptr = np.array([0, 2, 4], np.int32)
    for col in (np.array([0, 0, 1, 2], np.int32), np.array([0, 1, 1, 3], np.int32)):
        c = _bpdc._Csr(2, 3, 4, ptr.ctypes.data_as(_bpdc._i32p), col.ctypes.data_as(_bpdc._i32p))
        l, kl = _bpdc._csr(L)
        d, kd = _bpdc._csr(D)
        out = ctypes.c_void_p()
        rc = lib.bpdc_graph_create(ctypes.byref(c), ctypes.byref(l), ctypes.byref(d),
                                   p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None, 0,
                                   ctypes.byref(out))
        assert rc == _bpdc.ERR_INVALID_ARG
        assert lib.bpdc_last_error().decode()
    badptr = np.array([0, 3, 2], np.int32)
    col = np.array([0, 1, 2], np.int32)
    c = _bpdc._Csr(2, 3, 2, badptr.ctypes.data_as(_bpdc._i32p), col.ctypes.data_as(_bpdc._i32p))
    l, kl = _bpdc._csr(L)
    d, kd = _bpdc._csr(D)
    out = ctypes.c_void_p()
    assert lib.bpdc_graph_create(ctypes.byref(c), ctypes.byref(l), ctypes.byref(d),
                                 p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None, 0,
                                 ctypes.byref(out)) == _bpdc.ERR_INVALID_ARG
    # NULL arguments
    assert lib.bpdc_graph_create(None, None, None, None, None, 0, ctypes.byref(out)) == _bpdc.ERR_INVALID_ARG
    assert lib.bpdc_graph_create(None, None, None, None, None, 0, None) == _bpdc.ERR_INVALID_ARG
    assert lib.bpdc_decode(None, 1, None, 0, None, 1, None) == _bpdc.ERR_INVALID_ARG
    assert lib.bpdc_graph_get_info(None, None) == _bpdc.ERR_INVALID_ARG
    assert lib.bpdc_graph_destroy(None) == 0


def test_weighted_bp_calls_reject_a_null_graph(lib):
    n = ctypes.c_size_t()
    assert lib.bpdc_wbp_workspace_size(None, 1, 20, 5, ctypes.byref(n)) == _bpdc.ERR_INVALID_ARG
    assert lib.bpdc_wbp_forward(None, 1, None, None, 20, 20.0, 5, None, None, 0, None) == _bpdc.ERR_INVALID_ARG
    assert lib.bpdc_decode_backward(None, 1, None, None, 20, 20.0, 5, None, None, None, 0, None) \
        == _bpdc.ERR_INVALID_ARG


def test_host_decode_rejects_bad_arguments(lib):
    """bpdc_decode_host checks its batch list before it touches a GPU."""
    assert lib.bpdc_decode_host(None, 1, 0, None) == _bpdc.ERR_INVALID_ARG
    assert lib.bpdc_decode_host(None, 0, 0, None) == 0
    arr = (_bpdc._Batch * 1)()
    arr[0].B = 4
    assert lib.bpdc_decode_host(arr, 1, -1, None) == _bpdc.ERR_INVALID_ARG
    assert lib.bpdc_decode_host(arr, 1, 0, None) == _bpdc.ERR_INVALID_ARG   # no graph


def test_allocation_failure_hook_arguments(lib):
    assert lib.bpdc_debug_fail_allocations(-1, 1) == _bpdc.ERR_INVALID_ARG
    assert lib.bpdc_debug_fail_allocations(0, -1) == _bpdc.ERR_INVALID_ARG
    assert lib.bpdc_debug_fail_allocations(2, 1) == 0
    assert lib.bpdc_debug_fail_allocations(0, 0) == 0


def test_valid_problem_needs_a_device_or_succeeds(lib):
    H, L, D, p = _small()
    rc, out = _create(lib, H, L, D, p)
    import torch
    if torch.cuda.is_available():
        assert rc == 0
        assert lib.bpdc_graph_destroy(out) == 0
    else:
        assert rc in (_bpdc.ERR_CUDA, _bpdc.ERR_INVALID_ARG)


def test_smem_peak_rejects_bad_arguments(lib):
    d = ctypes.c_double()
    n = ctypes.c_int32()
    assert lib.bpdc_measure_smem_peak(0, 100, None, ctypes.byref(n)) == _bpdc.ERR_INVALID_ARG
    assert lib.bpdc_measure_smem_peak(0, 4, ctypes.byref(d), ctypes.byref(n)) == _bpdc.ERR_INVALID_ARG
