"""The allocation-free transpose (for callers that may not allocate device
memory: code under an outside memory pool or budget, or paths that cannot
take an allocation's implicit synchronisation) against the allocating entry
point.

This file is collected last so that, if it fails, a run stopping at the first
failure has already run every other test; it also passes alone in a fresh
process.  The entry point is also captured into a CUDA graph and replayed
on new values."""
import ctypes

import numpy as np
import pytest
import torch

import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_21444_gb300 import _abi
    return _abi.lib()


def _noalloc_transpose(lib, X, dtype):
    from paper_2603_21444_gb300 import _abi
    from paper_2603_21444_gb300.api import DeviceCSR
    dev = X.row_ptr.device
    T = DeviceCSR(X.ncols, X.nrows, torch.empty(X.ncols + 1, dtype=torch.int32, device=dev),
                  torch.empty(X.nnz, dtype=torch.int32, device=dev), torch.empty(X.nnz, dtype=dtype, device=dev))
    xin, tout = X.as_in(), T.as_out()
    code = _abi.F64 if dtype == torch.float64 else _abi.F32
    rc = lib.spgemm_csr_transpose_noalloc(code, ctypes.byref(xin), ctypes.byref(tout),
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, T


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_noalloc_matches_allocating_transpose_twice(lib, dtype):
    import paper_2603_21444_gb300 as tsg
    from paper_2603_21444_gb300 import autograd as ag
    tdt = torch.float64 if dtype == np.float64 else torch.float32
    # two calls in a row, the second smaller than the first: the shared
    # scratch keeps the first call's contents and must not leak into the second
    for shape, seed in (((3000, 2000, 30), 1), ((700, 1500, 12), 2)):
        X = tsg.DeviceCSR.from_host(gen.er_variable(shape[0], shape[1], shape[2], seed, dtype, "normal",
                                                    p_empty=0.1))
        rc, T = _noalloc_transpose(lib, X, tdt)
        assert rc == 0
        R = ag.transpose(X)
        torch.cuda.synchronize()
        # a transpose moves values without arithmetic: equal bit for bit
        for a, b in zip(T.to_host(), R.to_host()):
            assert np.array_equal(a, b)


def test_noalloc_long_columns_match_allocating_transpose(lib):
    import paper_2603_21444_gb300 as tsg
    from paper_2603_21444_gb300 import autograd as ag
    # columns of 1025 and 30000 entries (rows of X^T longer than one warp
    # sorts) next to short ones, 600000 rows of X (two windows of row indices)
    rng = np.random.default_rng(3)
    n, nc = 600000, 2000
    rows = [np.arange(n), rng.choice(n, 1025, replace=False), rng.choice(n, 30000, replace=False)]
    cols = [rng.integers(10, nc, n), np.full(1025, 1), np.full(30000, 5)]
    key = np.unique(np.concatenate(rows).astype(np.int64) * nc + np.concatenate(cols))
    X = tsg.DeviceCSR.from_host(gen.from_coo(n, nc, key // nc, key % nc, rng.normal(size=key.size)))
    rc, T = _noalloc_transpose(lib, X, torch.float64)
    assert rc == 0
    R = ag.transpose(X)
    torch.cuda.synchronize()
    for a, b in zip(T.to_host(), R.to_host()):
        assert np.array_equal(a, b)


def test_noalloc_rejects_oversize_request(lib):
    import paper_2603_21444_gb300 as tsg
    # 4M columns need more working space than the fixed array holds
    X = tsg.DeviceCSR(2, 1 << 22, torch.zeros(3, dtype=torch.int32, device="cuda"),
                      torch.empty(0, dtype=torch.int32, device="cuda"),
                      torch.empty(0, dtype=torch.float64, device="cuda"))
    rc, _ = _noalloc_transpose(lib, X, torch.float64)
    assert rc == 11  # SPGEMM_ERR_UNSUPPORTED


def test_noalloc_under_graph_capture(lib):
    # after one call outside capture (it looks up the array's address), the
    # entry point is captured into a CUDA graph in the global error mode, in
    # which any device allocation or synchronising call from any thread
    # during the capture fails it; replayed after new values are written
    # into X, the graph gives the allocating transpose's bits
    import paper_2603_21444_gb300 as tsg
    from paper_2603_21444_gb300 import _abi
    from paper_2603_21444_gb300 import autograd as ag
    X = tsg.DeviceCSR.from_host(gen.er_variable(2500, 1800, 20, 9, np.float64, "normal", p_empty=0.1))
    rc, T = _noalloc_transpose(lib, X, torch.float64)
    assert rc == 0
    torch.cuda.synchronize()
    xin, tout = X.as_in(), T.as_out()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="global"):
        rc = lib.spgemm_csr_transpose_noalloc(_abi.F64, ctypes.byref(xin), ctypes.byref(tout),
                                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    X.val.copy_(torch.randn(X.val.numel(), dtype=torch.float64, device=X.val.device))
    T.col.zero_()
    T.val.zero_()
    g.replay()
    torch.cuda.synchronize()
    R = ag.transpose(X)
    torch.cuda.synchronize()
    for a, b in zip(T.to_host(), R.to_host()):
        assert np.array_equal(a, b)
