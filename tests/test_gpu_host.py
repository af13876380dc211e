"""The product from host memory (inputs and output in page-locked host
memory, the output copied out in row panels while later panels run) against
the CPU oracle and the device entry points: identical bits."""
import numpy as np
import pytest
import torch

import gen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tsg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2603_21444_gb300 as m
    return m


def host(tsg, X):
    return tsg.DeviceCSR.from_host(X, device="cpu", pin=True)


@pytest.mark.parametrize("panels", [1, 3, 8, 1024])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_host_product_matches_oracle(tsg, panels, dtype):
    A = gen.er_variable(3000, 2000, 30, 11, dtype, "normal", p_empty=0.1)
    B = gen.er_variable(2000, 2500, 25, 12, dtype, "normal", p_empty=0.1)
    h = tsg.Handle()
    C = tsg.spgemm_host(host(tsg, A), host(tsg, B), h, panels=panels)
    ref, _ = oracle.spgemm(A, B, "f32" if dtype == np.float32 else "f64")
    assert C.row_ptr.device.type == "cpu" and C.col.is_pinned()
    assert np.array_equal(C.row_ptr.numpy(), ref.rowptr)
    assert np.array_equal(C.col.numpy(), ref.col)
    assert np.array_equal(C.val.numpy(), ref.val)
    assert h.device_status() == 0
    h.close()


def test_host_product_reuses_output_and_equals_device_path(tsg):
    A = gen.er(1 << 14, 1 << 14, 16, 0)
    B = gen.er(1 << 14, 1 << 14, 16, 1)
    hA, hB = host(tsg, A), host(tsg, B)
    h = tsg.Handle()
    C1 = tsg.spgemm_host(hA, hB, h)
    C2 = tsg.spgemm_host(hA, hB, h, out=C1)  # same buffers, second call
    assert C2.col.data_ptr() == C1.col.data_ptr()
    D = tsg.spgemm(tsg.DeviceCSR.from_host(A), tsg.DeviceCSR.from_host(B), h)
    torch.cuda.synchronize()
    for x, y in zip((C2.row_ptr.numpy().astype(np.int64), C2.col.numpy(), C2.val.numpy()), D.to_host()):
        assert np.array_equal(x, y)
    h.close()


def test_host_product_empty_and_tiny(tsg):
    h = tsg.Handle()
    A = gen.CSR(5, 4, np.zeros(6, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0))
    B = gen.er(4, 3, 2, 1)
    C = tsg.spgemm_host(host(tsg, A), host(tsg, B), h, panels=4)
    assert C.row_ptr.tolist() == [0] * 6 and C.col.numel() == 0
    A1 = gen.from_dense(np.array([[1.0, 2.0]]))
    B1 = gen.from_dense(np.array([[3.0, 0.0], [4.0, 5.0]]))
    C = tsg.spgemm_host(host(tsg, A1), host(tsg, B1), h, panels=16)
    assert C.row_ptr.tolist() == [0, 2] and C.col.tolist() == [0, 1] and C.val.tolist() == [11.0, 10.0]
    h.close()


def test_host_product_with_input_checks(tsg):
    # the panels' row_ptr views start at absolute offsets: with input checks
    # on, the whole matrices are checked once and the panels run unchecked
    import ctypes
    from paper_2603_21444_gb300 import _abi
    A = gen.er_variable(4000, 3000, 20, 31, np.float64, "normal", p_empty=0.05)
    B = gen.er_variable(3000, 3500, 20, 32, np.float64, "normal", p_empty=0.05)
    ref, _ = oracle.spgemm(A, B)
    h = tsg.Handle()
    t = tsg.default_tune()
    t.validate = 1
    h.set_tune(t)
    C = tsg.spgemm_host(host(tsg, A), host(tsg, B), h, panels=8)
    assert np.array_equal(C.col.numpy(), ref.col) and np.array_equal(C.val.numpy(), ref.val)
    # numeric on other host copies of the same matrices than the sizing call
    # saw: indices copied and checked again
    hA2, hB2 = host(tsg, A), host(tsg, B)
    C.col.zero_()
    C.val.zero_()
    ain, bin_, cout = hA2.as_in(), hB2.as_in(), C.as_out()
    _abi.check(_abi.lib().spgemm_host_numeric(h.ptr, _abi.F64, ctypes.byref(ain), ctypes.byref(bin_),
                                              ctypes.byref(cout), 5, ctypes.c_void_p(0)), "spgemm_host_numeric")
    assert np.array_equal(C.col.numpy(), ref.col) and np.array_equal(C.val.numpy(), ref.val)
    # a column index out of range is reported, not read
    Bad = gen.CSR(B.nrows, B.ncols, B.rowptr.copy(), B.col.copy(), B.val.copy())
    Bad.col[len(Bad.col) // 2] = B.ncols + 7
    with pytest.raises(RuntimeError):
        tsg.spgemm_host(host(tsg, A), host(tsg, Bad), h, panels=4)
    assert h.device_status() == 0
    h.set_tune(None)
    h.close()


def test_host_numeric_repeated_with_new_values(tsg):
    # the sizing call uploads the values for the numeric call right after it;
    # a later numeric call on the same arrays copies the (changed) values again
    import ctypes
    from paper_2603_21444_gb300 import _abi
    A = gen.er_variable(2500, 2000, 24, 51, np.float64, "normal", p_empty=0.05)
    B = gen.er_variable(2000, 2200, 24, 52, np.float64, "normal", p_empty=0.05)
    hA, hB = host(tsg, A), host(tsg, B)
    h = tsg.Handle()
    C = tsg.spgemm_host(hA, hB, h, panels=6)
    ref, _ = oracle.spgemm(A, B)
    assert np.array_equal(C.val.numpy(), ref.val)
    B2 = gen.CSR(B.nrows, B.ncols, B.rowptr, B.col, -3.0 * B.val + 0.5)
    hB.val.copy_(torch.from_numpy(B2.val))
    ain, bin_, cout = hA.as_in(), hB.as_in(), C.as_out()
    for panels in (1, 7):
        C.val.zero_()
        _abi.check(_abi.lib().spgemm_host_numeric(h.ptr, _abi.F64, ctypes.byref(ain), ctypes.byref(bin_),
                                                  ctypes.byref(cout), panels, ctypes.c_void_p(0)), "spgemm_host_numeric")
        ref2, _ = oracle.spgemm(A, B2)
        assert np.array_equal(C.col.numpy(), ref2.col) and np.array_equal(C.val.numpy(), ref2.val)
    # sizing without the values (-1), then the numeric call copies them
    nnz = ctypes.c_int64()
    _abi.check(_abi.lib().spgemm_host_symbolic(h.ptr, -1, ctypes.byref(ain), ctypes.byref(bin_),
                                               ctypes.c_void_p(C.row_ptr.data_ptr()), ctypes.byref(nnz),
                                               ctypes.c_void_p(0)), "spgemm_host_symbolic")
    assert nnz.value == C.nnz
    C.val.zero_()
    _abi.check(_abi.lib().spgemm_host_numeric(h.ptr, _abi.F64, ctypes.byref(ain), ctypes.byref(bin_),
                                              ctypes.byref(cout), 3, ctypes.c_void_p(0)), "spgemm_host_numeric")
    assert np.array_equal(C.val.numpy(), ref2.val)
    assert h.device_status() == 0
    h.close()
