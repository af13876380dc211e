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
