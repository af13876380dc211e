"""Host round trip of DeviceCSR.save_npz / load_npz (on the CPU device: no
library call is involved)."""
import numpy as np
import pytest
import torch

import gen


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_save_load_round_trip(tmp_path, dtype):
    from paper_2603_21444_gb300 import DeviceCSR
    X = gen.er_variable(57, 41, 9, 3, dtype, "normal", p_empty=0.2)
    D = DeviceCSR.from_host(X, device="cpu")
    path = tmp_path / "x.npz"
    D.save_npz(path)
    E = DeviceCSR.load_npz(path, device="cpu")
    assert (E.nrows, E.ncols) == (57, 41)
    assert torch.equal(E.row_ptr, D.row_ptr) and torch.equal(E.col, D.col) and torch.equal(E.val, D.val)
    assert E.row_ptr.dtype == torch.int32 and E.val.dtype == D.val.dtype


def test_pattern_only_and_empty(tmp_path):
    from paper_2603_21444_gb300 import DeviceCSR
    D = DeviceCSR(3, 5, torch.zeros(4, dtype=torch.int32), torch.zeros(0, dtype=torch.int32), None)
    D.save_npz(tmp_path / "e.npz")
    E = DeviceCSR.load_npz(tmp_path / "e.npz", device="cpu")
    assert (E.nrows, E.ncols, E.nnz, E.val) == (3, 5, 0, None)


def test_inconsistent_file_refused(tmp_path):
    from paper_2603_21444_gb300 import DeviceCSR
    np.savez(tmp_path / "bad.npz", shape=np.array([2, 2]), row_ptr=np.array([0, 1, 3]), col=np.array([0, 1]))
    with pytest.raises(ValueError):
        DeviceCSR.load_npz(tmp_path / "bad.npz", device="cpu")


@pytest.mark.parametrize("case", ["row_ptr_start", "row_ptr_decreasing", "col_negative", "col_too_large",
                                  "row_ptr_beyond_int32", "values_short", "negative_shape"])
def test_corrupt_file_refused_before_device(tmp_path, case):
    from paper_2603_21444_gb300 import DeviceCSR
    shape, rp, col, val = np.array([3, 4]), np.array([0, 1, 2, 3]), np.array([0, 3, 2]), np.ones(3)
    if case == "row_ptr_start":
        rp = np.array([1, 1, 2, 3])
    elif case == "row_ptr_decreasing":
        rp, col, val = np.array([0, 2, 1, 3]), np.array([0, 1, 2]), np.ones(3)
    elif case == "col_negative":
        col = np.array([0, -1, 2])
    elif case == "col_too_large":
        col = np.array([0, 4, 2])
    elif case == "row_ptr_beyond_int32":
        rp = np.array([0, 1, 2, 2**32 + 3], dtype=np.int64)  # wraps to 3 if cast without a check
    elif case == "values_short":
        val = np.ones(2)
    elif case == "negative_shape":
        shape = np.array([-1, 4])
    np.savez(tmp_path / "c.npz", shape=shape, row_ptr=rp, col=col, val=val)
    with pytest.raises(ValueError):
        DeviceCSR.load_npz(tmp_path / "c.npz", device="cpu")
