"""The C-ABI library loads and exports every symbol the public header
declares; host-only entry points work without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w \*]*?\b(spgemm_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2603_21444_gb300 import _abi, build
    build.build()
    return _abi.lib()


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("spgemm_symbolic", "spgemm_numeric", "spgemm_merge", "spgemm_batched", "spgemm_create",
                     "spgemm_destroy", "spgemm_status_str"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2603_21444_gb300 import _abi
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in _abi.SIGNATURES, f"binding lacks {name}"


def test_host_only_calls(lib):
    from paper_2603_21444_gb300 import _abi
    assert lib.spgemm_status_str(0) == b"ok"
    assert lib.spgemm_status_str(4) == b"output nnz exceeds int32"
    assert b"sm_103a" in lib.spgemm_version()
    t = _abi.Tune()
    assert lib.spgemm_default_tune(ctypes.byref(t)) == 0
    assert t.num_bins == 12
    assert list(t.bin_upper)[:12] == [16, 32, 64, 128, 256, 320, 384, 512, 1024, 2048, 4096, 8192]
    assert list(t.bin_kernel)[:12] == [10, 0, 1, 2, 3, 15, 9, 4, 11, 12, 13, 14]
    assert t.warps_per_block == 16 and t.sym_warps_per_block == 8
    assert lib.spgemm_default_tune(None) == 1
    assert lib.spgemm_destroy(None) == 0


def test_null_handle_rejected(lib):
    # argument checks happen before any CUDA call
    assert lib.spgemm_symbolic(None, None, None, None, None, None) == 1
    assert lib.spgemm_numeric(None, 1, None, None, None, None) == 1
    assert lib.spgemm_merge(None, 1, 1, None, None, None, None) == 1
    assert lib.spgemm_batched(None, 1, 1, None, None, 1, None, None, None, None, None) == 1
    assert lib.spgemm_set_wait_test(None, 1, 0) == 1
    assert lib.spgemm_set_workspace_limit(None, 0) == 1
    assert lib.spgemm_workspace_bytes(None, None) == 1


def test_create_without_device_reports_cuda_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    h = ctypes.c_void_p()
    assert lib.spgemm_create(ctypes.byref(h)) == 6
    assert not h.value


def test_product_path_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2603_21444_gb300 import _abi
    monkeypatch.setattr(_abi, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_abi, "_lib", None)
    with pytest.raises(RuntimeError, match="CUDA library missing"):
        _abi.lib()


def test_trident_schedule_matches_static_cannon(lib):
    import oracle
    from paper_2603_21444_gb300 import api
    for q, lam in [(1, 1), (2, 2), (3, 2), (4, 4), (5, 3)]:
        a, b, gp = api.trident_schedule(q, lam)
        assert gp == [g * q for g in range(q * q * lam + 1)]
        for i in range(q):
            for j in range(q):
                for k in range(lam):
                    g = (i * q + j) * lam + k
                    rounds = oracle.static_cannon_schedule(q, i, j)
                    for r, rr in enumerate(rounds):
                        assert a[gp[g] + r] == (i * lam + k) * q + rr
                        assert b[gp[g] + r] == rr * q + j


def test_trident_bounds_match_oracle():
    import oracle
    from paper_2603_21444_gb300 import api
    for n, q, lam in [(64, 2, 2), (97, 3, 2), (2 ** 21, 4, 4), (10, 4, 3), (5, 1, 1)]:
        assert api.trident_bounds(n, q, lam) == tuple(oracle.trident_bounds(n, q, lam))


def test_trident_bounds_host_call_matches_oracle(lib):
    # the library's split of [0, n) (Sec. 3.2) against the oracle's, host only
    import oracle
    from paper_2603_21444_gb300 import api
    for n, q, lam in [(0, 1, 1), (1, 4, 4), (17, 4, 4), (1000, 3, 2), (2**21, 4, 4), (2**31 - 1, 7, 5), (10, 16, 1)]:
        assert api.trident_bounds(n, q, lam) == tuple(map(list, oracle.trident_bounds(n, q, lam)))
    c = (ctypes.c_int32 * 2)()
    assert lib.spgemm_trident_bounds(-1, 1, 1, c, None) == 1
    assert lib.spgemm_trident_bounds(5, 0, 1, c, None) == 1
    assert lib.spgemm_trident_bounds(5, 1, 0, None, None) == 1
    assert lib.spgemm_trident_bounds(5, 1, 1, None, None) == 0
