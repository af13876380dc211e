"""Python front end of the trident SpGEMM library.

PyTorch supplies device memory and streams; every step runs in the CUDA
library through the C ABI (``_abi``).  There is no CPU fallback: without a
GPU and the built library these functions raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

from . import _abi
from ._abi import CsrIn, CsrOut, Tune, check

_DT = {torch.float32: _abi.F32, torch.float64: _abi.F64}


@dataclass
class DeviceCSR:
    """CSR matrix in device memory: int32 row_ptr / col, float32 or float64 val."""

    nrows: int
    ncols: int
    row_ptr: torch.Tensor
    col: torch.Tensor
    val: torch.Tensor | None

    @property
    def nnz(self) -> int:
        return int(self.col.numel())

    @property
    def dtype(self):
        return self.val.dtype if self.val is not None else None

    @staticmethod
    def from_host(host, device="cuda", dtype=None, pin: bool = False) -> "DeviceCSR":
        """Copy a host CSR (anything with nrows, ncols, rowptr, col, val numpy arrays)."""
        rp = torch.from_numpy(np.ascontiguousarray(host.rowptr, dtype=np.int32))
        col = torch.from_numpy(np.ascontiguousarray(host.col, dtype=np.int32))
        val = torch.from_numpy(np.ascontiguousarray(host.val))
        if dtype is not None:
            val = val.to(dtype)
        if pin:
            rp, col, val = rp.pin_memory(), col.pin_memory(), val.pin_memory()
        nb = pin
        return DeviceCSR(int(host.nrows), int(host.ncols), rp.to(device, non_blocking=nb),
                         col.to(device, non_blocking=nb), val.to(device, non_blocking=nb))

    def to_host(self):
        """(rowptr int64, col int32, val) numpy arrays."""
        return (self.row_ptr.cpu().numpy().astype(np.int64), self.col.cpu().numpy(),
                None if self.val is None else self.val.cpu().numpy())

    def save_npz(self, path) -> None:
        """Write the matrix to a host .npz file (shape, row_ptr, col, val), e.g.
        a Markov-clustering iterate between iterations."""
        rp, col, val = self.to_host()
        arrays = {"shape": np.array([self.nrows, self.ncols], dtype=np.int64), "row_ptr": rp, "col": col}
        if val is not None:
            arrays["val"] = val
        np.savez(path, **arrays)

    @staticmethod
    def load_npz(path, device="cuda") -> "DeviceCSR":
        """Read a matrix written by save_npz onto ``device``.  The file is
        checked on the host before anything reaches the device (kernels index
        with these arrays): shape non-negative and within int32, row_ptr of
        nrows + 1 non-decreasing entries from 0 to nnz < 2^31, every column
        in [0, ncols), values (if any) one per entry.  Raises ValueError
        otherwise."""
        def bad(why):
            return ValueError(f"invalid CSR file {path}: {why}")

        with np.load(path) as f:
            shape = np.asarray(f["shape"])
            rp64 = np.asarray(f["row_ptr"]).astype(np.int64)
            col64 = np.asarray(f["col"]).astype(np.int64)
            val = f["val"].copy() if "val" in f.files else None
        if shape.shape != (2,) or shape.min() < 0 or shape.max() > 2**31 - 1:
            raise bad("shape")
        nrows, ncols = int(shape[0]), int(shape[1])
        if rp64.ndim != 1 or rp64.size != nrows + 1:
            raise bad("row_ptr length")
        if rp64[0] != 0 or np.any(np.diff(rp64) < 0):
            raise bad("row_ptr must start at 0 and not decrease")
        if rp64[-1] != col64.size or col64.size > 2**31 - 1:
            raise bad("row_ptr[-1] must equal the number of columns stored, below 2^31")
        if col64.size and (col64.min() < 0 or col64.max() >= ncols):
            raise bad("column index outside [0, ncols)")
        if val is not None and val.size != col64.size:
            raise bad("one value per entry")
        rp = torch.from_numpy(rp64.astype(np.int32))
        col = torch.from_numpy(col64.astype(np.int32))
        val = None if val is None else torch.from_numpy(val)
        return DeviceCSR(nrows, ncols, rp.to(device), col.to(device), None if val is None else val.to(device))

    def as_in(self) -> CsrIn:
        return CsrIn(self.nrows, self.ncols, self.nnz, self.row_ptr.data_ptr(),
                     self.col.data_ptr() if self.nnz else None,
                     self.val.data_ptr() if (self.val is not None and self.nnz) else None)

    def as_out(self) -> CsrOut:
        return CsrOut(self.nrows, self.ncols, self.row_ptr.data_ptr(), self.col.data_ptr() or None,
                      (self.val.data_ptr() or None) if self.val is not None else None)


def _stream(stream) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dtype_code(t: torch.dtype) -> int:
    if t not in _DT:
        raise TypeError(f"unsupported value dtype {t}")
    return _DT[t]


def default_tune() -> Tune:
    t = Tune()
    check(_abi.lib().spgemm_default_tune(ctypes.byref(t)), "spgemm_default_tune")
    return t


class Handle:
    """Owns one library handle (workspace, bin lists, instrumentation)."""

    def __init__(self):
        self._h = ctypes.c_void_p()
        check(_abi.lib().spgemm_create(ctypes.byref(self._h)), "spgemm_create")

    @property
    def ptr(self):
        return self._h

    def close(self):
        if self._h:
            _abi.lib().spgemm_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tune(self, tune: Tune | None):
        check(_abi.lib().spgemm_set_tune(self._h, ctypes.byref(tune) if tune is not None else None),
              "spgemm_set_tune")

    def get_tune(self) -> Tune:
        t = Tune()
        check(_abi.lib().spgemm_get_tune(self._h, ctypes.byref(t)), "spgemm_get_tune")
        return t

    def launch_count(self) -> int:
        c = ctypes.c_int64()
        check(_abi.lib().spgemm_launch_count(self._h, ctypes.byref(c)), "spgemm_launch_count")
        return int(c.value)

    def device_status(self) -> int:
        return int(_abi.lib().spgemm_device_status(self._h))

    def mcl_paths(self):
        """Rows of the last ``mcl_step`` on this handle per path (per-block,
        window-summed, batched) and the pilot's products per distinct column."""
        rows = (ctypes.c_int64 * 3)()
        ratio = ctypes.c_double()
        check(_abi.lib().spgemm_mcl_paths(self._h, rows, ctypes.byref(ratio)), "spgemm_mcl_paths")
        return [int(x) for x in rows], float(ratio.value)

    def set_timing(self, on: bool):
        check(_abi.lib().spgemm_set_timing(self._h, 1 if on else 0), "spgemm_set_timing")

    def set_concurrent_bins(self, enable: bool):
        """Per-bin launches as parallel branches (default) or one after another."""
        check(_abi.lib().spgemm_set_concurrent_bins(self._h, 1 if enable else 0), "spgemm_set_concurrent_bins")

    def set_workspace_limit(self, nbytes: int | None):
        """Cap the device bytes this handle's workspace may hold (None: no
        cap); a call that would grow past it raises SPGEMM_ERR_OOM."""
        check(_abi.lib().spgemm_set_workspace_limit(self._h, -1 if nbytes is None else int(nbytes)),
              "spgemm_set_workspace_limit")

    def workspace_bytes(self) -> int:
        """Device bytes the handle's workspace holds now."""
        v = ctypes.c_int64()
        check(_abi.lib().spgemm_workspace_bytes(self._h, ctypes.byref(v)), "spgemm_workspace_bytes")
        return int(v.value)

    def set_wait_test(self, spin_limit: int = 0, hold_tile: int = -1):
        """Fault injection for the bounded look-back wait of the single-pass
        product: cap its polls at spin_limit (0: default) and withhold the
        entry of tile hold_tile (-1: none), which makes that call raise
        SPGEMM_ERR_DEVICE_TIMEOUT."""
        check(_abi.lib().spgemm_set_wait_test(self._h, int(spin_limit), int(hold_tile)), "spgemm_set_wait_test")

    def read_timing(self):
        """(ms per phase, intervals per phase) since the last read."""
        ms = (ctypes.c_double * _abi.NUM_PHASES)()
        cnt = (ctypes.c_int64 * _abi.NUM_PHASES)()
        check(_abi.lib().spgemm_read_timing(self._h, ms, cnt), "spgemm_read_timing")
        return list(ms), list(cnt)


_default = {}


def default_handle() -> Handle:
    dev = torch.cuda.current_device()
    if dev not in _default:
        _default[dev] = Handle()
    return _default[dev]


# -------------------------------------------------------------- the product

def symbolic(A: DeviceCSR, B: DeviceCSR, handle: Handle | None = None, stream=None):
    """Row pointer of C = A B and nnz(C) (one host synchronisation)."""
    h = handle or default_handle()
    rp = torch.empty(A.nrows + 1, dtype=torch.int32, device=A.row_ptr.device)
    nnz = ctypes.c_int64()
    a, b = A.as_in(), B.as_in()
    check(_abi.lib().spgemm_symbolic(h.ptr, ctypes.byref(a), ctypes.byref(b), ctypes.c_void_p(rp.data_ptr()),
                                     ctypes.byref(nnz), _stream(stream)), "spgemm_symbolic")
    return rp, int(nnz.value)


def numeric_into(A: DeviceCSR, B: DeviceCSR, C: DeviceCSR, handle: Handle | None = None, stream=None) -> DeviceCSR:
    """Fill C.col / C.val given C.row_ptr from ``symbolic`` (asynchronous)."""
    h = handle or default_handle()
    a, b, c = A.as_in(), B.as_in(), C.as_out()
    check(_abi.lib().spgemm_numeric(h.ptr, _dtype_code(A.val.dtype), ctypes.byref(a), ctypes.byref(b),
                                    ctypes.byref(c), _stream(stream)), "spgemm_numeric")
    return C


def spgemm(A: DeviceCSR, B: DeviceCSR, handle: Handle | None = None, stream=None) -> DeviceCSR:
    """C = A B (symbolic, allocate, numeric)."""
    if A.val is None or B.val is None or A.val.dtype != B.val.dtype:
        raise TypeError("A and B need values of one dtype")
    rp, nnz = symbolic(A, B, handle, stream)
    dev = A.row_ptr.device
    C = DeviceCSR(A.nrows, B.ncols, rp, torch.empty(nnz, dtype=torch.int32, device=dev),
                  torch.empty(nnz, dtype=A.val.dtype, device=dev))
    return numeric_into(A, B, C, handle, stream)


def spgemm_host(A: DeviceCSR, B: DeviceCSR, handle: Handle | None = None, panels: int = 8, out: DeviceCSR | None = None,
                stream=None) -> DeviceCSR:
    """C = A B with A, B and C in host memory (``spgemm_host_symbolic`` +
    ``spgemm_host_numeric``: the library copies the inputs in (the values
    while the sizing runs), computes C in row panels and copies each panel
    out while the next ones run).  A and B
    are DeviceCSR containers of CPU tensors, page-locked for full speed
    (``DeviceCSR.from_host(x, device="cpu", pin=True)``); ``out``, when its
    sizes match, receives C (pinned buffers reused across calls)."""
    if A.val is None or B.val is None or A.val.dtype != B.val.dtype:
        raise TypeError("A and B need values of one dtype")
    h = handle or default_handle()
    ain, bin_ = A.as_in(), B.as_in()
    rp = out.row_ptr if out is not None and out.row_ptr.numel() == A.nrows + 1 else \
        torch.empty(A.nrows + 1, dtype=torch.int32).pin_memory()
    nnz = ctypes.c_int64()
    check(_abi.lib().spgemm_host_symbolic(h.ptr, _dtype_code(A.val.dtype), ctypes.byref(ain), ctypes.byref(bin_),
                                          ctypes.c_void_p(rp.data_ptr()), ctypes.byref(nnz), _stream(stream)),
          "spgemm_host_symbolic")
    n = int(nnz.value)
    if out is not None and out.col.numel() == n and out.val is not None and out.val.dtype == A.val.dtype:
        col, val = out.col, out.val
    else:
        col = torch.empty(n, dtype=torch.int32).pin_memory()
        val = torch.empty(n, dtype=A.val.dtype).pin_memory()
    C = DeviceCSR(A.nrows, B.ncols, rp, col, val)
    cout = C.as_out()
    check(_abi.lib().spgemm_host_numeric(h.ptr, _dtype_code(A.val.dtype), ctypes.byref(ain), ctypes.byref(bin_),
                                         ctypes.byref(cout), int(panels), _stream(stream)), "spgemm_host_numeric")
    return C


def products(A: DeviceCSR, B: DeviceCSR, handle: Handle | None = None, stream=None) -> int:
    """Sum over rows of the intermediate-product counts (an upper bound of nnz(C))."""
    h = handle or default_handle()
    tot = ctypes.c_int64()
    a, b = A.as_in(), B.as_in()
    check(_abi.lib().spgemm_products(h.ptr, ctypes.byref(a), ctypes.byref(b), ctypes.byref(tot), _stream(stream)),
          "spgemm_products")
    return int(tot.value)


def fused_into(A: DeviceCSR, B: DeviceCSR, C: DeviceCSR, handle: Handle | None = None, stream=None) -> int:
    """Single-pass C = A B into C's buffers (capacity = C.col.numel()); returns nnz(C)."""
    h = handle or default_handle()
    a, b, c = A.as_in(), B.as_in(), C.as_out()
    nnz = ctypes.c_int64()
    check(_abi.lib().spgemm_fused(h.ptr, _dtype_code(A.val.dtype), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                  C.col.numel(), ctypes.byref(nnz), _stream(stream)), "spgemm_fused")
    return int(nnz.value)


def spgemm_single_pass(A: DeviceCSR, B: DeviceCSR, handle: Handle | None = None, stream=None) -> DeviceCSR:
    """C = A B without a separate symbolic pass (buffers sized by the product count)."""
    cap = products(A, B, handle, stream)
    dev = A.row_ptr.device
    C = DeviceCSR(A.nrows, B.ncols, torch.empty(A.nrows + 1, dtype=torch.int32, device=dev),
                  torch.empty(cap, dtype=torch.int32, device=dev), torch.empty(cap, dtype=A.val.dtype, device=dev))
    nnz = fused_into(A, B, C, handle, stream)
    C.col = C.col[:nnz]
    C.val = C.val[:nnz]
    return C


# ------------------------------------------------------------------ merge

def merge(parts: list[DeviceCSR], handle: Handle | None = None, stream=None) -> DeviceCSR:
    """C = parts[0] + parts[1] + ... (union pattern, added in part order)."""
    h = handle or default_handle()
    n = len(parts)
    arr = (CsrIn * n)(*[p.as_in() for p in parts])
    m, ncols, dt = parts[0].nrows, parts[0].ncols, parts[0].val.dtype
    dev = parts[0].row_ptr.device
    rp = torch.empty(m + 1, dtype=torch.int32, device=dev)
    out = CsrOut(m, ncols, rp.data_ptr(), None, None)
    nnz = ctypes.c_int64()
    check(_abi.lib().spgemm_merge(h.ptr, _dtype_code(dt), n, arr, ctypes.byref(out), ctypes.byref(nnz),
                                  _stream(stream)), "spgemm_merge(size)")
    C = DeviceCSR(m, ncols, rp, torch.empty(nnz.value, dtype=torch.int32, device=dev),
                  torch.empty(nnz.value, dtype=dt, device=dev))
    out = C.as_out()
    if nnz.value:
        check(_abi.lib().spgemm_merge(h.ptr, _dtype_code(dt), n, arr, ctypes.byref(out), None, _stream(stream)),
              "spgemm_merge(fill)")
    return C


# ---------------------------------------------------------------- batched

class BatchPlan:
    """Marshalled arguments of one batched problem (built once, called often)."""

    def __init__(self, As: list[DeviceCSR], Bs: list[DeviceCSR], group_ptr: list[int] | None = None):
        if len(As) != len(Bs) or not As:
            raise ValueError("need equally many A and B instances")
        self.As, self.Bs = As, Bs
        self.ninst = len(As)
        self.group_ptr = list(group_ptr) if group_ptr is not None else list(range(self.ninst + 1))
        self.ngroups = len(self.group_ptr) - 1
        self.dtype = As[0].val.dtype
        self.a_arr = (CsrIn * self.ninst)(*[a.as_in() for a in As])
        self.b_arr = (CsrIn * self.ninst)(*[b.as_in() for b in Bs])
        self.gp = (ctypes.c_int32 * (self.ngroups + 1))(*self.group_ptr)
        dev = As[0].row_ptr.device
        self.C = []
        for g in range(self.ngroups):
            t = self.group_ptr[g]
            self.C.append(DeviceCSR(As[t].nrows, Bs[t].ncols,
                                    torch.empty(As[t].nrows + 1, dtype=torch.int32, device=dev),
                                    torch.empty(0, dtype=torch.int32, device=dev),
                                    torch.empty(0, dtype=self.dtype, device=dev)))
        self.nnz = None

    def _out(self, sizing: bool):
        outs = (CsrOut * self.ngroups)()
        for g, C in enumerate(self.C):
            outs[g] = CsrOut(C.nrows, C.ncols, C.row_ptr.data_ptr(), None, None) if sizing else C.as_out()
        return outs

    def size(self, handle: Handle | None = None, tune: Tune | None = None, stream=None):
        h = handle or default_handle()
        nnz = (ctypes.c_int64 * self.ngroups)()
        outs = self._out(True)
        check(_abi.lib().spgemm_batched(h.ptr, _dtype_code(self.dtype), self.ninst, self.a_arr, self.b_arr,
                                        self.ngroups, self.gp, outs, nnz,
                                        ctypes.byref(tune) if tune is not None else None, _stream(stream)),
              "spgemm_batched(size)")
        self.nnz = [int(x) for x in nnz]
        return self.nnz

    def allocate(self):
        dev = self.As[0].row_ptr.device
        for C, n in zip(self.C, self.nnz):
            if C.col.numel() != n:
                C.col = torch.empty(n, dtype=torch.int32, device=dev)
                C.val = torch.empty(n, dtype=self.dtype, device=dev)

    def fill(self, handle: Handle | None = None, tune: Tune | None = None, stream=None):
        h = handle or default_handle()
        outs = self._out(False)
        check(_abi.lib().spgemm_batched(h.ptr, _dtype_code(self.dtype), self.ninst, self.a_arr, self.b_arr,
                                        self.ngroups, self.gp, outs, None,
                                        ctypes.byref(tune) if tune is not None else None, _stream(stream)),
              "spgemm_batched(fill)")
        return self.C

    def run(self, handle: Handle | None = None, tune: Tune | None = None, stream=None):
        self.size(handle, tune, stream)
        self.allocate()
        return self.fill(handle, tune, stream)


def batched(As, Bs, group_ptr=None, handle: Handle | None = None, tune: Tune | None = None, stream=None):
    """Outputs C[g] = sum over the group's instances (in order) of A[t] B[t]."""
    return BatchPlan(As, Bs, group_ptr).run(handle, tune, stream)


# ------------------------------------------------------ trident partition

def trident_bounds(n: int, q: int, lam: int = 1):
    """(coarse, fine) boundaries of the hybrid 2D + 1D split of [0, n) (paper
    Sec. 3.2) from the library (``spgemm_trident_bounds``): coarse tile t
    starts at floor(t n / q), each cut into lam contiguous slices."""
    coarse = (ctypes.c_int32 * (q + 1))()
    fine = (ctypes.c_int32 * (q * lam + 1))()
    check(_abi.lib().spgemm_trident_bounds(n, q, lam, coarse, fine), "spgemm_trident_bounds")
    return list(coarse), list(fine)


def tile_split(X: DeviceCSR, row_bounds, col_bounds, handle: Handle | None = None, stream=None):
    """Cut X into tiles[rp][cp] on the device (columns re-based to the tile)."""
    h = handle or default_handle()
    nrp, ncp = len(row_bounds) - 1, len(col_bounds) - 1
    rb = (ctypes.c_int32 * (nrp + 1))(*row_bounds)
    cb = (ctypes.c_int32 * (ncp + 1))(*col_bounds)
    dev = X.row_ptr.device
    dt = X.val.dtype if X.val is not None else torch.float64
    tiles = [[DeviceCSR(row_bounds[r + 1] - row_bounds[r], col_bounds[c + 1] - col_bounds[c],
                        torch.empty(row_bounds[r + 1] - row_bounds[r] + 1, dtype=torch.int32, device=dev),
                        torch.empty(0, dtype=torch.int32, device=dev), None)
              for c in range(ncp)] for r in range(nrp)]
    outs = (CsrOut * (nrp * ncp))()
    for r in range(nrp):
        for c in range(ncp):
            T = tiles[r][c]
            outs[r * ncp + c] = CsrOut(T.nrows, T.ncols, T.row_ptr.data_ptr(), None, None)
    nnz = (ctypes.c_int64 * (nrp * ncp))()
    xin = X.as_in()
    check(_abi.lib().spgemm_tile_split(h.ptr, _dtype_code(dt), ctypes.byref(xin), nrp, rb, ncp, cb, outs, nnz,
                                       _stream(stream)), "spgemm_tile_split(size)")
    for r in range(nrp):
        for c in range(ncp):
            T = tiles[r][c]
            n = int(nnz[r * ncp + c])
            T.col = torch.empty(n, dtype=torch.int32, device=dev)
            T.val = torch.empty(n, dtype=dt, device=dev) if X.val is not None else None
            outs[r * ncp + c] = T.as_out()
    check(_abi.lib().spgemm_tile_split(h.ptr, _dtype_code(dt), ctypes.byref(xin), nrp, rb, ncp, cb, outs, None,
                                       _stream(stream)), "spgemm_tile_split(fill)")
    return tiles


def permute(X: DeviceCSR, row_perm: torch.Tensor | None = None, col_perm: torch.Tensor | None = None,
            handle: Handle | None = None, stream=None) -> DeviceCSR:
    """Y = P X Q^T: Y[row_perm[i], col_perm[j]] = X[i, j] (int32 device maps,
    None = identity), rows sorted.  Raises if a map is not a permutation."""
    h = handle or default_handle()
    dev = X.row_ptr.device
    for m, n in ((row_perm, X.nrows), (col_perm, X.ncols)):
        if m is not None and (m.dtype != torch.int32 or m.numel() != n or m.device != dev or not m.is_contiguous()):
            raise ValueError("maps must be contiguous int32 device tensors of the matching length")
    Y = DeviceCSR(X.nrows, X.ncols, torch.empty(X.nrows + 1, dtype=torch.int32, device=dev),
                  torch.empty(X.nnz, dtype=torch.int32, device=dev),
                  torch.empty(X.nnz, dtype=X.val.dtype, device=dev) if X.val is not None else None)
    xin, yout = X.as_in(), Y.as_out()
    dt = X.val.dtype if X.val is not None else torch.float64
    check(_abi.lib().spgemm_csr_permute(h.ptr, _dtype_code(dt), ctypes.byref(xin),
                                        ctypes.c_void_p(row_perm.data_ptr() if row_perm is not None else 0),
                                        ctypes.c_void_p(col_perm.data_ptr() if col_perm is not None else 0),
                                        ctypes.byref(yout), _stream(stream)), "spgemm_csr_permute")
    return Y


def trident_loads(X: DeviceCSR, q: int, lam: int, handle: Handle | None = None, stream=None):
    """nnz of every process's part X_{ijk} of the trident partition (q x q
    coarse tiles, each cut into lam row slices; Sec. 3.2), as q*lam rows of q
    counts, counted on the device (the sizing pass of the tile split).  Their
    max / mean is the imbalance of the paper's Table 2."""
    h = handle or default_handle()
    _, fine = trident_bounds(X.nrows, q, lam)
    coarse_c, _ = trident_bounds(X.ncols, q, 1)
    nrp, ncp = len(fine) - 1, q
    rb = (ctypes.c_int32 * (nrp + 1))(*fine)
    cb = (ctypes.c_int32 * (ncp + 1))(*coarse_c)
    dev = X.row_ptr.device
    rps = [torch.empty(fine[r + 1] - fine[r] + 1, dtype=torch.int32, device=dev) for r in range(nrp) for _ in range(ncp)]
    outs = (CsrOut * (nrp * ncp))()
    for r in range(nrp):
        for c in range(ncp):
            outs[r * ncp + c] = CsrOut(fine[r + 1] - fine[r], coarse_c[c + 1] - coarse_c[c], rps[r * ncp + c].data_ptr(),
                                       None, None)
    nnz = (ctypes.c_int64 * (nrp * ncp))()
    xin = X.as_in()
    dt = X.val.dtype if X.val is not None else torch.float64
    check(_abi.lib().spgemm_tile_split(h.ptr, _dtype_code(dt), ctypes.byref(xin), nrp, rb, ncp, cb, outs, nnz,
                                       _stream(stream)), "spgemm_tile_split(size)")
    return [[int(nnz[r * ncp + c]) for c in range(ncp)] for r in range(nrp)]


def trident_schedule(q: int, lam: int):
    """Instances of the static-Cannon rounds (Alg. 1, Eq. 2) from the library:
    (a_tile, b_tile, group_ptr)."""
    n = q * q * lam * q
    a = (ctypes.c_int32 * n)()
    b = (ctypes.c_int32 * n)()
    gp = (ctypes.c_int32 * (q * q * lam + 1))()
    check(_abi.lib().spgemm_trident_schedule(q, lam, a, b, gp), "spgemm_trident_schedule")
    return list(a), list(b), list(gp)


def tune_cache_open(path: str | None = None) -> int:
    """Take the entries of a persistent autotune cache file into the process's
    cache and append later autotune choices to it (path None: the file named
    by TRIDENT_SPGEMM_TUNE_CACHE, else none).  Returns the entries taken."""
    n = ctypes.c_int64()
    check(_abi.lib().spgemm_tune_cache_open(None if path is None else os.fsencode(path), ctypes.byref(n)),
          "spgemm_tune_cache_open")
    return int(n.value)


def tune_cache_clear():
    """Empty the process's autotune cache and detach its file."""
    check(_abi.lib().spgemm_tune_cache_clear(), "spgemm_tune_cache_clear")


def tune_cache_store(key: int, tune: Tune):
    """Record a layout under a key (appended to the open cache file, if any)."""
    check(_abi.lib().spgemm_tune_cache_store(ctypes.c_uint64(key), ctypes.byref(tune)), "spgemm_tune_cache_store")


def tune_cache_entries() -> list[tuple[int, Tune]]:
    """(key, layout) of every entry of the process's autotune cache, in key order."""
    n = ctypes.c_int64()
    check(_abi.lib().spgemm_tune_cache_count(ctypes.byref(n)), "spgemm_tune_cache_count")
    out = []
    for i in range(n.value):
        k, t = ctypes.c_uint64(), Tune()
        check(_abi.lib().spgemm_tune_cache_entry(i, ctypes.byref(k), ctypes.byref(t)), "spgemm_tune_cache_entry")
        out.append((int(k.value), t))
    return out


class Plan:
    """A batched problem sized once (``spgemm_plan_create``) and executed many
    times (``spgemm_plan_execute``, replayed from a CUDA graph)."""

    def __init__(self, As: list[DeviceCSR], Bs: list[DeviceCSR], group_ptr: list[int] | None = None,
                 tune: Tune | None = None, stream=None):
        if len(As) != len(Bs) or not As:
            raise ValueError("need equally many A and B instances")
        self.As, self.Bs = As, Bs
        self.ninst = len(As)
        self.group_ptr = list(group_ptr) if group_ptr is not None else list(range(self.ninst + 1))
        self.ngroups = len(self.group_ptr) - 1
        self.dtype = As[0].val.dtype
        self.a_arr = (CsrIn * self.ninst)(*[a.as_in() for a in As])
        self.b_arr = (CsrIn * self.ninst)(*[b.as_in() for b in Bs])
        self.gp = (ctypes.c_int32 * (self.ngroups + 1))(*self.group_ptr)
        dev = As[0].row_ptr.device
        rps = [torch.empty(As[self.group_ptr[g]].nrows + 1, dtype=torch.int32, device=dev)
               for g in range(self.ngroups)]
        rp_arr = (ctypes.c_void_p * self.ngroups)(*[r.data_ptr() for r in rps])
        nnz = (ctypes.c_int64 * self.ngroups)()
        self._p = ctypes.c_void_p()
        check(_abi.lib().spgemm_plan_create(_dtype_code(self.dtype), self.ninst, self.a_arr, self.b_arr,
                                            self.ngroups, self.gp, rp_arr, nnz,
                                            ctypes.byref(tune) if tune is not None else None, _stream(stream),
                                            ctypes.byref(self._p)), "spgemm_plan_create")
        self.nnz = [int(x) for x in nnz]
        self.C = []
        for g in range(self.ngroups):
            t = self.group_ptr[g]
            self.C.append(DeviceCSR(As[t].nrows, Bs[t].ncols, rps[g],
                                    torch.empty(self.nnz[g], dtype=torch.int32, device=dev),
                                    torch.empty(self.nnz[g], dtype=self.dtype, device=dev)))
        self.outs = (CsrOut * self.ngroups)(*[C.as_out() for C in self.C])

    def execute(self, use_graph: bool = True, stream=None):
        check(_abi.lib().spgemm_plan_execute(self._p, self.outs, 1 if use_graph else 0, _stream(stream)),
              "spgemm_plan_execute")
        return self.C

    def autotune(self, stream=None) -> Tune:
        t = Tune()
        check(_abi.lib().spgemm_plan_autotune(self._p, self.outs, _stream(stream), ctypes.byref(t)),
              "spgemm_plan_autotune")
        return t

    def launch_count(self) -> int:
        c = ctypes.c_int64()
        check(_abi.lib().spgemm_plan_launch_count(self._p, ctypes.byref(c)), "spgemm_plan_launch_count")
        return int(c.value)

    def set_concurrent_bins(self, enable: bool):
        """Per-bin launches as parallel branches (default) or one after another."""
        check(_abi.lib().spgemm_plan_set_concurrent_bins(self._p, 1 if enable else 0),
              "spgemm_plan_set_concurrent_bins")

    def close(self):
        if self._p:
            _abi.lib().spgemm_plan_destroy(self._p)
            self._p = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class TridentPlan:
    """The trident grid q x q x lambda of C = A B on one device.

    The partition (Sec. 3.2) runs on the device; the rounds of every output
    block follow the static-Cannon stagger (Alg. 1, Eq. 2); each round's
    partial A_{i r' k} B_{r' j} uses the whole tile B_{r' j} (the allgather of
    Alg. 2 is the tile itself on one device).

    fused: one batched problem whose output rows accumulate their q rounds at
    once (partials never materialised), sized once, executed from a CUDA
    graph.  unfused: every partial is its own output, then each block is the
    ordered sum of its partials (the paper's spgeam step).  plain: the
    per-block loop of the paper's local step, one product call per round and
    one merge per block.  All three give identical bits.
    """

    def __init__(self, A: DeviceCSR, B: DeviceCSR, q: int, lam: int, handle: Handle | None = None):
        self.q, self.lam = q, lam
        self.h = handle or default_handle()
        _, rows_fine = trident_bounds(A.nrows, q, lam)
        kc, _ = trident_bounds(A.ncols, q, 1)
        nc, _ = trident_bounds(B.ncols, q, 1)
        self.row_bounds, self.k_bounds, self.col_bounds = rows_fine, kc, nc
        self.A_tiles = tile_split(A, rows_fine, kc, self.h)   # [i*lam + k][r]
        self.B_tiles = tile_split(B, kc, nc, self.h)          # [r][j]
        a_t, b_t, gp = trident_schedule(q, lam)
        self.As = [self.A_tiles[t // q][t % q] for t in a_t]
        self.Bs = [self.B_tiles[t // q][t % q] for t in b_t]
        self.group_ptr = gp
        self.fused = None
        self.partials = None

    def block_index(self, i: int, j: int, k: int) -> int:
        return (i * self.q + j) * self.lam + k

    def fused_plan(self, tune: Tune | None = None) -> Plan:
        if self.fused is None:
            self.fused = Plan(self.As, self.Bs, self.group_ptr, tune)
        return self.fused

    def run_fused(self, use_graph: bool = True, stream=None):
        return self.fused_plan().execute(use_graph, stream)

    def run_unfused(self, stream=None):
        if self.partials is None:
            self.partials = Plan(self.As, self.Bs)
        P = self.partials.execute(True, stream)
        return [merge(P[self.group_ptr[g]:self.group_ptr[g + 1]], self.h, stream)
                for g in range(len(self.group_ptr) - 1)]

    def run_plain(self, stream=None):
        out = []
        for g in range(len(self.group_ptr) - 1):
            parts = [spgemm(self.As[t], self.Bs[t], self.h, stream)
                     for t in range(self.group_ptr[g], self.group_ptr[g + 1])]
            out.append(merge(parts, self.h, stream))
        return out


# ------------------------------------------------------- Markov clustering

def mcl_step(Mt: DeviceCSR, inflation: float = 2.0, prune: float = 1e-4, topk: int = 1000,
             handle: Handle | None = None, stream=None, heavy: int = 0, window: int = 0) -> DeviceCSR:
    """One Markov-clustering iteration (Sec. 5.6) on the transposed
    column-stochastic matrix: expansion fused with inflation, pruning, top-k
    and renormalisation (``spgemm_mcl_expand`` / ``spgemm_mcl_collect``).
    ``heavy``: rows with at least this many products take the batched
    dense-accumulator path (0: the library's default, < 0: never);
    ``window``: rows from 4096 products below that summed window by window in
    shared memory -- 0 as a pilot decides, 1 always (positive values), -1 never."""
    h = handle or default_handle()
    prm = _abi.MclParams(float(inflation), float(prune), int(topk), int(heavy), int(window))
    dev = Mt.row_ptr.device
    rp = torch.empty(Mt.nrows + 1, dtype=torch.int32, device=dev)
    nnz = ctypes.c_int64()
    mi = Mt.as_in()
    check(_abi.lib().spgemm_mcl_expand(h.ptr, ctypes.byref(mi), ctypes.byref(prm), ctypes.c_void_p(rp.data_ptr()),
                                       ctypes.byref(nnz), _stream(stream)), "spgemm_mcl_expand")
    out = DeviceCSR(Mt.nrows, Mt.ncols, rp, torch.empty(nnz.value, dtype=torch.int32, device=dev),
                    torch.empty(nnz.value, dtype=torch.float32, device=dev))
    oo = out.as_out()
    check(_abi.lib().spgemm_mcl_collect(h.ptr, ctypes.byref(oo), _stream(stream)), "spgemm_mcl_collect")
    return out
