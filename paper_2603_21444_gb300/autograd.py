"""Differentiable SpGEMM on fixed sparsity patterns.

``SpGEMMFunction.apply(a_val, b_val, pat, deterministic)`` (or
``spgemm_values``) returns the values of C = A B on C's pattern, which a
``Pattern`` sizes once for the pattern pair (pat.A, pat.B); its backward
gives

    dA_ik = sum_{j in B_k} G_ij b_kj    on pattern(A)
    dB_kj = sum_{i: k in A_i} a_ik G_ij on pattern(B)

(the chain rule on C_ij = sum_k a_ik b_kj), both computed by the CUDA
library (``spgemm_backward``).  Values are float32 or float64 tensors on the
device; patterns are ``DeviceCSR`` objects whose ``val`` is ignored.
"""
from __future__ import annotations

import ctypes

import torch

from . import _abi
from .api import DeviceCSR, Handle, _dtype_code, _stream, default_handle, numeric_into, symbolic
from ._abi import CsrIn, CsrOut, check


def backward(A: DeviceCSR, B: DeviceCSR, C: DeviceCSR, grad: torch.Tensor, need_a: bool = True,
             need_b: bool = True, deterministic: bool = False, handle: Handle | None = None, stream=None):
    """(dA values, dB values) for upstream gradient ``grad`` on C's pattern."""
    h = handle or default_handle()
    dt = grad.dtype
    dA = torch.empty(A.nnz, dtype=dt, device=grad.device) if need_a else None
    dB = torch.empty(B.nnz, dtype=dt, device=grad.device) if need_b else None
    a, b = A.as_in(), B.as_in()
    c = CsrIn(C.nrows, C.ncols, C.nnz, C.row_ptr.data_ptr(), C.col.data_ptr() if C.nnz else None,
              grad.data_ptr() if C.nnz else None)
    check(_abi.lib().spgemm_backward(h.ptr, _dtype_code(dt), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                     ctypes.c_void_p(dA.data_ptr() if dA is not None and A.nnz else 0),
                                     ctypes.c_void_p(dB.data_ptr() if dB is not None and B.nnz else 0),
                                     1 if deterministic else 0, _stream(stream)), "spgemm_backward")
    return dA, dB


def transpose(X: DeviceCSR, handle: Handle | None = None, stream=None) -> DeviceCSR:
    """X^T with sorted rows."""
    h = handle or default_handle()
    dev = X.row_ptr.device
    T = DeviceCSR(X.ncols, X.nrows, torch.empty(X.ncols + 1, dtype=torch.int32, device=dev),
                  torch.empty(X.nnz, dtype=torch.int32, device=dev),
                  torch.empty(X.nnz, dtype=X.val.dtype, device=dev) if X.val is not None else None)
    xin, tout = X.as_in(), T.as_out()
    dt = X.val.dtype if X.val is not None else torch.float64
    check(_abi.lib().spgemm_csr_transpose(h.ptr, _dtype_code(dt), ctypes.byref(xin), ctypes.byref(tout),
                                          _stream(stream)), "spgemm_csr_transpose")
    return T


class Pattern:
    """Fixed patterns of A and B and the pattern of C = A B (sized once)."""

    def __init__(self, A: DeviceCSR, B: DeviceCSR, handle: Handle | None = None):
        self.A, self.B = A, B
        self.h = handle or default_handle()
        rp, nnz = symbolic(A, B, self.h)
        dev = A.row_ptr.device
        self.C = DeviceCSR(A.nrows, B.ncols, rp, torch.empty(nnz, dtype=torch.int32, device=dev), None)


class SpGEMMFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, a_val, b_val, pat: Pattern, deterministic: bool = False):
        A = DeviceCSR(pat.A.nrows, pat.A.ncols, pat.A.row_ptr, pat.A.col, a_val.contiguous())
        B = DeviceCSR(pat.B.nrows, pat.B.ncols, pat.B.row_ptr, pat.B.col, b_val.contiguous())
        C = DeviceCSR(pat.C.nrows, pat.C.ncols, pat.C.row_ptr, pat.C.col,
                      torch.empty(pat.C.nnz, dtype=a_val.dtype, device=a_val.device))
        numeric_into(A, B, C, pat.h)
        ctx.pat = pat
        ctx.deterministic = deterministic
        ctx.save_for_backward(A.val, B.val)
        return C.val

    @staticmethod
    def backward(ctx, grad):
        a_val, b_val = ctx.saved_tensors
        pat = ctx.pat
        A = DeviceCSR(pat.A.nrows, pat.A.ncols, pat.A.row_ptr, pat.A.col, a_val)
        B = DeviceCSR(pat.B.nrows, pat.B.ncols, pat.B.row_ptr, pat.B.col, b_val)
        dA, dB = backward(A, B, pat.C, grad.contiguous(), ctx.needs_input_grad[0], ctx.needs_input_grad[1],
                          ctx.deterministic, pat.h)
        return dA, dB, None, None


def spgemm_values(a_val: torch.Tensor, b_val: torch.Tensor, pat: Pattern, deterministic: bool = False):
    """Differentiable values of C = A B on ``pat.C``'s pattern."""
    return SpGEMMFunction.apply(a_val, b_val, pat, deterministic)
