"""Torch-facing wrappers of the C ABI: tensors in, tensors out.

Marshalling only -- every step of the computation runs in the CUDA library.
All tensors must live on the current CUDA device; calls are enqueued on the
current torch stream.
"""
import ctypes

import torch

from . import _ffi

INFO_OK, INFO_SINGULAR, INFO_NOCONV, INFO_NONFINITE = 0, 1, 2, 3


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check_dev(*ts):
    for t in ts:
        if t is not None and (not t.is_cuda or not t.is_contiguous()):
            raise ValueError("tensors must be contiguous CUDA tensors")


def paqif_workspace_size(n_sys, n, beta, mode):
    lib = _ffi.load()
    out = ctypes.c_size_t(0)
    _ffi.check(lib.ehl_paqif_workspace_size(n_sys, n, beta, mode, ctypes.byref(out)), "ehl_paqif_workspace_size")
    return out.value


def paqif_solve(band, rhs, beta, mode=0, active=None, x=None, workspace=None, stream=None):
    """Batched PAQIF solve.  ``band [n_sys, n, 2 beta + 1]``, ``rhs [n_sys, n]`` float64.

    Returns ``(x, iters, info)``; ``workspace`` (uint8 CUDA tensor) is optional.
    """
    lib = _ffi.load()
    if band.dim() == 2:
        band = band.unsqueeze(0)
        rhs = rhs.unsqueeze(0)
        if active is not None:
            active = active.unsqueeze(0)
    n_sys, n, w = band.shape
    if w != 2 * beta + 1 or rhs.shape != (n_sys, n):
        raise ValueError("band must be [n_sys, n, 2*beta+1] and rhs [n_sys, n]")
    if band.dtype != torch.float64 or rhs.dtype != torch.float64:
        raise ValueError("band and rhs must be float64")
    if active is not None and (active.dtype != torch.uint8 or active.shape != (n_sys, n)):
        raise ValueError("active must be uint8 [n_sys, n]")
    if x is None:
        x = torch.empty_like(rhs)
    iters = torch.empty(n_sys, dtype=torch.int32, device=band.device)
    info = torch.empty(n_sys, dtype=torch.int32, device=band.device)
    _check_dev(band, rhs, active, x, workspace)
    wbytes = 0
    if workspace is None:
        wbytes = paqif_workspace_size(n_sys, n, beta, mode)
        workspace = torch.empty(wbytes, dtype=torch.uint8, device=band.device)
    wbytes = workspace.numel()
    code = lib.ehl_paqif_solve(n_sys, n, beta, _ptr(band), _ptr(rhs), _ptr(active), mode, _ptr(x), _ptr(iters),
                               _ptr(info), _ptr(workspace), wbytes, _stream(stream))
    _ffi.check(code, "ehl_paqif_solve")
    return x, iters, info
