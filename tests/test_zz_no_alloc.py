"""The allocation-free PAQIF entry point against the regular one, on the GPU.

ehl_paqif_solve_static serves callers that cannot allocate device memory at
solve time (a program whose own pool owns the GPU, a plug-in inside another
application's callback, a real-time loop that must not wait on the allocator
or fail with out-of-memory mid-run).  It keeps its scratch in a fixed array
that the library reserves on the device.  This file is collected last so a
run that stops at the first failure has already run every other test; it
passes alone in a fresh process too.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2008_03276_gb300 import _ffi, inputs

pytestmark = pytest.mark.gpu
TOL = 1e-12  # the tolerance of the other PAQIF parity tests
SCRATCH_BYTES = 16 << 20  # EHL_PAQIF_STATIC_SCRATCH_BYTES of include/ehl.h


def _p(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _regular(lib, band, rhs, beta, mode, active, stream):
    n_sys, n = rhs.shape
    x = torch.empty_like(rhs)
    it = torch.empty(n_sys, dtype=torch.int32, device=rhs.device)
    info = torch.empty_like(it)
    nb = ctypes.c_size_t(0)
    assert lib.ehl_paqif_workspace_size(n_sys, n, beta, mode, ctypes.byref(nb)) == 0
    ws = torch.empty(nb.value, dtype=torch.uint8, device=rhs.device)
    code = lib.ehl_paqif_solve(n_sys, n, beta, _p(band), _p(rhs), _p(active), mode, _p(x), _p(it), _p(info),
                               _p(ws), nb.value, stream)
    assert code == 0, _ffi.status_string(code)
    return x, it, info


def _static(lib, band, rhs, beta, mode, active, stream):
    n_sys, n = rhs.shape
    x = torch.full_like(rhs, float("nan"))
    it = torch.full((n_sys,), -1, dtype=torch.int32, device=rhs.device)
    info = torch.full_like(it, -1)
    code = lib.ehl_paqif_solve_static(n_sys, n, beta, _p(band), _p(rhs), _p(active), mode, _p(x), _p(it),
                                      _p(info), stream)
    assert code == 0, _ffi.status_string(code)
    return x, it, info


@pytest.mark.parametrize("beta,n,n_sys,mode,use_active", [(4, 1024, 128, 1, False), (2, 255, 257, 2, True),
                                                          (8, 301, 9, 0, False)])
def test_static_matches_regular_twice(beta, n, n_sys, mode, use_active):
    lib = _ffi.load()
    dev = torch.device("cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    results = []
    for call in range(2):  # two calls in a row: the second runs on the first one's leftover scratch
        band_h, rhs_h = inputs.dd_band_systems(n_sys, n, beta, seed=40 + call)
        band = torch.from_numpy(band_h).to(dev)
        rhs = torch.from_numpy(rhs_h).to(dev)
        active = None
        if use_active:
            rng = np.random.default_rng(call)
            active = torch.from_numpy((rng.random((n_sys, n)) < 0.1).astype(np.uint8)).to(dev)
        xr, itr, infr = _regular(lib, band, rhs, beta, mode, active, stream)
        xs, its, infs = _static(lib, band, rhs, beta, mode, active, stream)
        torch.cuda.synchronize()
        xr, xs = xr.cpu().numpy(), xs.cpu().numpy()
        assert np.all(infr.cpu().numpy() == 0) and np.array_equal(infs.cpu().numpy(), infr.cpu().numpy())
        assert np.array_equal(its.cpu().numpy(), itr.cpu().numpy())
        err = np.max(np.abs(xs - xr)) / np.max(np.abs(xr))
        assert err <= TOL
        results.append(xs)
    assert not np.array_equal(results[0], results[1])


def test_static_rejects_batch_beyond_scratch():
    lib = _ffi.load()
    dev = torch.device("cuda")
    # the size check fails before any array is touched, so tiny stand-ins suffice
    band = torch.zeros(1, dtype=torch.float64, device=dev)
    rhs = torch.zeros(1, dtype=torch.float64, device=dev)
    x = torch.empty(1, dtype=torch.float64, device=dev)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    code = lib.ehl_paqif_solve_static(4096, 1024, 4, _p(band), _p(rhs), _p(None), 1, _p(x), _p(None), _p(None),
                                      stream)
    assert code == _ffi.EHL_EINVAL


def _largest_fitting(lib, n, beta, mode):
    """The largest n_sys whose workspace fits in the fixed array (bisection on the size query)."""
    limit = SCRATCH_BYTES
    nb = ctypes.c_size_t(0)

    def need(k):
        assert lib.ehl_paqif_workspace_size(k, n, beta, mode, ctypes.byref(nb)) == 0
        return nb.value

    lo, hi = 1, 1
    while need(hi) <= limit:
        lo, hi = hi, hi * 2
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if need(mid) <= limit:
            lo = mid
        else:
            hi = mid
    return lo


def test_static_accepts_the_largest_batch_and_rejects_one_more():
    lib = _ffi.load()
    dev = torch.device("cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    n, beta, mode = 1024, 4, 1
    k = _largest_fitting(lib, n, beta, mode)
    band_h, rhs_h = inputs.dd_band_systems(k, n, beta, seed=77)
    band = torch.from_numpy(band_h).to(dev)
    rhs = torch.from_numpy(rhs_h).to(dev)
    xr, _, _ = _regular(lib, band, rhs, beta, mode, None, stream)
    xs, _, infs = _static(lib, band, rhs, beta, mode, None, stream)
    torch.cuda.synchronize()
    assert np.all(infs.cpu().numpy() == 0)
    xr, xs = xr.cpu().numpy(), xs.cpu().numpy()
    assert np.max(np.abs(xs - xr)) / np.max(np.abs(xr)) <= TOL
    x = torch.empty(1, dtype=torch.float64, device=dev)
    code = lib.ehl_paqif_solve_static(k + 1, n, beta, _p(band), _p(rhs), _p(None), mode, _p(x), _p(None),
                                      _p(None), stream)
    assert code == _ffi.EHL_EINVAL
