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


def kernel_launches():
    """Kernels the CUDA library has launched in this process."""
    return int(_ffi.load().ehl_kernel_launches())


def paqif_partitions(n_sys, n, beta, partitions=0):
    """The blocks per system a batch is solved with: the library's choice for ``partitions`` = 0."""
    lib = _ffi.load()
    out = ctypes.c_int(0)
    _ffi.check(lib.ehl_paqif_partitions(n_sys, n, beta, partitions, ctypes.byref(out)), "ehl_paqif_partitions")
    return out.value


def paqif_workspace_size(n_sys, n, beta, mode, partitions=0):
    lib = _ffi.load()
    out = ctypes.c_size_t(0)
    if partitions:
        _ffi.check(lib.ehl_paqif_workspace_size_partitioned(n_sys, n, beta, partitions, mode, ctypes.byref(out)),
                   "ehl_paqif_workspace_size_partitioned")
    else:
        _ffi.check(lib.ehl_paqif_workspace_size(n_sys, n, beta, mode, ctypes.byref(out)), "ehl_paqif_workspace_size")
    return out.value


def paqif_solve(band, rhs, beta, mode=0, active=None, x=None, workspace=None, stream=None, partitions=0):
    """Batched PAQIF solve.  ``band [n_sys, n, 2 beta + 1]``, ``rhs [n_sys, n]`` float64.

    ``partitions`` > 0 cuts every system into that many blocks (the partitioned
    PAQIF); 0 lets the library choose.  Returns ``(x, iters, info)``;
    ``workspace`` (uint8 CUDA tensor) is optional.
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
        wbytes = paqif_workspace_size(n_sys, n, beta, mode, partitions)
        workspace = torch.empty(wbytes, dtype=torch.uint8, device=band.device)
    wbytes = workspace.numel()
    if partitions:
        code = lib.ehl_paqif_solve_partitioned(n_sys, n, beta, partitions, _ptr(band), _ptr(rhs), _ptr(active), mode,
                                               _ptr(x), _ptr(iters), _ptr(info), _ptr(workspace), wbytes,
                                               _stream(stream))
        _ffi.check(code, "ehl_paqif_solve_partitioned")
    else:
        code = lib.ehl_paqif_solve(n_sys, n, beta, _ptr(band), _ptr(rhs), _ptr(active), mode, _ptr(x), _ptr(iters),
                                   _ptr(info), _ptr(workspace), wbytes, _stream(stream))
        _ffi.check(code, "ehl_paqif_solve")
    return x, iters, info


def paqif_factor_size(n_sys, n, beta):
    lib = _ffi.load()
    out = ctypes.c_size_t(0)
    _ffi.check(lib.ehl_paqif_factor_size(n_sys, n, beta, ctypes.byref(out)), "ehl_paqif_factor_size")
    return out.value


def paqif_factor(band, rhs, beta, mode=0, x=None, factor=None, stream=None):
    """Factor a batch once (and solve it for ``rhs``).  Returns ``(x, info, factor)``; pass
    ``factor`` (uint8 CUDA tensor) to :func:`paqif_resolve` for new right-hand sides."""
    lib = _ffi.load()
    n_sys, n, w = band.shape
    if w != 2 * beta + 1 or rhs.shape != (n_sys, n) or band.dtype != torch.float64 or rhs.dtype != torch.float64:
        raise ValueError("band must be float64 [n_sys, n, 2*beta+1] and rhs float64 [n_sys, n]")
    if x is None:
        x = torch.empty_like(rhs)
    if factor is None:
        factor = torch.empty(paqif_factor_size(n_sys, n, beta), dtype=torch.uint8, device=band.device)
    info = torch.empty(n_sys, dtype=torch.int32, device=band.device)
    _check_dev(band, rhs, x, factor)
    _ffi.check(lib.ehl_paqif_factor(n_sys, n, beta, _ptr(band), _ptr(rhs), mode, _ptr(x), _ptr(info), _ptr(factor),
                                    factor.numel(), _stream(stream)), "ehl_paqif_factor")
    return x, info, factor


def paqif_resolve(factor, rhs, beta, mode=0, x=None, stream=None):
    """Solve a batch factored by :func:`paqif_factor` for a new ``rhs [n_sys, n]``.  Returns ``(x, info)``."""
    lib = _ffi.load()
    n_sys, n = rhs.shape
    if rhs.dtype != torch.float64:
        raise ValueError("rhs must be float64")
    if x is None:
        x = torch.empty_like(rhs)
    info = torch.empty(n_sys, dtype=torch.int32, device=rhs.device)
    _check_dev(rhs, x, factor)
    _ffi.check(lib.ehl_paqif_resolve(n_sys, n, beta, _ptr(rhs), mode, _ptr(x), _ptr(info), _ptr(factor),
                                     factor.numel(), _stream(stream)), "ehl_paqif_resolve")
    return x, info


def default_params(dim=1, **overrides):
    """``ehl_params`` filled by ``ehl_params_default`` with keyword overrides."""
    lib = _ffi.load()
    p = _ffi.EhlParams()
    lib.ehl_params_default(ctypes.byref(p), dim)
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


class Context:
    """An ``ehl_ctx`` for ``n_inst`` instances.

    Device arrays are ``[n_inst][nx_max]``, ``nx_max`` the largest grid of the
    batch; instance ``k`` uses the first ``nxs[k]`` entries of its row (a
    ragged batch when the grids differ).
    """

    def __init__(self, params, n_inst=1, per_inst=None, stream=None):
        lib = _ffi.load()
        self._lib = lib
        self.params = params
        self.per_inst = per_inst
        self.n_inst = n_inst
        self.dim = params.dim
        self.nxs = [q.nx for q in per_inst] if per_inst is not None else [params.nx] * n_inst
        self.nx = max([params.nx] + self.nxs)
        self.ny = params.ny if self.dim == 2 else 1
        self.ragged = any(v != self.nx for v in self.nxs)
        # nodal arrays: [n_inst][nx] (line) or [n_inst][ny][nx] (point, x fastest)
        self.node_shape = (n_inst, self.nx) if self.dim == 1 else (n_inst, self.ny, self.nx)
        self.beta = params.halfband
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        arr = None
        if per_inst is not None:
            arr = (_ffi.EhlParams * n_inst)(*per_inst)
        h = ctypes.c_void_p(0)
        code = lib.ehl_create(ctypes.byref(params), n_inst, arr, ctypes.c_void_p(self._stream.cuda_stream),
                              ctypes.byref(h))
        _ffi.check(code, "ehl_create")
        self._h = h

    def close(self):
        if self._h is not None and self._h.value:
            _ffi.check(self._lib.ehl_destroy(self._h), "ehl_destroy")
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self):
        return torch.device("cuda", torch.cuda.current_device())

    def _check(self, P, H0, rough=None, v=None, v_h0=None):
        _check_dev(P, H0, rough, v, v_h0)
        ns = self.node_shape
        for t, shape in ((P, ns), (H0, (self.n_inst,)), (rough, ns), (v, ns), (v_h0, (self.n_inst,))):
            if t is not None and (tuple(t.shape) != shape or t.dtype != torch.float64):
                raise ValueError(f"expected a float64 tensor of shape {shape}, got {tuple(t.shape)} {t.dtype}")

    def residual(self, P, H0, rough=None):
        self._check(P, H0, rough)
        R = torch.zeros_like(P) if self.ragged else torch.empty_like(P)
        H = torch.zeros_like(P) if self.ragged else torch.empty_like(P)
        comp = torch.empty((self.n_inst, 2), dtype=torch.float64, device=P.device)
        code = self._lib.ehl_residual(self._h, _ptr(P), _ptr(H0), _ptr(rough), _ptr(R), _ptr(H), _ptr(comp))
        _ffi.check(code, "ehl_residual")
        return R, H, comp

    def jacobian_band(self, P, H0, kind=0, rough=None):
        """Band Jacobian: [n_inst][nx-2][2 beta + 1] (line) or the x-line bands
        [n_inst][ny-2][nx-2][2 beta + 1] of the exact Jacobian (point, kind 1), or its
        y-line bands [n_inst][nx-2][ny-2][2 beta + 1] (point, kind 2; act stays [ny-2][nx-2])."""
        self._check(P, H0, rough)
        rows = (self.nx - 2,) if self.dim == 1 else (self.ny - 2, self.nx - 2)
        if self.dim == 2 and kind == 2:
            alloc = torch.empty
            band = alloc((self.n_inst, self.nx - 2, self.ny - 2, 2 * self.beta + 1), dtype=torch.float64,
                         device=P.device)
            act = alloc((self.n_inst,) + rows, dtype=torch.uint8, device=P.device)
            code = self._lib.ehl_jacobian_band(self._h, _ptr(P), _ptr(H0), _ptr(rough), kind, _ptr(band), _ptr(act))
            _ffi.check(code, "ehl_jacobian_band")
            return band, act
        alloc = torch.zeros if self.ragged else torch.empty
        band = alloc((self.n_inst,) + rows + (2 * self.beta + 1,), dtype=torch.float64, device=P.device)
        act = alloc((self.n_inst,) + rows, dtype=torch.uint8, device=P.device)
        code = self._lib.ehl_jacobian_band(self._h, _ptr(P), _ptr(H0), _ptr(rough), kind, _ptr(band), _ptr(act))
        _ffi.check(code, "ehl_jacobian_band")
        return band, act

    def jacobian_apply(self, P, H0, v, v_h0, rough=None):
        self._check(P, H0, rough, v, v_h0)
        out = torch.zeros_like(P) if self.ragged else torch.empty_like(P)
        code = self._lib.ehl_jacobian_apply(self._h, _ptr(P), _ptr(H0), _ptr(rough), _ptr(v), _ptr(v_h0), _ptr(out))
        _ffi.check(code, "ehl_jacobian_apply")
        return out

    def solve(self, P=None, H0=None, rough=None, check=True):
        dev = self._dev()
        init = 1
        if P is None:
            init = 0
            P = torch.zeros(self.node_shape, dtype=torch.float64, device=dev)
            H0 = torch.zeros(self.n_inst, dtype=torch.float64, device=dev)
        else:
            P = P.clone()
            H0 = H0.clone()
        self._check(P, H0, rough)
        iters = torch.zeros(self.n_inst, dtype=torch.int32, device=dev)
        res = torch.zeros((self.n_inst, 2), dtype=torch.float64, device=dev)
        code = self._lib.ehl_solve(self._h, _ptr(P), _ptr(H0), _ptr(rough), init, _ptr(iters), _ptr(res))
        if check:
            _ffi.check(code, "ehl_solve")
        return P, H0, iters, res, code

    def adjoint(self, P, H0, gP=None, gH=None, gH0=None, rough=None, tol=1e-10, max_cycles=10, check=True):
        """Gradients of J(P, H, H0) at a converged state from its partials ``gP``, ``gH``
        ([n_inst][nx]) and ``gH0`` ([n_inst]): ``(grad_rough [n_inst][nx], grad_ML [n_inst][2],
        relres [n_inst], code)``."""
        self._check(P, H0, rough, gP, gH0)
        self._check(P, H0, gH)
        grad_rough = torch.zeros_like(P)
        grad_ML = torch.zeros((self.n_inst, 2), dtype=torch.float64, device=P.device)
        relres = torch.zeros(self.n_inst, dtype=torch.float64, device=P.device)
        code = self._lib.ehl_adjoint(self._h, _ptr(P), _ptr(H0), _ptr(rough), _ptr(gP), _ptr(gH), _ptr(gH0),
                                     _ptr(grad_rough), _ptr(grad_ML), _ptr(relres), float(tol), int(max_cycles))
        if check:
            _ffi.check(code, "ehl_adjoint")
        return grad_rough, grad_ML, relres, code


class _SolveFunction(torch.autograd.Function):
    """Converged ``(P, H, H0)`` as a differentiable function of ``(rough, ML)``."""

    @staticmethod
    def forward(fctx, ctx, rough, ML, P0, H00, tol, max_cycles):
        ML_host = ML.detach().cpu().tolist()
        for k, (M, L) in enumerate(ML_host):
            q = ctx.per_inst[k] if ctx.per_inst is not None else ctx.params
            if abs(M - q.M) > 1e-12 * abs(q.M) or abs(L - q.L) > 1e-12 * abs(q.L):
                raise ValueError("ML must hold the context's (M, L) of every instance")
        r = rough.detach().contiguous()
        if P0 is None:
            P, H0, iters, res, code = ctx.solve(rough=r)
        else:
            P, H0, iters, res, code = ctx.solve(P0, H00, rough=r)
        _, H, _ = ctx.residual(P, H0, r)
        fctx.ehl = ctx
        fctx.tol = tol
        fctx.max_cycles = max_cycles
        fctx.save_for_backward(P, H0, r)
        return P, H, H0

    @staticmethod
    def backward(fctx, gP, gH, gH0):
        P, H0, r = fctx.saved_tensors
        ctx = fctx.ehl
        z = lambda g, t: (g if g is not None else torch.zeros_like(t)).contiguous()
        grad_rough, grad_ML, relres, code = ctx.adjoint(P, H0, z(gP, P), z(gH, P), z(gH0, H0), rough=r,
                                                        tol=fctx.tol, max_cycles=fctx.max_cycles)
        return None, grad_rough, grad_ML, None, None, None, None


def solve_differentiable(ctx, rough, ML, P0=None, H00=None, tol=1e-10, max_cycles=10):
    """Solve through ``ctx`` and return ``(P, H, H0)`` differentiable with respect to the
    roughness ``rough`` ([n_inst][nx]) and ``ML`` ([n_inst][2], the (M, L) the context was
    created with); the backward pass is one ``ehl_adjoint`` call."""
    return _SolveFunction.apply(ctx, rough, ML, P0, H00, tol, max_cycles)


# ---- linear convection-diffusion workload of the line splittings (Sec. 3.1) ----------------------

def cd_params(n, a=1.0, b=0.0, eps=1e-6, kappa=0.0, splitting="Ls0", order="lexicographic", omega=1.0, lo=-1.0,
              hi=1.0):
    """``ehl_cd_params`` for an n x n grid (splitting "Ls0"/"Ls1", order "lexicographic"/"jacobi")."""
    return _ffi.EhlCdParams(int(n), float(lo), float(hi), float(a), float(b), float(eps), float(kappa),
                            {"Ls0": 0, "Ls1": 1}[splitting], {"lexicographic": 0, "jacobi": 1}[order], float(omega))


def cd_residual(p, u, f, stream=None):
    """``(r, rmax)`` of ``u, f`` ([n_inst][n][n] float64, x fastest)."""
    lib = _ffi.load()
    _check_dev(u, f)
    n_inst = u.shape[0]
    r = torch.empty_like(u)
    rmax = torch.empty(n_inst, dtype=torch.float64, device=u.device)
    code = lib.ehl_cd_residual(ctypes.byref(p), n_inst, _ptr(u), _ptr(f), _ptr(r), _ptr(rmax), _stream(stream))
    _ffi.check(code, "ehl_cd_residual")
    return r, rmax


def cd_relax(p, u, f, sweeps, workspace=None, stream=None):
    """``sweeps`` line-relaxation sweeps on ``u`` in place; returns ``(rmax_hist [sweeps][n_inst], info)``."""
    lib = _ffi.load()
    _check_dev(u, f, workspace)
    n_inst = u.shape[0]
    hist = torch.empty((max(sweeps, 1), n_inst), dtype=torch.float64, device=u.device)
    info = torch.empty(n_inst, dtype=torch.int32, device=u.device)
    wbytes = 0
    if workspace is not None:
        wbytes = workspace.numel()
    code = lib.ehl_cd_relax(ctypes.byref(p), n_inst, _ptr(u), _ptr(f), int(sweeps), _ptr(hist), _ptr(info),
                            _ptr(workspace), wbytes, _stream(stream))
    _ffi.check(code, "ehl_cd_relax")
    return hist[:sweeps], info


def cd_workspace_size(p, n_inst):
    nb = ctypes.c_size_t(0)
    _ffi.check(_ffi.load().ehl_cd_workspace_size(ctypes.byref(p), int(n_inst), ctypes.byref(nb)),
               "ehl_cd_workspace_size")
    return nb.value


def paqif_autotune(band, rhs, beta, mode=0, reps=3, stream=None):
    """Fastest partition count for this batch shape (``ehl_paqif_autotune``): ``(r, ms_per_r)``
    with ``ms_per_r[r - 1]`` the best time of each admissible r (-1 where not admissible)."""
    lib = _ffi.load()
    _check_dev(band, rhs)
    n_sys, n, _ = band.shape
    x = torch.empty_like(rhs)
    r = ctypes.c_int(0)
    ms = (ctypes.c_float * 32)()
    code = lib.ehl_paqif_autotune(n_sys, n, beta, mode, _ptr(band), _ptr(rhs), _ptr(x), int(reps), _stream(stream),
                                  ctypes.byref(r), ms)
    _ffi.check(code, "ehl_paqif_autotune")
    return r.value, list(ms)
