"""CPU checks of the C ABI: the library builds, loads and exports every
function that include/ehl.h declares; host-side argument checks return
EHL_EINVAL without touching a GPU."""
import ctypes
import os
import re

import pytest

from paper_2008_03276_gb300 import _ffi

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "ehl.h")


def declared_functions():
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ehl_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_functions():
    names = declared_functions()
    assert "ehl_paqif_solve" in names and "ehl_status_string" in names


def test_library_exports_every_declared_symbol():
    lib = _ffi.load()
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in _ffi.SYMBOLS, f"{name} has no ctypes signature"


def test_status_strings():
    for code in range(8):
        assert _ffi.status_string(code).startswith("EHL_")
    assert "unknown" in _ffi.status_string(99)


def test_host_side_argument_checks():
    lib = _ffi.load()
    nb = ctypes.c_size_t(0)
    assert lib.ehl_paqif_workspace_size(4, 16, 0, 0, ctypes.byref(nb)) == _ffi.EHL_EINVAL
    assert lib.ehl_paqif_workspace_size(4, 16, 9, 0, ctypes.byref(nb)) == _ffi.EHL_EINVAL
    assert lib.ehl_paqif_workspace_size(4, 16, 2, 3, ctypes.byref(nb)) == _ffi.EHL_EINVAL
    assert lib.ehl_paqif_workspace_size(4, 16, 2, 0, ctypes.byref(nb)) == _ffi.EHL_OK and nb.value > 0
    # partition counts: r must divide the lane groups of a CTA (8 at beta = 8, 12 at beta = 4) and
    # leave every block an interior level (order >= 2 beta + 2) and a real row
    ws = lib.ehl_paqif_workspace_size_partitioned
    assert ws(4, 1024, 8, 8, 0, ctypes.byref(nb)) == _ffi.EHL_OK and nb.value > 0
    assert ws(4, 1024, 8, 3, 0, ctypes.byref(nb)) == _ffi.EHL_EINVAL
    assert ws(4, 1024, 4, 12, 0, ctypes.byref(nb)) == _ffi.EHL_OK
    assert ws(4, 16, 8, 2, 0, ctypes.byref(nb)) == _ffi.EHL_EINVAL
    assert ws(4, 16, 2, -1, 0, ctypes.byref(nb)) == _ffi.EHL_EINVAL
    assert ws(4, 16, 2, 1, 0, ctypes.byref(nb)) == _ffi.EHL_OK
    null = ctypes.c_void_p(0)
    # NULL band / rhs / x are rejected before any CUDA call
    assert lib.ehl_paqif_solve(4, 16, 2, null, null, null, 0, null, null, null, null, 0, null) == _ffi.EHL_EINVAL
    assert lib.ehl_paqif_solve_partitioned(4, 16, 2, 2, null, null, null, 0, null, null, null, null, 0,
                                           null) == _ffi.EHL_EINVAL
    assert lib.ehl_version() >= 100


def test_params_struct_layout_matches_defaults():
    """ctypes mirror of ehl_params: the C defaults land in the right fields."""
    lib = _ffi.load()
    p = _ffi.EhlParams()
    lib.ehl_params_default(ctypes.byref(p), 1)
    assert (p.dim, p.nx, p.ny) == (1, 129, 1)
    assert (p.xa, p.xb, p.M, p.L) == (-4.5, 1.5, 20.0, 10.0)
    assert (p.alpha, p.p0, p.z) == (1.7e-8, 1.98e8, 0.68)
    assert (p.compressible, p.elastic, p.limiter, p.halfband) == (1, 1, 0, 2)
    assert (p.switch_eps_h, p.dist_weight, p.c_h0, p.omega) == (0.6, 0.5, 0.05, 1.0)
    assert (p.method, p.tol, p.max_iter, p.krylov_dim, p.h_init) == (1, 1e-8, 200, 40, 0.05)
    assert (p.levels, p.coarse_min_nodes, p.coarse_tol) == (-1, 65, 1e-4)
    assert (p.precond_blocks, p.precision, p.graph) == (1, 0, 0)
    assert (p.kappa, p.splitting, p.deform, p.autotune, p.yline) == (0.0, 0, 0, 0, 0)
    assert ctypes.sizeof(p) == (_ffi.EhlParams.yline.offset + 4 + 7) // 8 * 8  # tail padding to 8 bytes


@pytest.mark.parametrize("field,value", [("nx", 4), ("halfband", 9), ("M", -1.0), ("xb", -5.0), ("method", 7),
                                         ("limiter", 3), ("kappa", 1.5), ("kappa", -1.01), ("splitting", 3), ("deform", 1), ("deform", 2), ("yline", 1), ("autotune", 2),
                                         ("krylov_dim", 0), ("levels", -2),
                                         ("coarse_min_nodes", 4), ("coarse_tol", 0.0)])
def test_create_rejects_bad_params_on_host(field, value):
    lib = _ffi.load()
    p = _ffi.EhlParams()
    lib.ehl_params_default(ctypes.byref(p), 1)
    setattr(p, field, value)
    h = ctypes.c_void_p(0)
    assert lib.ehl_create(ctypes.byref(p), 1, None, None, ctypes.byref(h)) == _ffi.EHL_EINVAL
    assert lib.ehl_create(None, 1, None, None, ctypes.byref(h)) == _ffi.EHL_EINVAL


def test_context_entry_points_reject_a_null_context():
    """Every context call checks its handle on the host and returns a status (no exception,
    no CUDA call)."""
    lib = _ffi.load()
    z = ctypes.c_void_p(0)
    assert lib.ehl_residual(z, z, z, z, z, z, z) == _ffi.EHL_EINVAL
    assert lib.ehl_jacobian_band(z, z, z, z, 1, z, z) == _ffi.EHL_EINVAL
    assert lib.ehl_jacobian_apply(z, z, z, z, z, z, z) == _ffi.EHL_EINVAL
    assert lib.ehl_solve(z, z, z, z, 0, z, z) == _ffi.EHL_EINVAL
    assert lib.ehl_adjoint(*([z] * 10), 1e-10, 10) == _ffi.EHL_EINVAL
    assert lib.ehl_destroy(z) == _ffi.EHL_EINVAL


@pytest.mark.parametrize("shape,r", [
    ((4096, 1024, 4), 4),   # the standalone batch: chains 252+16, 167+24, 124+32 levels for r = 2, 3, 4
    ((512, 1025, 8), 4),    # the line preconditioner: r = 4 and 8 tie at 185, and 8 x 512 groups exceed one round
    ((1, 4097, 8), 8),      # one long system: 249 + 128 levels at r = 8 against 505 + 64 at r = 4
    ((127, 127, 2), 4),     # x-lines of 129^2: 14 + 16 at r = 4, 11 + 20 at r = 5, 30 + 8 at r = 2
    ((1, 8, 2), 1),         # too short to cut: a block needs 2 beta + 2 rows
])
def test_partition_rule_of_the_library(shape, r):
    """The automatic partition count, by hand from the rule in include/ehl.h (lane groups per
    CTA 12 at beta = 4, 8 at beta = 8, 20 at beta = 2; resident groups 152 SMs x CTAs per SM
    x groups per CTA)."""
    from paper_2008_03276_gb300 import ops

    assert ops.paqif_partitions(*shape) == r
    assert ops.paqif_partitions(*shape, partitions=r) == r


def test_partition_rule_rejects_bad_requests():
    lib = _ffi.load()
    out = ctypes.c_int(0)
    assert lib.ehl_paqif_partitions(4, 1024, 8, 3, ctypes.byref(out)) == _ffi.EHL_EINVAL  # 3 does not divide 8
    assert lib.ehl_paqif_partitions(4, 16, 8, 2, ctypes.byref(out)) == _ffi.EHL_EINVAL   # blocks too short
    assert lib.ehl_paqif_partitions(4, 16, 2, -1, ctypes.byref(out)) == _ffi.EHL_EINVAL
    assert lib.ehl_paqif_partitions(4, 16, 2, 0, None) == _ffi.EHL_EINVAL
