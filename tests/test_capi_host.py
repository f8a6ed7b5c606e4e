"""Host-side checks of the C ABI: the library loads, exports what include/lbm.h
declares, and rejects bad arguments before any launch.  No GPU is touched:
none of the calls below reaches a kernel or a CUDA copy."""
import ctypes
import os
import re

import pytest

from paper_2201_11330_b300 import build as B
from paper_2201_11330_b300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return lbm.load()


def _header_functions():
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", text)))


def test_header_matches_binding():
    assert _header_functions() == sorted(lbm.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _header_functions():
        assert hasattr(lib, name), name


def test_default_opts_and_tau(lib):
    o = lbm.lbm_default_opts()
    assert o.storage == lbm.LBM_F32 and o.aa == 0 and o.compressible == 0
    assert o.rho0 == 1.0 and list(o.lid_u) == [0.0, 0.0, 0.0]
    assert o.collision == lbm.LBM_COLL_BGK and o.trt_lambda == 3 / 16
    assert lbm.lbm_tau_from_paper(0.3) == 0.8
    assert lbm.lbm_error_string(lbm.LBM_ERR_ARG) == "invalid argument"
    assert lbm.lbm_error_string(12345) == "unknown status"


def test_workspace_bytes(lib):
    o = lbm.lbm_default_opts()
    N = 64 * 48 * 40
    ab = lbm.lbm_workspace_bytes(lbm.LBM_D3Q19, 64, 48, 40, o)
    assert ab >= 2 * 19 * N * 4
    o.aa = 1
    aa = lbm.lbm_workspace_bytes(lbm.LBM_D3Q19, 64, 48, 40, o)
    assert 19 * N * 4 <= aa < ab
    o.storage = lbm.LBM_F16S
    assert lbm.lbm_workspace_bytes(lbm.LBM_D3Q19, 64, 48, 40, o) < aa
    # invalid shapes and options
    assert lbm.lbm_workspace_bytes(lbm.LBM_D2Q9, 8, 8, 2, o) == 0
    assert lbm.lbm_workspace_bytes(lbm.LBM_D3Q19, 0, 8, 8, o) == 0
    assert lbm.lbm_workspace_bytes(7, 8, 8, 8, o) == 0
    assert lbm.lbm_workspace_bytes(lbm.LBM_D3Q27, 2048, 2048, 1024, o) == 0  # N >= 2^31
    o.storage = 9
    assert lbm.lbm_workspace_bytes(lbm.LBM_D3Q19, 8, 8, 8, o) == 0


def _create(lib, lattice=lbm.LBM_D3Q19, shape=(8, 8, 8), tau=0.8, bc=lbm.LBM_BC_CAVITY,
            opts=None, ws=256 * 1024, nbytes=None):
    o = opts or lbm.lbm_default_opts()
    need = lbm.lbm_workspace_bytes(lattice, *shape, o)
    ctx = ctypes.c_void_p()
    rc = lib.lbm_create(lattice, *shape, tau, bc, ctypes.byref(o), ctypes.c_void_p(ws),
                        need if nbytes is None else nbytes, None, ctypes.byref(ctx))
    return rc, ctx


def test_create_validates_before_touching_memory(lib):
    # The workspace pointer below is never dereferenced: lbm_create only
    # records it, and every failing case returns before that.
    assert _create(lib, tau=0.5)[0] == lbm.LBM_ERR_ARG
    assert _create(lib, tau=float("nan"))[0] == lbm.LBM_ERR_ARG
    assert _create(lib, bc=5)[0] == lbm.LBM_ERR_ARG
    assert _create(lib, lattice=lbm.LBM_D2Q9, shape=(8, 8, 3))[0] == lbm.LBM_ERR_ARG
    assert _create(lib, ws=256 + 8)[0] == lbm.LBM_ERR_ARG  # misaligned workspace
    assert _create(lib, ws=0)[0] == lbm.LBM_ERR_ARG
    assert _create(lib, nbytes=1024)[0] == lbm.LBM_ERR_NOMEM
    o = lbm.lbm_default_opts()
    o.rho0 = -1.0
    assert _create(lib, opts=o)[0] == lbm.LBM_ERR_ARG
    # two-relaxation-time collision: Lambda > 0, incompressible model only
    o = lbm.lbm_default_opts()
    o.collision = 7
    assert _create(lib, opts=o)[0] == lbm.LBM_ERR_ARG
    o.collision = lbm.LBM_COLL_TRT
    for lam in (0.0, -0.1, float("inf"), float("nan")):
        o.trt_lambda = lam
        assert _create(lib, opts=o)[0] == lbm.LBM_ERR_ARG
    o.trt_lambda = 3 / 16
    o.compressible = 1
    assert _create(lib, opts=o)[0] == lbm.LBM_ERR_ARG
    # MRT: FP64 / FP32 storage, incompressible, rates 0 or in (0, 2)
    o = lbm.lbm_default_opts()
    o.collision = lbm.LBM_COLL_MRT
    for st, rc in ((lbm.LBM_F64, lbm.LBM_OK), (lbm.LBM_F32, lbm.LBM_OK),
                   (lbm.LBM_F16S, lbm.LBM_ERR_ARG), (lbm.LBM_BF16S, lbm.LBM_ERR_ARG)):
        o.storage = st
        r, ctx = _create(lib, opts=o)
        assert r == rc, st
        if r == lbm.LBM_OK:
            lib.lbm_destroy(ctx)
    o.storage = lbm.LBM_F32
    o.compressible = 1
    assert _create(lib, opts=o)[0] == lbm.LBM_ERR_ARG
    o.compressible = 0
    for bad in (2.0, -0.5, float("nan")):
        o.mrt_odd = bad
        assert _create(lib, opts=o)[0] == lbm.LBM_ERR_ARG
    o.mrt_odd = 1.5
    r, ctx = _create(lib, opts=o)
    assert r == lbm.LBM_OK
    lib.lbm_destroy(ctx)
    # the compressible model runs with every storage type
    o = lbm.lbm_default_opts()
    o.compressible = 1
    for st, rc in ((lbm.LBM_F64, lbm.LBM_OK), (lbm.LBM_F32, lbm.LBM_OK),
                   (lbm.LBM_F16S, lbm.LBM_OK), (lbm.LBM_BF16S, lbm.LBM_OK)):
        o.storage = st
        r, ctx = _create(lib, opts=o)
        assert r == rc, st
        if r == lbm.LBM_OK:
            lib.lbm_destroy(ctx)


def test_state_machine_errors_without_launch(lib):
    rc, ctx = _create(lib)
    assert rc == lbm.LBM_OK
    try:
        assert lib.lbm_step_count(ctx) == 0
        # not initialised: these return before any launch
        assert lib.lbm_step(ctx, 1) == lbm.LBM_ERR_STATE
        assert lib.lbm_step(ctx, -1) == lbm.LBM_ERR_ARG
        out = (ctypes.c_double * 6)()
        assert lib.lbm_reduce(ctx, out) == lbm.LBM_ERR_STATE
        assert lib.lbm_macroscopic(ctx, None, None, 3) == lbm.LBM_ERR_ARG
        # force needs has_force at creation
        assert lib.lbm_set_force(ctx, ctypes.c_void_p(512)) == lbm.LBM_ERR_STATE
        bad = (ctypes.c_double * 3)(float("inf"), 0, 0)
        assert lib.lbm_set_lid(ctx, bad) == lbm.LBM_ERR_ARG
        assert lib.lbm_state_bytes(ctx) == 19 * 512 * 4
        assert lib.lbm_adjoint_workspace_bytes(ctx, 0, 1) == 0
        # graph replays: even step counts, 0 (off) or -1 (automatic)
        for bad in (3, -2, 1):
            assert lib.lbm_set_graph_steps(ctx, bad) == lbm.LBM_ERR_ARG
        for good in (0, 2, 32, -1):
            assert lib.lbm_set_graph_steps(ctx, good) == lbm.LBM_OK
    finally:
        lib.lbm_destroy(ctx)
    o = lbm.lbm_default_opts()
    o.collision = lbm.LBM_COLL_TRT
    rc, ctx = _create(lib, opts=o)
    assert rc == lbm.LBM_OK
    try:  # the adjoint covers BGK only
        assert lib.lbm_adjoint_workspace_bytes(ctx, 10, 2) == 0
    finally:
        lib.lbm_destroy(ctx)
    assert lib.lbm_step_count(None) == -1


def test_noalloc_reduction_refuses_faces_and_obstacles(lib):
    # Checked on the host before any device call (the pointers are never used).
    out = (ctypes.c_double * 6)()
    o = lbm.lbm_default_opts()
    assert lib.lbm_reduce_state_noalloc(lbm.LBM_D3Q19, 8, 8, 8, lbm.LBM_BC_FACES,
                                        ctypes.byref(o), ctypes.c_void_p(256), 0, None, None,
                                        out) == lbm.LBM_ERR_ARG
    o.geometry = 1
    assert lib.lbm_reduce_state_noalloc(lbm.LBM_D3Q19, 8, 8, 8, lbm.LBM_BC_CAVITY,
                                        ctypes.byref(o), ctypes.c_void_p(256), 0, None, None,
                                        out) == lbm.LBM_ERR_ARG


def test_noalloc_reduction_refuses_what_lbm_create_refuses(lib):
    # The same option checks as lbm_create, on the host before any device call.
    out = (ctypes.c_double * 6)()
    for field, value in (("storage", 9), ("rho0", -1.0), ("collision", 7),
                         ("p_outflow", 0.0), ("trt_lambda", -1.0)):
        o = lbm.lbm_default_opts()
        if field == "trt_lambda":
            o.collision = lbm.LBM_COLL_TRT
        setattr(o, field, value)
        assert lib.lbm_reduce_state_noalloc(lbm.LBM_D3Q19, 8, 8, 8, lbm.LBM_BC_CAVITY,
                                            ctypes.byref(o), ctypes.c_void_p(256), 0, None,
                                            None, out) == lbm.LBM_ERR_ARG, field
