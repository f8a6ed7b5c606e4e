"""The allocation-free monitor reduction, lbm_reduce_state_noalloc.

Callers that may not allocate device memory (a frozen memory pool, a host
callback, a tool that only inspects buffers handed to it) can reduce a state
buffer they already hold.  This file checks, through the C ABI, that the
entry point gives the same six values as the context-based lbm_reduce, on
two calls in a row, for both schemes and both AA layouts, and that a shape
needing more partial sums than its fixed scratch holds is refused before any
launch.  It is collected last so that a failure here does not hide the
others; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_2201_11330_b300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_11330_b300 import build
    build.build()


CASES = [
    # lattice, shape, bc, storage, aa, steps, force
    ("d3q19", (50, 40, 30), "cavity", "f32", True, 13, False),   # AA, streamed layout
    ("d3q19", (50, 40, 30), "cavity", "f32", True, 12, False),   # AA, swapped layout
    ("d3q27", (33, 21, 17), "channel", "f64", False, 9, True),   # pull scheme, force
    ("d2q9", (300, 47, 1), "periodic", "f16s", True, 7, True),
    ("d3q19", (64, 64, 64), "cavity", "bf16s", False, 20, False),
]


@pytest.mark.parametrize("lattice,shape,bc,storage,aa,steps,force", CASES)
def test_noalloc_matches_lbm_reduce(lattice, shape, bc, storage, aa, steps, force):
    from paper_2201_11330_b300 import lbm
    nx, ny, nz = shape
    d = 2 if lattice == "d2q9" else 3
    p0, u0 = W.random_smooth_state(nx, ny, nz, d, amp_u=0.05, seed=17)
    lat = lbm.Lattice(lattice, nx, ny, nz, 0.7, bc, storage=storage, aa=aa,
                      lid=(0.1, 0.0, 0.0), has_force=force)
    F = None
    if force:
        F = torch.from_numpy(W.fourier_force(nx, ny, nz, amplitude=1e-4, seed=3, dims=d)).cuda()
        lat.set_force(F)
    lat.init(torch.from_numpy(p0).cuda(), torch.from_numpy(u0).cuda())
    lat.step(steps)
    ref = lat.reduce()
    want = [ref["mass"], *ref["momentum"], ref["kinetic_energy"], ref["max_speed"]]
    buf, step = lat.get_state()
    stream = torch.cuda.current_stream().cuda_stream
    # the per-node values and the warp sums are those of lbm_reduce bit for
    # bit; only the order of the FP64 additions across blocks differs, so the
    # sums agree to FP64 rounding and the maximum exactly
    N = nx * ny * nz
    for _ in range(2):  # two calls in a row share the static scratch
        got = lbm.lbm_reduce_state_noalloc(lbm.LATTICES[lattice], nx, ny, nz, lbm.BCS[bc],
                                           lat.opts, buf.data_ptr(), step,
                                           None if F is None else F.data_ptr(), stream)
        assert abs(got[0] - want[0]) <= 1e-13 * N
        assert np.allclose(got[1:4], want[1:4], rtol=0, atol=1e-13 * N)
        assert abs(got[4] - want[4]) <= 1e-12 * abs(want[4])
        assert got[5] == want[5]


def test_noalloc_refuses_shapes_beyond_its_scratch():
    from paper_2201_11330_b300 import lbm
    nx, ny, nz = 32, 1, 9000  # 9000 partials > LBM_NOALLOC_MAX_PARTIALS = 8192
    opts = lbm.lbm_default_opts()
    state = torch.zeros(19 * nx * ny * nz, dtype=torch.float32, device="cuda")
    out = (ctypes.c_double * 6)()
    rc = lbm.load().lbm_reduce_state_noalloc(lbm.LBM_D3Q19, nx, ny, nz, lbm.LBM_BC_CAVITY,
                                             ctypes.byref(opts), state.data_ptr(), 0, None,
                                             None, out)
    assert rc == lbm.LBM_ERR_NOMEM
    # one z-plane past the limit is refused too
    rc = lbm.load().lbm_reduce_state_noalloc(lbm.LBM_D3Q19, nx, ny, 8193, lbm.LBM_BC_CAVITY,
                                             ctypes.byref(opts), state.data_ptr(), 0, None,
                                             None, out)
    assert rc == lbm.LBM_ERR_NOMEM
    # exactly the limit (8192 z-planes of one x-segment) works on the same buffer
    rc = lbm.load().lbm_reduce_state_noalloc(lbm.LBM_D3Q19, nx, ny, 8192, lbm.LBM_BC_CAVITY,
                                             ctypes.byref(opts), state.data_ptr(), 0, None,
                                             None, out)
    assert rc == lbm.LBM_OK
    assert out[0] == 32 * 8192  # shifted zeros: P = 1 at every node
