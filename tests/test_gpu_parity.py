"""GPU (CUDA path through the C ABI) against the FP64 CPU oracle.

Tolerances: FP64 fields 1e-12, FP32 velocity 1e-5, shifted half storage 2e-3,
all as max_x |a - b| / scale with scale = U_ref for velocity and
rho0 U_ref^2 for pressure.  Both sides get identical seeded inputs; the
force field is FP32 on both (the oracle reads it widened to FP64).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2201_11330_b300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_11330_b300 import build
    build.build()


def gpu_run(lattice, shape, tau, bc, steps, *, storage="f64", aa=False, lid=None, F=None,
            p0=None, u0=None, compressible=False, rho0=1.0, f32_unshifted=False,
            trt_lambda=None, kernel="auto", mrt=None):
    from paper_2201_11330_b300.lbm import Lattice
    nx, ny, nz = shape
    lat = Lattice(lattice, nx, ny, nz, tau, bc, storage=storage, aa=aa,
                  compressible=compressible, rho0=rho0, lid=lid or (0, 0, 0),
                  has_force=F is not None, f32_unshifted=f32_unshifted,
                  trt_lambda=trt_lambda, kernel=kernel, mrt=mrt)
    if F is not None:
        lat.set_force(torch.from_numpy(np.ascontiguousarray(F, dtype=np.float32)).cuda())
    lat.init(None if p0 is None else torch.from_numpy(p0).cuda(),
             None if u0 is None else torch.from_numpy(np.ascontiguousarray(u0)).cuda())
    lat.step(steps)
    p, u = lat.macroscopic()
    out = p.cpu().numpy(), u.cpu().numpy(), lat
    torch.cuda.synchronize()
    return out


def oracle_run(lattice, shape, tau, bc, steps, *, lid=None, F=None, p0=None, u0=None,
               compressible=False, rho0=1.0, trt_lambda=None, mrt=None):
    nx, ny, nz = shape
    F64 = None if F is None else np.asarray(F, dtype=np.float32).astype(np.float64)
    return oracle.run(lattice, nx, ny, nz, tau, bc, steps, lid=lid, F=F64, p0=p0,
                      u0=None if u0 is None else np.ascontiguousarray(u0).ravel(),
                      compressible=compressible, rho0=rho0, trt_lambda=trt_lambda, mrt=mrt)


def errors(gpu, ref, uref, rho0=1.0):
    pg, ug = gpu[0], gpu[1]
    pr, ur = ref
    eu = np.abs(ug - ur).max() / uref
    ep = np.abs(pg - pr).max() / (rho0 * uref * uref)
    return eu, ep


TOL = {"f64": 1e-12, "f32": 1e-5, "f16s": 2e-3}


# ---------------------------------------------------------------------------
# D2Q9 lid-driven cavity 64 x 64, FP64, Re = 100, 1000 steps


@pytest.fixture(scope="module")
def cavity2d_ref():
    c = W.cavity_params(64, 100.0, 0.1)
    return c, oracle_run("d2q9", (64, 64, 1), c["tau"], "cavity", 1000, lid=c["lid"])


@pytest.mark.parametrize("aa", [False, True])
@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_cavity2d_64(cavity2d_ref, aa, storage):
    c, ref = cavity2d_ref
    got = gpu_run("d2q9", (64, 64, 1), c["tau"], "cavity", 1000, storage=storage, aa=aa,
                  lid=c["lid"])
    eu, ep = errors(got, ref, 0.1)
    assert eu < TOL[storage] and ep < (TOL[storage] if storage == "f64" else 1e-4), (eu, ep)


# ---------------------------------------------------------------------------
# Ragged multi-tile 3D boxes with random initial states, every BC and lattice


CASES3D = [
    ("d3q19", (37, 29, 23), "cavity"),
    ("d3q19", (300, 7, 5), "channel"),
    ("d3q19", (33, 17, 19), "periodic"),
    ("d3q27", (35, 21, 13), "cavity"),
    ("d3q27", (19, 11, 9), "periodic"),
    ("d3q27", (41, 9, 6), "channel"),
    ("d2q9", (301, 67, 1), "cavity"),
    ("d2q9", (45, 33, 1), "periodic"),
    ("d2q9", (29, 17, 1), "channel"),
]


@pytest.mark.parametrize("lattice,shape,bc", CASES3D)
@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("aa", [False, True])
def test_random_state_parity(lattice, shape, bc, storage, aa):
    Q, d = oracle.dims(lattice)
    nx, ny, nz = shape
    p0, u0 = W.random_smooth_state(nx, ny, nz, d, amp_u=0.04, amp_p=2e-3, seed=21)
    lid = (0.08, 0.0, 0.02) if bc != "periodic" else None
    F = W.fourier_force(nx, ny, nz, amplitude=2e-5, seed=5, dims=d)
    steps = 61  # odd: the AA state ends in its streamed form
    ref = oracle_run(lattice, shape, 0.62, bc, steps, lid=lid, F=F, p0=p0, u0=u0)
    got = gpu_run(lattice, shape, 0.62, bc, steps, storage=storage, aa=aa, lid=lid, F=F,
                  p0=p0, u0=u0)
    eu, ep = errors(got, ref, 0.05)
    assert eu < TOL[storage] and ep < 10 * TOL[storage], (eu, ep)


@pytest.mark.parametrize("lattice,shape,bc", [("d3q19", (21, 18, 14), "cavity"),
                                              ("d2q9", (40, 31, 1), "periodic"),
                                              ("d3q27", (15, 13, 12), "channel")])
@pytest.mark.parametrize("storage", ["f64", "f32", "f16s"])
def test_compressible_parity(lattice, shape, bc, storage):
    Q, d = oracle.dims(lattice)
    nx, ny, nz = shape
    p0, u0 = W.random_smooth_state(nx, ny, nz, d, amp_u=0.04, amp_p=5e-3, seed=8)
    lid = (0.05, 0.0, 0.0) if bc != "periodic" else None
    F = W.fourier_force(nx, ny, nz, amplitude=1e-5, seed=6, dims=d)
    for steps in (40, 41):
        ref = oracle_run(lattice, shape, 0.7, bc, steps, lid=lid, F=F, p0=p0, u0=u0,
                         compressible=True)
        for aa in (False, True):
            got = gpu_run(lattice, shape, 0.7, bc, steps, storage=storage, aa=aa, lid=lid, F=F,
                          p0=p0, u0=u0, compressible=True)
            eu, ep = errors(got, ref, 0.05)
            assert eu < TOL[storage] and ep < 10 * TOL[storage], (steps, aa, eu, ep)


def test_rho0_and_unshifted_f32():
    shape = (23, 19, 11)
    p0, u0 = W.random_smooth_state(*shape, 3, amp_u=0.03, seed=4)
    ref = oracle_run("d3q19", shape, 0.75, "cavity", 30, lid=(0.05, 0, 0), p0=p0, u0=u0, rho0=1.3)
    for unshifted in (False, True):
        got = gpu_run("d3q19", shape, 0.75, "cavity", 30, storage="f32", lid=(0.05, 0, 0),
                      p0=p0, u0=u0, rho0=1.3, f32_unshifted=unshifted)
        eu, _ = errors(got, ref, 0.05, rho0=1.3)
        assert eu < 1e-5


# ---------------------------------------------------------------------------
# Edge cases


@pytest.mark.parametrize("lattice,shape,bc", [("d3q19", (1, 1, 1), "periodic"),
                                              ("d3q27", (1, 1, 1), "cavity"),
                                              ("d2q9", (1, 1, 1), "channel"),
                                              ("d3q19", (3, 3, 3), "cavity"),
                                              ("d3q27", (2, 3, 2), "periodic"),
                                              ("d2q9", (3, 3, 1), "cavity"),
                                              ("d3q19", (1, 16, 1), "channel"),
                                              ("d3q19", (2, 1, 5), "periodic")])
@pytest.mark.parametrize("aa", [False, True])
def test_tiny_grids(lattice, shape, bc, aa):
    Q, d = oracle.dims(lattice)
    p0, u0 = W.random_smooth_state(*shape, d, amp_u=0.03, seed=2)
    lid = (0.05, 0, 0.01) if bc != "periodic" else None
    F = np.full((d, int(np.prod(shape))), 1e-5, dtype=np.float32)
    for steps in (0, 1, 2, 7):
        ref = oracle_run(lattice, shape, 0.7, bc, steps, lid=lid, F=F, p0=p0, u0=u0)
        got = gpu_run(lattice, shape, 0.7, bc, steps, storage="f64", aa=aa, lid=lid, F=F,
                      p0=p0, u0=u0)
        eu, ep = errors(got, ref, 0.05)
        assert eu < 1e-12 and ep < 1e-11, (steps, eu, ep)


def test_poiseuille_on_gpu():
    """Channel with a body force at (tau - 1/2)^2 = 3/16: exact parabola."""
    ny, G = 14, 1e-6
    tau = 0.5 + math.sqrt(3 / 16)
    nu = W.viscosity(tau)
    F = np.zeros((3, ny), dtype=np.float32)
    F[0] = G
    _, u, _ = gpu_run("d3q19", (1, ny, 1), tau, "channel", int(25 * ny * ny / nu), storage="f64",
                      F=F)
    y = np.arange(ny)
    parabola = np.float64(np.float32(G)) / (2 * nu) * (y + 0.5) * (ny - 0.5 - y)
    assert np.abs(u[0] - parabola).max() < 1e-9 * parabola.max()


# ---------------------------------------------------------------------------
# Two-relaxation-time collision


TRT_CASES = [
    ("d3q19", (37, 29, 23), "cavity", 3 / 16),
    ("d3q27", (41, 9, 6), "channel", 1 / 4),
    ("d2q9", (45, 33, 1), "periodic", 1 / 12),
    ("d3q19", (300, 7, 5), "channel", 3 / 16),
]


@pytest.mark.parametrize("lattice,shape,bc,lam", TRT_CASES)
@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("aa", [False, True])
def test_trt_parity(lattice, shape, bc, lam, storage, aa):
    Q, d = oracle.dims(lattice)
    nx, ny, nz = shape
    p0, u0 = W.random_smooth_state(nx, ny, nz, d, amp_u=0.04, amp_p=2e-3, seed=23)
    lid = (0.08, 0.0, 0.02) if bc != "periodic" else None
    F = W.fourier_force(nx, ny, nz, amplitude=2e-5, seed=7, dims=d)
    steps = 61
    ref = oracle_run(lattice, shape, 0.62, bc, steps, lid=lid, F=F, p0=p0, u0=u0,
                     trt_lambda=lam)
    got = gpu_run(lattice, shape, 0.62, bc, steps, storage=storage, aa=aa, lid=lid, F=F,
                  p0=p0, u0=u0, trt_lambda=lam)
    eu, ep = errors(got, ref, 0.05)
    assert eu < TOL[storage] and ep < 10 * TOL[storage], (eu, ep)
    # and it is not BGK: the same run without TRT differs well above rounding
    if storage == "f64":
        bgk = oracle_run(lattice, shape, 0.62, bc, steps, lid=lid, F=F, p0=p0, u0=u0)
        assert errors(got, bgk, 0.05)[0] > 1e3 * TOL["f64"]


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_trt_poiseuille_on_gpu(storage):
    """TRT with Lambda = 3/16 at tau = 1.5: the exact parabola (BGK misses it by 3 %)."""
    ny, G, tau = 14, 1e-5, 1.5
    nu = W.viscosity(tau)
    F = np.zeros((3, ny), dtype=np.float32)
    F[0] = G
    _, u, _ = gpu_run("d3q19", (1, ny, 1), tau, "channel", int(30 * ny * ny / nu),
                      storage=storage, F=F, trt_lambda=3 / 16)
    y = np.arange(ny)
    parabola = np.float64(np.float32(G)) / (2 * nu) * (y + 0.5) * (ny - 0.5 - y)
    tol = 1e-9 if storage == "f64" else 1e-3
    assert np.abs(u[0] - parabola).max() < tol * parabola.max()


@pytest.mark.parametrize("storage", ["f64", "f32", "f16s", "bf16s"])
@pytest.mark.parametrize("bc", ["cavity", "channel"])
def test_trt_aa_equals_pull_bitwise(storage, bc):
    shape = (45, 26, 19)
    p0, u0 = W.random_smooth_state(*shape, 3, amp_u=0.04, seed=13)
    F = W.fourier_force(*shape, amplitude=2e-5, seed=3, dims=3)
    for steps in (10, 11):
        a = gpu_run("d3q19", shape, 0.6, bc, steps, storage=storage, aa=False, lid=(0.07, 0, 0),
                    p0=p0, u0=u0, F=F, trt_lambda=3 / 16)
        b = gpu_run("d3q19", shape, 0.6, bc, steps, storage=storage, aa=True, lid=(0.07, 0, 0),
                    p0=p0, u0=u0, F=F, trt_lambda=3 / 16)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), steps


@pytest.mark.parametrize("lattice,shape", [("d3q19", (520, 9, 7)), ("d3q27", (264, 7, 6)),
                                           ("d2q9", (304, 37, 1))])
@pytest.mark.parametrize("storage", ["f32", "f16s", "bf16s"])
def test_trt_kernel_variants_bitwise(lattice, shape, storage):
    """Plain and (16-bit) paired kernels give identical TRT results."""
    Q, d = oracle.dims(lattice)
    p0, u0 = W.random_smooth_state(*shape, d, amp_u=0.04, seed=45)
    F = W.fourier_force(*shape, amplitude=2e-5, seed=9, dims=d)
    kernels = ["plain"] + (["paired"] if storage != "f32" else [])
    from paper_2201_11330_b300.lbm import Lattice, LBMError
    lat = Lattice(lattice, *shape, 0.6, "cavity", storage=storage, trt_lambda=3 / 16)
    with pytest.raises(LBMError):  # 2: no such variant
        lat.set_kernel(2)
    for aa, steps in ((False, 9), (True, 9), (True, 10)):
        outs = [gpu_run(lattice, shape, 0.6, "cavity", steps, storage=storage, aa=aa,
                        lid=(0.07, 0.0, 0.01), p0=p0, u0=u0, F=F, trt_lambda=3 / 16,
                        kernel=k) for k in kernels]
        for k, o in zip(kernels[1:], outs[1:]):
            assert outs[0][2].kernel == "plain" and o[2].kernel == k
            assert np.array_equal(outs[0][0], o[0]) and np.array_equal(outs[0][1], o[1]), \
                (k, aa, steps)


# ---------------------------------------------------------------------------
# AA against the pull scheme: same arithmetic, bitwise equal


@pytest.mark.parametrize("storage", ["f64", "f32", "f16s", "bf16s"])
@pytest.mark.parametrize("bc", ["cavity", "periodic", "channel"])
def test_aa_equals_pull_bitwise(storage, bc):
    shape = (45, 26, 19)
    p0, u0 = W.random_smooth_state(*shape, 3, amp_u=0.04, seed=12)
    lid = (0.07, 0, 0) if bc != "periodic" else None
    for steps in (10, 11):
        a = gpu_run("d3q19", shape, 0.6, bc, steps, storage=storage, aa=False, lid=lid, p0=p0, u0=u0)
        b = gpu_run("d3q19", shape, 0.6, bc, steps, storage=storage, aa=True, lid=lid, p0=p0, u0=u0)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), steps


# ---------------------------------------------------------------------------
# Reductions, checkpoint / resume, failure detection


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("aa", [False, True])
def test_reduce_matches_fields(storage, aa):
    shape = (50, 40, 30)
    p0, u0 = W.random_smooth_state(*shape, 3, amp_u=0.05, seed=3)
    for steps in (12, 13):
        p, u, lat = gpu_run("d3q19", shape, 0.7, "cavity", steps, storage=storage, aa=aa,
                            lid=(0.1, 0, 0), p0=p0, u0=u0)
        r = lat.reduce()
        N = p.size
        tol = 1e-12 if storage == "f64" else 2e-6
        assert abs(r["mass"] - 3 * p.sum()) <= tol * N
        assert np.allclose(r["momentum"], u.sum(axis=1), atol=tol * N * 0.05, rtol=0)
        assert abs(r["kinetic_energy"] - 0.5 * (u * u).sum()) <= tol * 0.5 * (u * u).sum() + 1e-300
        assert abs(r["max_speed"] - np.sqrt((u * u).sum(axis=0)).max()) <= tol
        # closed cavity: mass is conserved
        assert abs(r["mass"] - 3 * p0.sum()) <= (1e-12 if storage == "f64" else 1e-6) * N


@pytest.mark.parametrize("aa", [False, True])
def test_checkpoint_resume_bitwise(aa):
    shape = (40, 33, 21)
    p0, u0 = W.random_smooth_state(*shape, 3, amp_u=0.05, seed=30)
    pa, ua, _ = gpu_run("d3q19", shape, 0.6, "cavity", 40, storage="f32", aa=aa,
                        lid=(0.1, 0, 0), p0=p0, u0=u0)
    _, _, lat = gpu_run("d3q19", shape, 0.6, "cavity", 15, storage="f32", aa=aa,
                        lid=(0.1, 0, 0), p0=p0, u0=u0)
    buf, step = lat.get_state()
    assert step == 15
    lat.step(7)  # wander off, then restore
    lat.set_state(buf, step)
    lat.step(25)
    pb, ub = lat.macroscopic()
    assert np.array_equal(pa, pb.cpu().numpy()) and np.array_equal(ua, ub.cpu().numpy())


def test_nan_is_reported_as_unstable():
    from paper_2201_11330_b300.lbm import LBMError, LBM_ERR_UNSTABLE
    shape = (16, 16, 16)
    p0, u0 = W.random_smooth_state(*shape, 3, seed=1)
    u0 = u0.copy()
    u0[0, 100] = np.nan
    _, _, lat = gpu_run("d3q19", shape, 0.7, "cavity", 3, storage="f32", p0=p0, u0=u0)
    with pytest.raises(LBMError) as ei:
        lat.reduce()
    assert ei.value.status == LBM_ERR_UNSTABLE


# ---------------------------------------------------------------------------
# Taylor-Green vortex 512 x 512, 5000 steps: oracle parity and analytic decay


@pytest.fixture(scope="module")
def tgv512_ref():
    n = 512
    p0, u0 = W.taylor_green_2d(n, n, 0.05)
    ref = oracle_run("d2q9", (n, n, 1), 0.8, "periodic", 5000, p0=p0, u0=u0)
    return p0, u0, ref


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_taylor_green_512(tgv512_ref, storage):
    p0, u0, ref = tgv512_ref
    n = 512
    got = gpu_run("d2q9", (n, n, 1), 0.8, "periodic", 5000, storage=storage, aa=True, p0=p0, u0=u0)
    eu, ep = errors(got, ref, 0.05)
    # the targets, max |du| / U: FP64 1e-12, FP32 1e-5
    assert eu < TOL[storage], eu
    # analytic decay of the amplitude, exp(-nu (kx^2 + ky^2) t)
    x, y, _ = W.grid(n, n, 1)
    k = 2 * math.pi / n
    mode = -np.cos(k * x) * np.sin(k * y)
    amp = (got[1][0] * mode).sum() / (mode * mode).sum() / 0.05
    assert abs(amp / math.exp(-W.taylor_green_rate(n, n, 0.8) * 5000) - 1) < 0.01
    # exact conservation on the periodic box
    lat = got[2]
    r = lat.reduce()
    assert abs(r["mass"] - 3 * p0.sum()) <= (1e-12 if storage == "f64" else 1e-6) * n * n


# ---------------------------------------------------------------------------
# FP32 momentum on a periodic box: the collision keeps the total momentum, so
# a drift measures arithmetic bias.  Every FP32 lattice weight rounds up by
# 7.45e-9 relative; applied as single floats they scaled the equilibrium's
# momentum by 1 + 7.45e-9 omega per collision, a drift of ~6e-5 over these
# 5000 steps (omega = 1.6).  With the weights as hi + lo pairs what is left
# is unbiased rounding noise.


@pytest.mark.parametrize("lattice,shape", [("d2q9", (256, 128, 1)), ("d3q19", (48, 40, 36)),
                                           ("d3q27", (40, 36, 32))])
@pytest.mark.parametrize("storage,aa,trt", [("f32", True, None), ("f32", False, None),
                                            ("f32", True, 3 / 16)])
def test_fp32_momentum_has_no_drift_on_periodic_box(lattice, shape, storage, aa, trt):
    from paper_2201_11330_b300.lbm import Lattice
    Q, d = oracle.dims(lattice)
    p0, u0 = W.random_smooth_state(*shape, d, amp_u=0.02, seed=61)
    u0 = u0 + np.array([0.04, -0.03, 0.02][:d]).reshape(d, 1)
    lat = Lattice(lattice, *shape, 0.625, "periodic", storage=storage, aa=aa, trt_lambda=trt)
    lat.init(torch.from_numpy(p0).cuda(), torch.from_numpy(np.ascontiguousarray(u0)).cuda())
    j0 = np.array(lat.reduce()["momentum"][:d])
    lat.step(5000)
    j1 = np.array(lat.reduce()["momentum"][:d])
    drift = np.abs(j1 - j0).max() / np.abs(j0).max()
    assert drift < 2e-6, drift


# ---------------------------------------------------------------------------
# The paired kernel (16-bit storage, two nodes per thread, shuffle realignment)
# against the plain kernel: bitwise equal, including row ends, warp and block
# edges, ragged blocks and 2-node rows.

def _variant_run(lattice, shape, bc, storage, aa, steps, kernel, force):
    from paper_2201_11330_b300.lbm import Lattice
    Q, d = oracle.dims(lattice)
    p0, u0 = W.random_smooth_state(*shape, d, amp_u=0.04, seed=44)
    lat = Lattice(lattice, *shape, 0.6, bc, storage=storage, aa=aa, kernel=kernel,
                  lid=(0.07, 0.0, 0.01) if bc != "periodic" else (0, 0, 0), has_force=force)
    if force:
        lat.set_force(torch.from_numpy(W.fourier_force(*shape, amplitude=2e-5, seed=8,
                                                       dims=d)).cuda())
    lat.init(torch.from_numpy(p0).cuda(), torch.from_numpy(u0).cuda())
    lat.step(steps)
    assert lat.kernel == kernel
    p, u = lat.macroscopic()
    return p.cpu().numpy(), u.cpu().numpy()


PAIRED_SHAPES = [("d3q19", (520, 9, 7)), ("d3q19", (66, 13, 11)), ("d3q27", (264, 7, 6)),
                 ("d2q9", (300, 37, 1)), ("d3q19", (2, 3, 3)), ("d3q27", (4, 1, 5)),
                 ("d2q9", (2, 5, 1)), ("d3q19", (258, 5, 4))]


@pytest.mark.parametrize("lattice,shape", PAIRED_SHAPES)
@pytest.mark.parametrize("storage", ["f16s", "bf16s"])
@pytest.mark.parametrize("bc", ["cavity", "periodic", "channel"])
def test_paired_equals_plain_bitwise(lattice, shape, storage, bc):
    for aa, steps, force in ((False, 9, True), (True, 9, False), (True, 10, True),
                             (True, 7, True)):
        a = _variant_run(lattice, shape, bc, storage, aa, steps, "plain", force)
        b = _variant_run(lattice, shape, bc, storage, aa, steps, "paired", force)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), (aa, steps, force)


@pytest.mark.parametrize("lattice,shape", [("d3q19", (66, 13, 11)), ("d3q27", (264, 7, 6)),
                                           ("d2q9", (300, 37, 1))])
@pytest.mark.parametrize("storage", ["f16s", "bf16s"])
def test_compressible_paired_equals_plain_bitwise(lattice, shape, storage):
    Q, d = oracle.dims(lattice)
    p0, u0 = W.random_smooth_state(*shape, d, amp_u=0.04, amp_p=5e-3, seed=46)
    F = W.fourier_force(*shape, amplitude=2e-5, seed=10, dims=d)
    for aa, steps in ((False, 9), (True, 9), (True, 10)):
        outs = [gpu_run(lattice, shape, 0.6, "cavity", steps, storage=storage, aa=aa,
                        lid=(0.07, 0.0, 0.01), p0=p0, u0=u0, F=F, compressible=True, kernel=k)
                for k in ("plain", "paired")]
        assert outs[0][2].kernel == "plain" and outs[1][2].kernel == "paired"
        assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


# ---------------------------------------------------------------------------
# lbm_step_reduce: the monitor fused into the last step kernel


@pytest.mark.parametrize("lattice,shape,bc", [("d3q19", (50, 40, 30), "cavity"),
                                              ("d3q27", (36, 21, 17), "channel"),
                                              ("d2q9", (130, 67, 1), "periodic"),
                                              ("d3q19", (301, 9, 7), "cavity")])
@pytest.mark.parametrize("storage", ["f64", "f32", "f16s", "bf16s"])
@pytest.mark.parametrize("aa", [False, True])
def test_step_reduce_matches_reduce(lattice, shape, bc, storage, aa):
    from paper_2201_11330_b300.lbm import Lattice
    Q, d = oracle.dims(lattice)
    p0, u0 = W.random_smooth_state(*shape, d, amp_u=0.05, seed=71)
    F = torch.from_numpy(W.fourier_force(*shape, amplitude=2e-5, seed=3, dims=d)).cuda()
    lid = (0.1, 0.0, 0.0) if bc != "periodic" else (0, 0, 0)
    outs = []
    for fused in (False, True):
        lat = Lattice(lattice, *shape, 0.7, bc, storage=storage, aa=aa, lid=lid, has_force=True)
        lat.set_force(F)
        lat.init(torch.from_numpy(p0).cuda(), torch.from_numpy(u0).cuda())
        for steps in (4, 5):
            if fused:
                r = lat.step_reduce(steps)
            else:
                lat.step(steps)
                r = lat.reduce()
            outs.append(r)
        outs.append(lat.macroscopic())
    N = int(np.prod(shape))
    # same state either way
    assert torch.equal(outs[2][0], outs[5][0]) and torch.equal(outs[2][1], outs[5][1])
    # same monitor values, up to the order of summation and the storage
    # rounding: lbm_reduce reads the stored (rounded) post-collision state,
    # the fused step uses the populations before they are stored
    tol = {"f64": 1e-12, "f32": 2e-6, "f16s": 1e-4, "bf16s": 1e-3}[storage]
    rel = {"f64": 1e-11, "f32": 2e-5, "f16s": 3e-3, "bf16s": 2e-2}[storage]
    for a, b in ((outs[0], outs[3]), (outs[1], outs[4])):
        assert abs(a["mass"] - b["mass"]) <= tol * N
        assert np.allclose(a["momentum"], b["momentum"], rtol=0, atol=tol * N * 0.05)
        assert abs(a["kinetic_energy"] - b["kinetic_energy"]) <= rel * a["kinetic_energy"]
        assert abs(a["max_speed"] - b["max_speed"]) <= rel * a["max_speed"]


# ---------------------------------------------------------------------------
# CUDA-graph replays of lbm_step: bit for bit the direct launches, also
# across parameter changes between calls


@pytest.mark.parametrize("storage", ["f32", "f16s", "f64"])
@pytest.mark.parametrize("aa", [False, True])
def test_graph_replays_equal_direct_launches(storage, aa):
    from paper_2201_11330_b300.lbm import Lattice
    shape = (37, 22, 19)
    p0, u0 = W.random_smooth_state(*shape, 3, amp_u=0.04, seed=51)
    F1 = torch.from_numpy(W.fourier_force(*shape, amplitude=2e-5, seed=1, dims=3)).cuda()
    F2 = torch.from_numpy(W.fourier_force(*shape, amplitude=2e-5, seed=2, dims=3)).cuda()
    outs = []
    for graph in (0, 4):
        lat = Lattice("d3q19", *shape, 0.6, "cavity", storage=storage, aa=aa, lid=(0.05, 0, 0),
                      has_force=True)
        lat.set_graph_steps(graph)
        lat.set_force(F1)
        lat.init(torch.from_numpy(p0).cuda(), torch.from_numpy(u0).cuda())
        lat.step(17)              # odd: the next call starts on an odd step
        lat.set_lid((0.07, 0, 0.01))
        lat.step(13)
        lat.set_force(F2)         # a new force pointer must reach the replays
        lat.step(21)
        r = lat.step_reduce(1)
        p, u = lat.macroscopic()
        outs.append((p.cpu().numpy(), u.cpu().numpy(), r["kinetic_energy"], lat.step_count))
    assert outs[0][3] == outs[1][3] == 52
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    assert outs[0][2] == outs[1][2]


def test_graph_replays_with_faces_and_obstacles():
    from paper_2201_11330_b300.lbm import Lattice
    nx, ny, nz = 40, 18, 12
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    sol = ((x - 12) ** 2 + (y - 9) ** 2 + (z - 6) ** 2 <= 9).astype(np.uint8)
    inl = torch.zeros((3, ny * nz), device="cuda")
    inl[0] = 0.04
    outs = []
    for graph in (0, 6):
        lat = Lattice("d3q27", nx, ny, nz, 0.6, ["inlet", "outflow", "symmetry", "symmetry",
                                                 "periodic", "periodic"],
                      storage="f32", obstacles=True)
        lat.set_graph_steps(graph)
        lat.set_geometry(torch.from_numpy(sol.ravel()).cuda())
        lat.set_inlet(inl)
        lat.init()
        lat.step(40)
        f = lat.step_force(1)
        p, u = lat.macroscopic()
        outs.append((p.cpu().numpy(), u.cpu().numpy(), f))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    assert outs[0][2] == outs[1][2]


@pytest.mark.parametrize("storage", ["f32", "f16s"])
def test_init_from_fp32_fields(storage):
    """lbm_init_f32 equals lbm_init on the same (FP32-representable) fields."""
    from paper_2201_11330_b300.lbm import Lattice
    shape = (33, 20, 17)
    p0, u0 = W.random_smooth_state(*shape, 3, amp_u=0.04, seed=52)
    p0 = p0.astype(np.float32).astype(np.float64)
    u0 = u0.astype(np.float32).astype(np.float64)
    outs = []
    for dt in (torch.float64, torch.float32):
        lat = Lattice("d3q19", *shape, 0.6, "cavity", storage=storage, aa=True, lid=(0.05, 0, 0))
        lat.init(torch.from_numpy(p0).to("cuda", dt), torch.from_numpy(u0).to("cuda", dt))
        lat.step(5)
        p, u = lat.macroscopic()
        outs.append((p.cpu().numpy(), u.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
