"""Storage precision and full-size checks of the D3Q19 lid-driven cavity.

* 64^3 copy of the Re = 1000 cavity (tau from Re at 64 nodes), 2000 steps,
  AA single lattice: FP32, FP16-shifted and BF16-shifted storage against the
  FP64 oracle, error per field.
* 512^3 at the benchmark's launch configuration: properties that hold at any
  size (mass conservation, z-mirror symmetry), AA == pull scheme, and the
  nodes near the lid, walls and corners after a few steps against small
  oracle boxes that contain their whole domain of dependence.
"""
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


def _run(shape, tau, steps, storage, aa, lid=(0.1, 0.0, 0.0)):
    from paper_2201_11330_b300.lbm import Lattice
    lat = Lattice("d3q19", *shape, tau, "cavity", storage=storage, aa=aa, lid=lid)
    lat.init()
    lat.step(steps)
    return lat


@pytest.fixture(scope="module")
def cav64_ref():
    c = W.cavity_params(64, 1000.0, 0.1)
    p, u = oracle.run("d3q19", 64, 64, 64, c["tau"], "cavity", 2000, lid=c["lid"])
    return c, p, u


# velocity bound per storage (max norm over the box, relative to U): the
# targets of FP32 storage, 1e-5, and of FP16-shifted storage, 2e-3; BF16
# keeps 8 mantissa bits and has no target (its bound is a regression check).
@pytest.mark.parametrize("storage,tol_u", [("f32", 1e-5), ("f16s", 2e-3), ("bf16s", 5e-2)])
def test_cavity64_storage_error(cav64_ref, storage, tol_u, record_property):
    c, pr, ur = cav64_ref
    lat = _run((64, 64, 64), c["tau"], 2000, storage, aa=True)
    p, u = lat.macroscopic()
    p, u = p.cpu().numpy(), u.cpu().numpy()
    U = 0.1
    eu = np.abs(u - ur).max() / U
    ep = np.abs(p - pr).max() / (U * U)
    eu_rms = np.sqrt(((u - ur) ** 2).sum(axis=0).mean()) / U
    record_property("velocity_error", float(eu))
    record_property("velocity_error_rms", float(eu_rms))
    record_property("pressure_error", float(ep))
    print(f"\n[cavity64 Re=1000 2000 steps] {storage}: max|du|/U = {eu:.3e}, "
          f"rms|du|/U = {eu_rms:.3e}, max|dp|/(rho0 U^2) = {ep:.3e}")
    assert eu < tol_u


def _big():
    return 512, W.cavity_params(512, 1000.0, 0.1)


@pytest.mark.parametrize("storage,trt", [("f32", None), ("f16s", None), ("bf16s", None),
                                         ("f32", 3 / 16)])
def test_full_size_properties(storage, trt):
    from paper_2201_11330_b300.lbm import Lattice
    n, c = _big()
    lat = Lattice("d3q19", n, n, n, c["tau"], "cavity", storage=storage, aa=True, lid=c["lid"],
                  trt_lambda=trt)
    lat.init()
    lat.step(300)
    r = lat.reduce()
    N = n ** 3
    assert abs(r["mass"] - N) < {"f32": 1e-6, "f16s": 1e-4, "bf16s": 1e-3}[storage] * N
    assert 0.05 < r["max_speed"] < 0.2
    _, u = lat.macroscopic(torch.float32)
    uz = u[2].view(n, n, n)
    ux = u[0].view(n, n, n)
    tol = {"f32": 1e-6, "f16s": 2e-4, "bf16s": 2e-3}[storage]
    assert (uz + uz.flip(0)).abs().max().item() < tol
    assert (ux - ux.flip(0)).abs().max().item() < tol
    del lat, u, uz, ux
    torch.cuda.empty_cache()


def test_full_size_aa_equals_pull():
    n, c = _big()
    for steps in (10, 11):
        a = _run((n, n, n), c["tau"], steps, "f32", aa=True)
        ua = a.macroscopic(torch.float32)[1]
        del a
        b = _run((n, n, n), c["tau"], steps, "f32", aa=False)
        ub = b.macroscopic(torch.float32)[1]
        del b
        assert torch.equal(ua, ub)
        del ua, ub
        torch.cuda.empty_cache()


@pytest.mark.parametrize("steps", [6, 7])
@pytest.mark.parametrize("storage,tol", [("f32", 1e-5), ("f16s", 2e-3)])
def test_full_size_light_cone_samples(steps, storage, tol):
    """After k steps from rest, a node depends only on nodes within k of it.
    A 16^3 oracle cavity has the same walls and lid within k = 6, 7 of its
    own corner region, and a 1 x 16 x 1 oracle channel (periodic x, z) has
    the same lid within reach of the 512^3 lid's interior nodes."""
    n, c = _big()
    lat = _run((n, n, n), c["tau"], steps, storage, aa=True)
    _, u = lat.macroscopic(torch.float64)
    u = u.view(3, n, n, n).cpu().numpy()  # (component, z, y, x)
    U = 0.1
    m = 16
    _, uo = oracle.run("d3q19", m, m, m, c["tau"], "cavity", steps, lid=c["lid"])
    uo = uo.reshape(3, m, m, m)
    r = 8  # corner region [0, 8] is more than k from the small box's far walls
    lo, hi = slice(0, r + 1), slice(m - r - 1, m)
    # bottom corner and lid corner, both x/z corners
    for zs in (lo,):
        for ys_small, ys_big in ((lo, slice(0, r + 1)), (hi, slice(n - r - 1, n))):
            for xs_small, xs_big in ((lo, slice(0, r + 1)), (hi, slice(n - r - 1, n))):
                d = np.abs(u[:, zs, ys_big, xs_big] - uo[:, zs, ys_small, xs_small]).max() / U
                assert d < tol, (ys_big, xs_big, d)
    _, uc = oracle.run("d3q19", 1, m, 1, c["tau"], "channel", steps, lid=c["lid"])
    band = u[:, 200:300:17, n - m:, 200:300:13]  # interior of the lid, top m rows
    d = np.abs(band - uc[:, None, :, None]).max() / U
    assert d < tol
    assert np.abs(uc[0]).max() > 1e-3  # the lid has started to drive the flow


# ---------------------------------------------------------------------------
# D3Q27 768^3, FP16-shifted AA storage (the bench's D3Q27 launch configuration)


def _d3q27_768(steps):
    from paper_2201_11330_b300.lbm import Lattice
    n = 768
    c = W.cavity_params(n, 2000.0, 0.1)
    lat = Lattice("d3q27", n, n, n, c["tau"], "cavity", storage="f16s", aa=True, lid=c["lid"])
    lat.init()
    lat.step(steps)
    return n, c, lat


def test_d3q27_768_properties():
    n, c, lat = _d3q27_768(120)
    r = lat.reduce()
    N = n ** 3
    assert abs(r["mass"] - N) < 1e-4 * N
    assert 0.05 < r["max_speed"] < 0.2
    _, u = lat.macroscopic(torch.float32)
    del lat
    torch.cuda.empty_cache()
    u = u.view(3, n, n, n)
    assert (u[2] + u[2].flip(0)).abs().max().item() < 2e-4  # z-mirror symmetry
    assert (u[0] - u[0].flip(0)).abs().max().item() < 2e-4
    del u
    torch.cuda.empty_cache()


@pytest.mark.parametrize("steps", [6, 7])
def test_d3q27_768_light_cone_samples(steps):
    """After k steps from rest a node depends only on nodes within k of it: the
    768^3 cavity's corner regions equal a 16^3 oracle cavity's, and its lid
    interior equals a 1 x 16 x 1 oracle channel under the same lid."""
    n, c, lat = _d3q27_768(steps)
    _, u = lat.macroscopic(torch.float32)
    del lat
    u = u.view(3, n, n, n)
    U, m, r = 0.1, 16, 8
    _, uo = oracle.run("d3q27", m, m, m, c["tau"], "cavity", steps, lid=c["lid"])
    uo = uo.reshape(3, m, m, m)
    for ys_small, ys_big in ((slice(0, r + 1), slice(0, r + 1)), (slice(m - r - 1, m),
                                                                   slice(n - r - 1, n))):
        for xs_small, xs_big in ((slice(0, r + 1), slice(0, r + 1)), (slice(m - r - 1, m),
                                                                       slice(n - r - 1, n))):
            big = u[:, 0:r + 1, ys_big, xs_big].double().cpu().numpy()
            d = np.abs(big - uo[:, 0:r + 1, ys_small, xs_small]).max() / U
            assert d < 2e-3, (ys_big, xs_big, d)
    _, uc = oracle.run("d3q27", 1, m, 1, c["tau"], "channel", steps, lid=c["lid"])
    band = u[:, 300:460:23, n - m:, 300:460:19].double().cpu().numpy()
    assert np.abs(band - uc[:, None, :, None]).max() / U < 2e-3
    assert np.abs(uc[0]).max() > 1e-3
    del u
    torch.cuda.empty_cache()


def test_near_maximum_size_d3q19_1280():
    """1280^3 = 2,097,152,000 nodes, just under the 2^31 node-index limit
    (D3Q19 FP16-shifted AA, 80 GB): the far corner of the box, where the
    32-bit node index and the 64-bit slot offsets are largest, and the near
    corner both equal a 16^3 oracle cavity's after 6 steps; mass is kept."""
    from paper_2201_11330_b300.lbm import Lattice
    n = 1280
    assert n ** 3 < 2 ** 31
    c = W.cavity_params(n, 1000.0, 0.1)
    lat = Lattice("d3q19", n, n, n, c["tau"], "cavity", storage="f16s", aa=True, lid=c["lid"])
    lat.init()
    lat.step(6)
    r = lat.reduce()
    assert abs(r["mass"] - n ** 3) < 1e-4 * n ** 3
    _, u = lat.macroscopic(torch.float32)
    del lat
    torch.cuda.empty_cache()
    u = u.view(3, n, n, n)
    m, r8 = 16, 8
    _, uo = oracle.run("d3q19", m, m, m, c["tau"], "cavity", 6, lid=c["lid"])
    uo = uo.reshape(3, m, m, m)
    lo, hi = slice(0, r8 + 1), slice(m - r8 - 1, m)
    near = u[:, 0:r8 + 1, 0:r8 + 1, 0:r8 + 1].double().cpu().numpy()
    far = u[:, n - r8 - 1:, n - r8 - 1:, n - r8 - 1:].double().cpu().numpy()
    assert np.abs(near - uo[:, lo, lo, lo]).max() / 0.1 < 2e-3
    assert np.abs(far - uo[:, hi, hi, hi]).max() / 0.1 < 2e-3
    assert np.abs(uo[:, hi, hi, hi]).max() > 1e-3  # the lid corner is moving
    del u
    torch.cuda.empty_cache()
