"""The general step kernel (per-face boundaries, solid obstacles, momentum
exchange) against the FP64 oracle, through the C ABI.

Cases follow the paper's Sec. 4-5 workloads at oracle scale: a channel with a
parabolic velocity inlet, a pressure outlet and a cylinder (D2Q9); flow past
a sphere between symmetry planes with periodic top/bottom (D3Q27); a cavity
with an obstacle block; every face type on one ragged box.  Boxes are ragged
(not multiples of the block size) and obstacles touch faces.
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


TOL_U = {"f64": 1e-12, "f32": 1e-5, "f16s": 2e-3, "bf16s": 5e-2}


def cylinder(nx, ny, cx, cy, r):
    x, y = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    return ((x - cx) ** 2 + (y - cy) ** 2 <= r * r).astype(np.uint8)


def sphere(nx, ny, nz, c, r):
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return ((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2 <= r * r).astype(np.uint8)


def parabola(n, umax):
    s = np.arange(n)
    return umax * (s + 0.5) * (n - 0.5 - s) / (n / 2) ** 2


def run_pair(lattice, shape, tau, faces, steps, *, storage, solid=None, inlet=None, lid=None,
             F=None, p0=None, u0=None, trt_lambda=None, compressible=False, p_outflow=1 / 3,
             force_out=False, bc=None):
    """(gpu p, gpu u, gpu force), (oracle p, oracle u, oracle force)."""
    from paper_2201_11330_b300.lbm import Lattice
    nx, ny, nz = shape
    lat = Lattice(lattice, nx, ny, nz, tau, bc or faces, storage=storage,
                  obstacles=solid is not None, lid=lid or (0, 0, 0), has_force=F is not None,
                  trt_lambda=trt_lambda, compressible=compressible, p_outflow=p_outflow)
    if solid is not None:
        lat.set_geometry(torch.from_numpy(np.ascontiguousarray(solid).ravel()).cuda())
    if inlet is not None:
        lat.set_inlet(torch.from_numpy(np.ascontiguousarray(inlet, np.float32)).cuda())
    if F is not None:
        lat.set_force(torch.from_numpy(np.ascontiguousarray(F, np.float32)).cuda())
    lat.init(None if p0 is None else torch.from_numpy(p0).cuda(),
             None if u0 is None else torch.from_numpy(np.ascontiguousarray(u0)).cuda())
    fg = None
    if force_out:
        lat.step(steps - 1)
        fg = np.array(lat.step_force(1))
    else:
        lat.step(steps)
    p, u = lat.macroscopic()
    got = (p.cpu().numpy(), u.cpu().numpy(), fg, lat)
    ref = oracle.run(lattice, nx, ny, nz, tau, bc or faces, steps, lid=lid,
                     F=None if F is None else np.asarray(F, np.float32).astype(np.float64),
                     p0=p0, u0=None if u0 is None else np.ascontiguousarray(u0).ravel(),
                     solid=solid, inlet=None if inlet is None else
                     np.asarray(inlet, np.float32).astype(np.float64),
                     trt_lambda=trt_lambda, compressible=compressible, p_outflow=p_outflow,
                     want_force=True)
    return got, ref


def field_errors(got, ref, uref):
    eu = np.abs(got[1] - ref[1]).max() / uref
    ep = np.abs(got[0] - ref[0]).max() / (uref * uref)
    return eu, ep


CHANNEL2D = ["inlet", "outflow", "wall", "wall", "periodic", "periodic"]
SPHERE3D = ["inlet", "outflow", "symmetry", "symmetry", "periodic", "periodic"]
MIXED3D = ["outflow", "inlet", "symmetry", "wall", "symmetry", "symmetry"]


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_cylinder_channel_2d(storage):
    nx, ny = 301, 67
    U = 0.06
    inl = np.zeros((2, ny))
    inl[0] = parabola(ny, U)
    sol = cylinder(nx, ny, 40.3, 33.7, 8.2)
    got, ref = run_pair("d2q9", (nx, ny, 1), 0.56, CHANNEL2D, 300, storage=storage, solid=sol,
                        inlet=inl, force_out=True)
    eu, ep = field_errors(got, ref, U)
    assert eu < TOL_U[storage] and ep < 10 * TOL_U[storage], (eu, ep)
    fscale = np.abs(ref[2]).max()
    assert fscale > 0.01
    assert np.abs(got[2] - ref[2]).max() < (1e-12 if storage == "f64" else 1e-4) * fscale
    # solid nodes report zero
    s = sol.ravel() != 0
    assert np.all(got[0][s] == 0) and np.all(got[1][:, s] == 0)


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_sphere_between_symmetry_planes_3d(storage):
    nx, ny, nz = 45, 21, 17
    U = 0.05
    inl = np.zeros((3, ny * nz))
    inl[0] = U
    sol = sphere(nx, ny, nz, (14.2, 10.0, 8.0), 4.3)
    u0 = np.zeros((3, nx * ny * nz))
    u0[0] = U
    u0[:, sol.ravel() != 0] = 0
    got, ref = run_pair("d3q27", (nx, ny, nz), 0.58, SPHERE3D, 120, storage=storage, solid=sol,
                        inlet=inl, u0=u0, force_out=True)
    eu, ep = field_errors(got, ref, U)
    assert eu < TOL_U[storage] and ep < 10 * TOL_U[storage], (eu, ep)
    fscale = np.abs(ref[2]).max()
    assert np.abs(got[2] - ref[2]).max() < (1e-12 if storage == "f64" else 1e-4) * fscale


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("lattice", ["d3q19", "d3q27"])
def test_every_face_type_with_obstacles(lattice, storage):
    """Outflow on -x, inlet on +x (flow towards -x), symmetry on -y, moving
    wall on +y, symmetry on both z faces; obstacles touching the -y and +x
    faces; random initial state, Fourier force."""
    nx, ny, nz = 37, 19, 13
    p0, u0 = W.random_smooth_state(nx, ny, nz, 3, amp_u=0.03, amp_p=2e-3, seed=31)
    sol = np.zeros((nz, ny, nx), np.uint8)
    sol[3:7, 0:4, 10:15] = 1
    sol[5:9, 8:12, 33:37] = 1
    u0[:, sol.ravel() != 0] = 0
    inl = np.zeros((3, ny * nz))
    y, z = np.meshgrid(np.arange(ny), np.arange(nz), indexing="xy")
    inl[0] = (-0.04 * (1 + 0.2 * np.sin(2 * np.pi * z / nz)) * (y + 0.5) / ny).ravel()
    inl[1] = 0.005
    F = W.fourier_force(nx, ny, nz, amplitude=2e-5, seed=12, dims=3)
    got, ref = run_pair(lattice, (nx, ny, nz), 0.62, MIXED3D, 61, storage=storage, solid=sol,
                        inlet=inl, lid=(0.05, 0.0, 0.01), F=F, p0=p0, u0=u0, force_out=True,
                        p_outflow=0.335)
    eu, ep = field_errors(got, ref, 0.05)
    assert eu < TOL_U[storage] and ep < 10 * TOL_U[storage], (eu, ep)
    fscale = np.abs(ref[2]).max()
    assert np.abs(got[2] - ref[2]).max() < (1e-12 if storage == "f64" else 1e-4) * fscale


@pytest.mark.parametrize("model", ["trt", "compressible"])
def test_models_with_faces_and_obstacles(model):
    nx, ny, nz = 33, 15, 11
    p0, u0 = W.random_smooth_state(nx, ny, nz, 3, amp_u=0.03, amp_p=3e-3, seed=32)
    sol = sphere(nx, ny, nz, (12.0, 7.0, 5.0), 3.1)
    u0[:, sol.ravel() != 0] = 0
    inl = np.zeros((3, ny * nz))
    inl[0] = 0.04
    kw = {"trt_lambda": 3 / 16} if model == "trt" else {"compressible": True}
    for storage in ("f64", "f32"):
        got, ref = run_pair("d3q19", (nx, ny, nz), 0.6, SPHERE3D, 40, storage=storage, solid=sol,
                            inlet=inl, p0=p0, u0=u0, **kw)
        eu, ep = field_errors(got, ref, 0.05)
        assert eu < TOL_U[storage] and ep < 10 * TOL_U[storage], (storage, eu, ep)


@pytest.mark.parametrize("storage", ["f64", "f32", "f16s", "bf16s"])
def test_cavity_with_obstacle_and_reduce(storage):
    """A named box type with obstacles: the monitor sums run over fluid nodes."""
    nx, ny, nz = 40, 28, 22
    sol = np.zeros((nz, ny, nx), np.uint8)
    sol[8:14, 10:16, 12:20] = 1
    got, ref = run_pair("d3q19", (nx, ny, nz), 0.6, None, 50, storage=storage, solid=sol,
                        lid=(0.08, 0, 0), bc="cavity")
    eu, _ = field_errors(got, ref, 0.08)
    assert eu < TOL_U[storage], eu
    lat = got[3]
    r = lat.reduce()
    fl = sol.ravel() == 0
    mass = (3 * ref[0][fl]).sum()
    assert abs(r["mass"] - mass) < (1e-9 if storage == "f64" else 1e-3) * fl.sum() ** 0.5 + 1e-9
    # closed box: the fluid's mass is kept (to the storage's rounding)
    mtol = {"f64": 1e-12, "f32": 1e-6, "f16s": 2e-6, "bf16s": 2e-5}[storage]
    assert abs(r["mass"] - fl.sum()) < mtol * fl.sum()
    s = lat.step_reduce(1)
    assert abs(s["mass"] - fl.sum()) < mtol * fl.sum()


@pytest.mark.parametrize("storage", ["f64", "f32", "f16s", "bf16s"])
@pytest.mark.parametrize("named,faces", [
    ("cavity", ["wall"] * 6),
    ("channel", ["periodic", "periodic", "wall", "wall", "periodic", "periodic"]),
    ("periodic", ["periodic"] * 6)])
def test_general_kernel_equals_named_boxes_bitwise(storage, named, faces):
    """The named box types through the general kernel give exactly the plain
    kernel's result (same gathers, same collision)."""
    from paper_2201_11330_b300.lbm import Lattice
    shape = (45, 26, 19)
    p0, u0 = W.random_smooth_state(*shape, 3, amp_u=0.04, seed=14)
    F = torch.from_numpy(W.fourier_force(*shape, amplitude=2e-5, seed=4, dims=3)).cuda()
    outs = []
    for bc in (named, faces):
        lat = Lattice("d3q19", *shape, 0.6, bc, storage=storage, lid=(0.07, 0, 0.01),
                      has_force=True, kernel="plain" if bc == named else "auto")
        lat.set_force(F)
        lat.init(torch.from_numpy(p0).cuda(), torch.from_numpy(u0).cuda())
        lat.step(9)
        p, u = lat.macroscopic()
        outs.append((p.cpu().numpy(), u.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_obstacle_momentum_balance_on_gpu():
    """Periodic box, body force, obstacle: per step the fluid's momentum
    changes by the body force minus the momentum-exchange force (FP64)."""
    from paper_2201_11330_b300.lbm import Lattice
    nx, ny, nz = 40, 30, 24
    sol = sphere(nx, ny, nz, (20.0, 15.0, 12.0), 5.5)
    fl = sol.ravel() == 0
    Fb = np.zeros((3, nx * ny * nz), np.float32)
    Fb[0] = 1e-5
    Fb[:, ~fl] = 0
    lat = Lattice("d3q19", nx, ny, nz, 0.8, "periodic", storage="f64", obstacles=True,
                  has_force=True)
    lat.set_geometry(torch.from_numpy(sol.ravel()).cuda())
    lat.set_force(torch.from_numpy(Fb).cuda())
    lat.init()
    lat.step(200)
    m0 = np.array(lat.reduce()["momentum"])
    f = np.array(lat.step_force(1))
    m1 = np.array(lat.reduce()["momentum"])
    want = Fb.astype(np.float64)[:, fl].sum(axis=1) - f
    assert np.abs((m1 - m0) - want).max() < 1e-12 * np.abs(f).max() + 1e-13
    assert f[0] > 0.1 * Fb[0, fl].sum()  # the obstacle holds a good part of the load


def test_geometry_argument_checks():
    from paper_2201_11330_b300 import lbm
    from paper_2201_11330_b300.lbm import Lattice, LBMError
    with pytest.raises(LBMError):  # AA with per-face boundaries
        Lattice("d3q19", 8, 8, 8, 0.6, SPHERE3D, aa=True)
    with pytest.raises(LBMError):  # unpaired periodic face
        Lattice("d3q19", 8, 8, 8, 0.6, ["periodic", "wall"] + ["periodic"] * 4)
    with pytest.raises(LBMError):  # two inlets
        Lattice("d3q19", 8, 8, 8, 0.6, ["inlet", "inlet"] + ["periodic"] * 4)
    lat = Lattice("d3q19", 8, 8, 8, 0.6, "cavity")
    with pytest.raises(LBMError) as e:  # obstacles were not reserved
        lat.set_geometry(torch.zeros(512, dtype=torch.uint8, device="cuda"))
    assert e.value.status == lbm.LBM_ERR_STATE
    with pytest.raises(LBMError):  # no inlet face
        lat.set_inlet(torch.zeros((3, 64), device="cuda"))
    lat = Lattice("d3q19", 8, 8, 8, 0.6, "cavity", obstacles=True)
    lat.set_geometry(torch.zeros(512, dtype=torch.uint8, device="cuda"))
    with pytest.raises(LBMError):  # geometry invalidates the state
        lat.step(1)
    lat.init()
    with pytest.raises(LBMError):  # 2: no such variant
        lat.set_kernel(2)
    with pytest.raises(LBMError):  # paired needs 16-bit storage
        lat.set_kernel("paired")
    assert lat.kernel == "plain"
    lat16 = Lattice("d3q19", 8, 8, 8, 0.6, "cavity", storage="f16s", obstacles=True)
    assert lat16.kernel == "paired"
    lat16.set_kernel("plain")
    assert lat16.kernel == "plain"


@pytest.fixture(scope="module")
def sphere_full():
    """The Sec. 5-6 sphere case at the paper's size and its FP64 oracle run
    (12 steps): D3Q27, 512 x 128 x 128, sphere of radius 8 centred at
    (64, 64, 64), inlet on the back face (-x), outflow on the front (+x),
    symmetry planes left/right (y), periodic top/bottom (z)."""
    nx, ny, nz = 512, 128, 128
    U = 0.05
    sol = sphere(nx, ny, nz, (64, 64, 64), 8)
    inl = np.zeros((3, ny * nz), np.float32)  # the GPU reads the inlet in FP32
    inl[0] = U
    u0 = np.zeros((3, nx * ny * nz))
    u0[0] = U
    u0[:, sol.ravel() != 0] = 0
    ref = oracle.run("d3q27", nx, ny, nz, 0.53, SPHERE3D, 12, u0=u0.ravel(), solid=sol,
                     inlet=inl.astype(np.float64), want_force=True)
    return (nx, ny, nz), U, sol, inl, u0, ref


@pytest.mark.parametrize("storage", ["f64", "f32", "f16s"])
def test_sphere_512x128x128_matches_oracle_at_point_a(sphere_full, storage):
    """Sec. 5 "validation of GPU offloading" at the paper's own size, in the
    bench's launch configuration: the GPU against the FP64 oracle on the host,
    over the whole field, at point A = (72, 72, 72), and for the drag."""
    from paper_2201_11330_b300.lbm import Lattice
    (nx, ny, nz), U, sol, inl, u0, ref = sphere_full
    lat = Lattice("d3q27", nx, ny, nz, 0.53, SPHERE3D, storage=storage, obstacles=True)
    lat.set_geometry(torch.from_numpy(sol.ravel()).cuda())
    lat.set_inlet(torch.from_numpy(inl).cuda())
    lat.init(None, torch.from_numpy(u0).cuda())
    lat.step(11)
    f = np.array(lat.step_force(1))
    p, u = lat.macroscopic()
    got = (p.cpu().numpy(), u.cpu().numpy())
    eu, ep = field_errors(got, ref, U)
    tol = {"f64": 1e-12, "f32": 1e-5, "f16s": 2e-3}[storage]
    assert eu < tol and ep < 10 * tol, (eu, ep)
    a = 72 + nx * (72 + ny * 72)
    assert np.abs(got[1][:, a] - ref[1][:, a]).max() < max(1e-15, tol * U)
    assert np.abs(got[1][:, a] - U * np.array([1, 0, 0])).max() > 1e-6  # A sees the sphere
    ftol = {"f64": 1e-12, "f32": 1e-4, "f16s": 2e-2}[storage]
    assert np.abs(f - ref[2]).max() < ftol * np.abs(ref[2]).max()
    del lat, p, u
    torch.cuda.empty_cache()


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("lattice,shape,faces,obst", [
    ("d3q19", (29, 23, 17), ["nodal"] * 6, True),
    ("d3q27", (25, 19, 14), ["inlet", "outflow", "nodal", "nodal", "symmetry", "nodal"], True),
    ("d2q9", (61, 37, 1), ["nodal", "nodal", "nodal", "nodal", "periodic", "periodic"], False),
])
def test_nodal_bounce_back_parity(lattice, shape, faces, obst, storage):
    """The paper's nodal bounce-back faces (with a lid on +y, obstacles
    touching nodal faces, an inlet and an outflow) against the oracle."""
    Q, d = oracle.dims(lattice)
    nx, ny, nz = shape
    p0, u0 = W.random_smooth_state(nx, ny, nz, d, amp_u=0.03, amp_p=2e-3, seed=33)
    sol = None
    if obst:
        sol = np.zeros((nz, ny, nx), np.uint8)
        sol[2:6, 0:3, 8:12] = 1
        sol[nz // 2:nz // 2 + 3, 9:12, 0:4] = 1
        u0[:, sol.ravel() != 0] = 0
    inl = None
    if "inlet" in faces:
        inl = np.zeros((d, ny * nz))
        inl[0] = 0.03
    F = W.fourier_force(nx, ny, nz, amplitude=2e-5, seed=13, dims=d)
    got, ref = run_pair(lattice, shape, 0.63, faces, 45, storage=storage, solid=sol, inlet=inl,
                        lid=(0.06, 0.0, 0.01), F=F, p0=p0, u0=u0, force_out=obst)
    eu, ep = field_errors(got, ref, 0.05)
    assert eu < TOL_U[storage] and ep < 10 * TOL_U[storage], (eu, ep)
    if obst:
        assert np.abs(got[2] - ref[2]).max() < (1e-12 if storage == "f64" else 1e-4) * \
            np.abs(ref[2]).max()


def test_nodal_couette_on_gpu():
    """Nodal walls put the Couette profile's ends on the wall nodes (FP64)."""
    from paper_2201_11330_b300.lbm import Lattice
    ny, U, tau = 12, 0.02, 1.3
    nu = W.viscosity(tau)
    lat = Lattice("d3q19", 1, ny, 1, tau, ["periodic", "periodic", "nodal", "nodal", "periodic",
                                           "periodic"], storage="f64", lid=(U, 0, 0))
    lat.init()
    lat.step(int(30 * ny * ny / nu))
    _, u = lat.macroscopic()
    assert np.abs(u[0].cpu().numpy() - U * np.arange(ny) / (ny - 1)).max() < 1e-10 * U


@pytest.mark.parametrize("storage", ["f16s", "bf16s"])
def test_paired_and_plain_bulk_agree_with_faces_and_obstacles(storage):
    """With 16-bit storage the nodes away from open faces and obstacles run
    on the paired kernel; forcing the plain kernel gives the same bits."""
    from paper_2201_11330_b300.lbm import Lattice
    nx, ny, nz = 58, 21, 15
    p0, u0 = W.random_smooth_state(nx, ny, nz, 3, amp_u=0.03, seed=41)
    sol = sphere(nx, ny, nz, (20.0, 10.0, 7.0), 3.2)
    u0[:, sol.ravel() != 0] = 0
    inl = torch.zeros((3, ny * nz), device="cuda")
    inl[0] = 0.04
    outs = []
    for kernel in ("auto", "plain"):
        lat = Lattice("d3q19", nx, ny, nz, 0.6, ["inlet", "outflow", "wall", "symmetry",
                                                 "periodic", "periodic"],
                      storage=storage, obstacles=True, lid=(0.05, 0, 0))
        lat.set_kernel(kernel)
        lat.set_geometry(torch.from_numpy(sol.ravel()).cuda())
        lat.set_inlet(inl)
        lat.init(torch.from_numpy(p0).cuda(), torch.from_numpy(u0).cuda())
        lat.step(9)
        f = lat.step_force(1)
        r = lat.step_reduce(1)
        p, u = lat.macroscopic()
        outs.append((p.cpu().numpy(), u.cpu().numpy(), f, r["mass"]))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    # same link terms, summed in other block groupings (FP32 partial sums)
    assert np.allclose(outs[0][2], outs[1][2], rtol=2e-5, atol=1e-9)
    assert abs(outs[0][3] - outs[1][3]) < 1e-6 * nx * ny * nz


# The node list takes the first / last 32 bytes of every row next to an open x
# face (4 FP64, 8 FP32, 16 FP16 nodes); row lengths below, at and above twice
# that, so that rows are wholly listed, split, or mostly plain.
@pytest.mark.parametrize("storage,nx", [("f64", 3), ("f64", 8), ("f64", 9), ("f64", 17),
                                        ("f32", 15), ("f32", 16), ("f32", 17), ("f32", 41),
                                        ("f16s", 16), ("f16s", 32), ("f16s", 34),
                                        ("f16s", 66), ("f16s", 33)])
def test_open_x_faces_for_row_lengths_around_the_list_margin(storage, nx):
    ny, nz = 6, 5
    p0, u0 = W.random_smooth_state(nx, ny, nz, 3, amp_u=0.03, amp_p=2e-3, seed=50 + nx)
    sol = np.zeros((nz, ny, nx), np.uint8)
    sol[1:3, 2:4, nx // 2] = 1
    u0[:, sol.ravel() != 0] = 0
    inl = np.zeros((3, ny * nz))
    inl[0] = 0.04
    got, ref = run_pair("d3q19", (nx, ny, nz), 0.7,
                        ["inlet", "outflow", "wall", "wall", "periodic", "periodic"], 23,
                        storage=storage, solid=sol, inlet=inl, lid=(0.05, 0.0, 0.0), p0=p0,
                        u0=u0, force_out=True)
    eu, ep = field_errors(got, ref, 0.05)
    assert eu < TOL_U[storage] and ep < 10 * TOL_U[storage], (eu, ep)
    fscale = np.abs(ref[2]).max()
    tol_f = {"f64": 1e-12, "f32": 1e-4, "f16s": 3e-2}[storage]
    assert np.abs(got[2] - ref[2]).max() < tol_f * fscale
