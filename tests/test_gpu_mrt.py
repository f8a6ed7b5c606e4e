"""Multiple-relaxation-time collision on the GPU against the FP64 oracle.

MRT is not in the paper (d'Humieres et al. 2002): the non-equilibrium part
relaxes in an orthogonal moment basis, the stress at 1/tau and the bulk, even
and odd higher moments at their own rates.  The oracle builds its basis at run
time by Gram-Schmidt; the CUDA library carries integer tables checked at
compile time.  Tolerances as elsewhere: FP64 1e-12, FP32 1e-5 of the reference
speed on velocity (10x on pressure).
"""
import numpy as np
import pytest

import oracle
from paper_2201_11330_b300 import workloads as W
from test_gpu_parity import TOL, errors, gpu_run, oracle_run

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_11330_b300 import build
    build.build()


MRT_CASES = [
    ("d3q19", (37, 29, 23), "cavity", (1.4, 1.2, 1.1)),
    ("d3q27", (41, 9, 6), "channel", (1.1, 1.6, 0.9)),
    ("d2q9", (45, 33, 1), "periodic", (1.5, 1.3, 1.7)),
    ("d3q19", (300, 7, 5), "channel", (0.8, 1.0, 1.9)),
]


@pytest.mark.parametrize("lattice,shape,bc,rates", MRT_CASES)
@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("aa", [False, True])
def test_mrt_parity(lattice, shape, bc, rates, storage, aa):
    Q, d = oracle.dims(lattice)
    nx, ny, nz = shape
    p0, u0 = W.random_smooth_state(nx, ny, nz, d, amp_u=0.04, amp_p=2e-3, seed=24)
    lid = (0.08, 0.0, 0.02) if bc != "periodic" else None
    F = W.fourier_force(nx, ny, nz, amplitude=2e-5, seed=8, dims=d)
    steps = 61
    ref = oracle_run(lattice, shape, 0.62, bc, steps, lid=lid, F=F, p0=p0, u0=u0, mrt=rates)
    got = gpu_run(lattice, shape, 0.62, bc, steps, storage=storage, aa=aa, lid=lid, F=F,
                  p0=p0, u0=u0, mrt=rates)
    eu, ep = errors(got, ref, 0.05)
    assert eu < TOL[storage] and ep < 10 * TOL[storage], (eu, ep)
    if storage == "f64":  # and it is neither BGK nor the same MRT with other rates
        bgk = oracle_run(lattice, shape, 0.62, bc, steps, lid=lid, F=F, p0=p0, u0=u0)
        assert errors(got, bgk, 0.05)[0] > 1e3 * TOL["f64"]


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_mrt_with_equal_rates_is_bgk(storage):
    """Every rate at 1/tau (the default rates 0): the BGK fields, to rounding."""
    shape = (33, 21, 17)
    p0, u0 = W.random_smooth_state(*shape, 3, amp_u=0.04, seed=14)
    F = W.fourier_force(*shape, amplitude=2e-5, seed=4, dims=3)
    a = gpu_run("d3q19", shape, 0.7, "cavity", 40, storage=storage, lid=(0.07, 0, 0), F=F,
                p0=p0, u0=u0)
    b = gpu_run("d3q19", shape, 0.7, "cavity", 40, storage=storage, lid=(0.07, 0, 0), F=F,
                p0=p0, u0=u0, mrt=(0.0, 0.0, 0.0))
    tol = 1e-13 if storage == "f64" else 2e-6
    assert np.abs(a[1] - b[1]).max() < tol * 0.07


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("bc", ["cavity", "periodic"])
def test_mrt_aa_equals_pull_bitwise(storage, bc):
    shape = (45, 26, 19)
    p0, u0 = W.random_smooth_state(*shape, 3, amp_u=0.04, seed=15)
    F = W.fourier_force(*shape, amplitude=2e-5, seed=5, dims=3)
    lid = (0.07, 0, 0) if bc != "periodic" else None
    for steps in (10, 11):
        a = gpu_run("d3q19", shape, 0.6, bc, steps, storage=storage, aa=False, lid=lid,
                    p0=p0, u0=u0, F=F, mrt=(1.3, 1.2, 1.1))
        b = gpu_run("d3q19", shape, 0.6, bc, steps, storage=storage, aa=True, lid=lid,
                    p0=p0, u0=u0, F=F, mrt=(1.3, 1.2, 1.1))
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), steps


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_mrt_with_faces_and_obstacles(storage):
    """The general kernel runs MRT too: a channel past a sphere with an inlet, a
    pressure outlet and symmetry planes, against the oracle."""
    from paper_2201_11330_b300.lbm import Lattice
    nx, ny, nz = 33, 15, 11
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    sol = (((x - 12) ** 2 + (y - 7) ** 2 + (z - 5) ** 2) <= 9.6).astype(np.uint8)
    faces = ["inlet", "outflow", "symmetry", "symmetry", "periodic", "periodic"]
    inl = np.zeros((3, ny * nz))
    inl[0] = 0.04
    rates = (1.2, 1.4, 1.1)
    lat = Lattice("d3q19", nx, ny, nz, 0.6, faces, storage=storage, obstacles=True, mrt=rates)
    lat.set_geometry(torch.from_numpy(sol.ravel()).cuda())
    lat.set_inlet(torch.from_numpy(inl.astype(np.float32)).cuda())
    lat.init()
    lat.step(40)
    p, u = lat.macroscopic()
    pr, ur = oracle.run("d3q19", nx, ny, nz, 0.6, faces, 40, solid=sol,
                        inlet=inl.astype(np.float32).astype(np.float64), mrt=rates)
    eu = np.abs(u.cpu().numpy() - ur).max() / 0.04
    assert eu < TOL[storage], eu
