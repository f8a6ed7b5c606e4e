"""Adjoint on the GPU against the FP64 CPU adjoint and central differences.

* FP64 GPU adjoint == FP64 oracle adjoint (1e-11) on small boxes, every BC.
* FP32 GPU adjoint vs FP64 CPU adjoint, D3Q19 periodic 32^3, T = 2000,
  K = 100, Fourier force A = 1e-5: 1e-4 relative.
* GPU adjoint vs central differences of FP64 GPU forward runs
  (h = 1e-3 relative): 1e-3 relative, for the force and the lid velocity.
* the torch.autograd.Function returns the same gradients.
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


def make(lattice, shape, tau, bc, storage, lid, F, p0=None, u0=None):
    from paper_2201_11330_b300.lbm import Lattice
    lat = Lattice(lattice, *shape, tau, bc, storage=storage, lid=lid or (0, 0, 0), has_force=True)
    lat.set_force(torch.from_numpy(np.ascontiguousarray(F, dtype=np.float32)).cuda())
    lat.init(None if p0 is None else torch.from_numpy(p0).cuda(),
             None if u0 is None else torch.from_numpy(np.ascontiguousarray(u0)).cuda())
    return lat


def gpu_adjoint(lattice, shape, tau, bc, T, K, storage, lid, F, p0=None, u0=None):
    lat = make(lattice, shape, tau, bc, storage, lid, F, p0, u0)
    J, g, gU = lat.adjoint(T, K)
    return J, g.cpu().numpy(), gU.numpy()


def gpu_J(lattice, shape, tau, bc, T, storage, lid, F, p0=None, u0=None):
    lat = make(lattice, shape, tau, bc, storage, lid, F, p0, u0)
    lat.step(T)
    return lat.reduce()["kinetic_energy"]


@pytest.mark.parametrize("lattice,shape,bc", [("d3q19", (12, 10, 8), "cavity"),
                                              ("d3q19", (9, 11, 7), "channel"),
                                              ("d3q27", (8, 7, 6), "periodic"),
                                              ("d2q9", (21, 17, 1), "cavity")])
@pytest.mark.parametrize("K", [1, 6, 50])
def test_fp64_adjoint_matches_oracle(lattice, shape, bc, K):
    Q, d = oracle.dims(lattice)
    T = 20
    lid = (0.05, 0.0, 0.01) if bc != "periodic" else None
    F = W.fourier_force(*shape, amplitude=1e-4, seed=3, dims=d)
    p0, u0 = W.random_smooth_state(*shape, d, amp_u=0.03, seed=5)
    Jr, gr, gUr = oracle.adjoint(lattice, *shape, 0.7, bc, T, K, lid=lid,
                                 F=F.astype(np.float64), p0=p0, u0=u0.ravel())
    Jg, gg, gUg = gpu_adjoint(lattice, shape, 0.7, bc, T, K, "f64", lid, F, p0, u0)
    assert abs(Jg - Jr) <= 1e-12 * Jr
    assert np.abs(gg - gr).max() <= 1e-11 * np.abs(gr).max()
    if lid is not None:
        assert np.abs(gUg - gUr).max() <= 1e-11 * np.abs(gUr).max()
    else:
        assert np.all(gUg == 0)


@pytest.fixture(scope="module")
def periodic32():
    n, T, K = 32, 2000, 100
    F = W.fourier_force(n, n, n, amplitude=1e-5, seed=2201)
    J, g, gU = oracle.adjoint("d3q19", n, n, n, 0.8, "periodic", T, K, F=F.astype(np.float64))
    return n, T, K, F, J, g


def test_fp32_adjoint_matches_cpu_adjoint_32(periodic32):
    n, T, K, F, Jr, gr = periodic32
    Jg, gg, _ = gpu_adjoint("d3q19", (n, n, n), 0.8, "periodic", T, K, "f32", None, F)
    assert abs(Jg - Jr) <= 1e-4 * Jr
    assert np.abs(gg - gr).max() <= 1e-4 * np.abs(gr).max()


def test_adjoint_matches_finite_differences(periodic32):
    """Central differences of FP64 GPU forward runs along random directions."""
    n, T, K, F, _, _ = periodic32
    shape = (n, n, n)
    J, g, _ = gpu_adjoint("d3q19", shape, 0.8, "periodic", T, K, "f32", None, F)
    rng = np.random.default_rng(0)
    h = 1e-3 * np.abs(F).max()
    for _ in range(2):
        v = rng.standard_normal(F.shape).astype(np.float32)
        Fp = (F.astype(np.float64) + h * v).astype(np.float32)
        Fm = (F.astype(np.float64) - h * v).astype(np.float32)
        # use the exactly representable perturbation actually applied
        dv = (Fp.astype(np.float64) - Fm.astype(np.float64)) / 2
        fd = (gpu_J("d3q19", shape, 0.8, "periodic", T, "f64", None, Fp)
              - gpu_J("d3q19", shape, 0.8, "periodic", T, "f64", None, Fm)) / 2
        ad = float((g * dv).sum())
        assert abs(fd - ad) <= 1e-3 * abs(fd), (fd, ad)


def test_lid_gradient_matches_finite_differences():
    n, T, K = 24, 400, 50
    shape = (n, n, n)
    F = W.fourier_force(n, n, n, amplitude=1e-5, seed=2201)
    lid = [0.05, 0.0, 0.0]
    _, _, gU = gpu_adjoint("d3q19", shape, 0.6, "cavity", T, K, "f32", lid, F)
    for k in (0, 2):
        h = 1e-3 * 0.05
        lp, lm = list(lid), list(lid)
        lp[k] += h
        lm[k] -= h
        fd = (gpu_J("d3q19", shape, 0.6, "cavity", T, "f64", lp, F)
              - gpu_J("d3q19", shape, 0.6, "cavity", T, "f64", lm, F)) / (2 * h)
        assert abs(fd - gU[k]) <= 1e-3 * abs(fd) + 1e-12, (k, fd, gU[k])


def test_autograd_function():
    from paper_2201_11330_b300.autograd import kinetic_energy
    from paper_2201_11330_b300.lbm import Lattice
    n, T, K = 16, 60, 16
    F = torch.from_numpy(W.fourier_force(n, n, n, amplitude=1e-4, seed=9)).cuda().requires_grad_()
    U = torch.tensor([0.05, 0.0, 0.0], dtype=torch.float64, requires_grad=True)
    lat = Lattice("d3q19", n, n, n, 0.7, "cavity", storage="f64", has_force=True)
    J = kinetic_energy(lat, F, U, T, K)
    J.backward()
    Jr, gr, gUr = oracle.adjoint("d3q19", n, n, n, 0.7, "cavity", T, K, lid=[0.05, 0, 0],
                                 F=F.detach().cpu().numpy().astype(np.float64))
    assert abs(J.item() - Jr) <= 1e-12 * Jr
    assert np.abs(F.grad.cpu().numpy() - gr).max() <= 1e-6 * np.abs(gr).max()
    assert np.abs(U.grad.numpy() - gUr).max() <= 1e-11 * np.abs(gUr).max()
