"""The paper's Sec. 5 example: 2D channel flow past a cylinder (D2Q9), run
through the general step kernel, drag and lift from the momentum exchange.

Laminar case: channel 1024 x 1024, cylinder of diameter D = 32 centred 512
from the inlet on the centreline, relaxation parameter 1.8, Re = U D / nu = 20
with U the inlet's centreline speed; the paper's drag coefficient
F / (rho U^2 r) converges to 2.06.  Shedding case: channel 512 x 128, D = 16
centred 64 from the inlet, relaxation parameter 1.953, Re = 100, started from
the inlet profile with a small random perturbation; the drag oscillates
around 1.46 with periodic vortex shedding.  Parabolic velocity inlet,
no-slip walls, pressure outlet (reading of the paper's convective outflow).
FP32 arithmetic, shifted FP32 storage.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_11330_b300 import build
    build.build()


def cylinder_channel(nx, ny, D, xc, omega, Re, perturb, seed=7):
    from paper_2201_11330_b300.lbm import Lattice
    tau = 1.0 / omega  # relaxation parameter 1/(tau_paper + 1/2) = 1/tau
    nu = (tau - 0.5) / 3
    U = Re * nu / D
    yc = (ny - 1) / 2
    x, y = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    solid = ((x - xc) ** 2 + (y - yc) ** 2 <= (D / 2) ** 2).astype(np.uint8)
    s = np.arange(ny)
    prof = U * (s + 0.5) * (ny - 0.5 - s) / (ny / 2) ** 2
    lat = Lattice("d2q9", nx, ny, 1, tau, ["inlet", "outflow", "wall", "wall", "periodic",
                                           "periodic"], storage="f32", obstacles=True)
    lat.set_geometry(torch.from_numpy(solid.ravel()).cuda())
    lat.set_inlet(torch.from_numpy(np.stack([prof, 0 * prof]).astype(np.float32)).cuda())
    u0 = np.zeros((2, ny, nx))
    u0[0] = prof[:, None]
    u0 += perturb * U * np.random.default_rng(seed).standard_normal(u0.shape)
    u0[:, solid != 0] = 0
    lat.init(None, torch.from_numpy(u0.reshape(2, -1)).cuda())
    return lat, U


def coefficients(lat, U, D, steps, every):
    """(drag, lift) = F / (rho0 U^2 r) every `every` steps."""
    out = []
    for _ in range(steps // every):
        lat.step(every - 1)
        f = lat.step_force(1)
        out.append((f[0] / (U * U * D / 2), f[1] / (U * U * D / 2)))
    return np.array(out)


def test_cylinder_re20_drag():
    lat, U = cylinder_channel(1024, 1024, 32, 511.5, 1.8, 20, 0.0)
    c = coefficients(lat, U, 32, 240000, 4000)
    assert abs(c[-1, 0] / 2.06 - 1) < 0.03, c[:, 0]
    assert np.abs(c[-5:, 0] - c[-1, 0]).max() < 0.01 * c[-1, 0]  # converged
    assert abs(c[-1, 1]) < 1e-3  # symmetric: no lift
    r = lat.reduce()
    assert np.isfinite(r["kinetic_energy"])


def test_cylinder_re100_shedding():
    lat, U = cylinder_channel(512, 128, 16, 63.5, 1.953, 100, 0.01)
    c = coefficients(lat, U, 16, 80000, 50)
    late = c[len(c) // 2:]
    assert abs(late[:, 0].mean() / 1.46 - 1) < 0.1, late[:, 0].mean()
    cl = late[:, 1]
    assert cl.max() > 0.1 and cl.min() < -0.1  # the lift oscillates: vortex shedding
    ups = np.where(np.diff(np.sign(cl)) > 0)[0]
    assert len(ups) >= 4  # several periods, not a drift
    periods = np.diff(ups)
    assert periods.std() < 0.05 * periods.mean()  # periodic
