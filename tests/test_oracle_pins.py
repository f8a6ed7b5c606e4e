"""Pins of the FP64 CPU oracle against facts the paper and the mathematics fix.

None of these tests compares the oracle with itself or with the CUDA path:
each checks a closed form, an invariant, an analytic flow or a finite
difference, so that a dropped term, a wrong sign, a wrong index or a
transposed operand in the oracle fails at least one of them.
"""
from fractions import Fraction
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from paper_2201_11330_b300 import workloads as W

LATTICES = ["d2q9", "d3q19", "d3q27"]
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Sec. 2.1: the velocity sets


def test_d2q9_table_matches_sec2_1():
    """The D2Q9 matrix and weights equal the ones printed in Sec. 2.1."""
    rows = {}
    with open(os.path.join(GOLDEN, "d2q9_table_sec2_1.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            key, *vals = line.split()
            rows[key] = vals
    e, t, opp = oracle.tables("d2q9")
    assert [int(v) for v in rows["e_x"]] == list(e[:, 0])
    assert [int(v) for v in rows["e_y"]] == list(e[:, 1])
    assert np.all(e[:, 2] == 0)
    want = [float(Fraction(v)) for v in rows["t"]]
    assert list(t) == want
    # "opposite of a is m-1-a" (Sec. 2.1)
    assert list(opp) == list(range(8, -1, -1))


@pytest.mark.parametrize("lattice", LATTICES)
def test_velocity_set_isotropy(lattice):
    """Weights reproduce the Maxwellian moments up to fourth order, c_s^2 = 1/3."""
    e, t, opp = oracle.tables(lattice)
    Q, d = oracle.dims(lattice)
    assert len(t) == Q == {"d2q9": 9, "d3q19": 19, "d3q27": 27}[lattice]
    assert len({tuple(v) for v in e}) == Q
    assert list(opp) == list(range(Q - 1, -1, -1))
    assert np.all(e[opp] == -e)
    assert abs(t.sum() - 1) < 1e-15
    E = e[:, :d].astype(float)
    assert np.abs(t @ E).max() < 1e-16
    I = np.eye(d)
    assert np.abs(np.einsum("a,ai,aj->ij", t, E, E) - I / 3).max() < 1e-15
    assert np.abs(np.einsum("a,ai,aj,ak->ijk", t, E, E, E)).max() < 1e-16
    four = np.einsum("a,ai,aj,ak,al->ijkl", t, E, E, E, E)
    want = (np.einsum("ij,kl->ijkl", I, I) + np.einsum("ik,jl->ijkl", I, I)
            + np.einsum("il,jk->ijkl", I, I)) / 9
    assert np.abs(four - want).max() < 1e-15


# --------------------------------------------------------------------------
# Sec. 2.1: equilibria


@pytest.mark.parametrize("lattice", LATTICES)
@pytest.mark.parametrize("compressible", [False, True])
def test_equilibrium_moments(lattice, compressible):
    """Zeroth, first and second moments of Eq. (incompressible_feq) / Eq. (feq)."""
    rng = np.random.default_rng(11)
    e, t, _ = oracle.tables(lattice)
    Q, d = oracle.dims(lattice)
    E = e[:, :d].astype(float)
    for _ in range(5):
        P = 1.0 + 0.1 * rng.standard_normal()
        u = 0.08 * rng.standard_normal(d)
        rho0 = 1.0 + 0.2 * rng.random()
        feq = oracle.equilibrium(lattice, P, u, rho0=rho0, compressible=compressible)
        r = P if compressible else rho0
        assert abs(feq.sum() - P) < 1e-14
        assert np.abs(E.T @ feq - r * u).max() < 1e-15
        second = np.einsum("a,ai,aj->ij", feq, E, E)
        assert np.abs(second - (P / 3 * np.eye(d) + r * np.outer(u, u))).max() < 1e-14


@pytest.mark.parametrize("lattice", LATTICES)
def test_collision_invariants(lattice):
    """Eq. (collision) keeps P and j; feq is its fixed point; the force adds F to j."""
    rng = np.random.default_rng(5)
    e, t, _ = oracle.tables(lattice)
    Q, d = oracle.dims(lattice)
    E = e[:, :d].astype(float)
    for tau in (0.55, 0.8, 1.7):
        f = t * (1 + 0.05 * rng.standard_normal(Q))
        out = oracle.collide_node(lattice, f, tau)
        assert abs(out.sum() - f.sum()) < 1e-15
        assert np.abs(E.T @ out - E.T @ f).max() < 1e-15
        # rest fraction relaxes by exactly (1 - omega) away from equilibrium
        P = f.sum()
        u = E.T @ f
        feq = oracle.equilibrium(lattice, P, u)
        assert np.abs(out - (feq + (1 - 1 / tau) * (f - feq))).max() < 1e-15
        assert np.abs(oracle.collide_node(lattice, feq, tau) - feq).max() < 1e-15
        F = 1e-4 * rng.standard_normal(d)
        outF = oracle.collide_node(lattice, f, tau, F=F)
        assert abs(outF.sum() - f.sum()) < 1e-15
        assert np.abs(E.T @ outF - (E.T @ f + F)).max() < 1e-15


def _moment(E, f, powers):
    """sum_a e_ax^i e_ay^j e_az^k f_a for powers = (i, j, k)."""
    m = np.ones(len(f))
    for k, p in enumerate(powers):
        if p:
            m = m * E[:, k] ** p
    return (m * f).sum()


@pytest.mark.parametrize("lattice", LATTICES)
def test_trt_collision_moments(lattice):
    """TRT keeps P and j (the force adds F), leaves feq fixed, relaxes the
    non-equilibrium part of every even moment by (1 - omega) and of every odd
    moment by (1 - omega_m); Lambda = (tau - 1/2)^2 is BGK."""
    rng = np.random.default_rng(9)
    e, t, _ = oracle.tables(lattice)
    Q, d = oracle.dims(lattice)
    E = np.zeros((Q, 3))
    E[:, :d] = e[:, :d]
    for tau, lam in ((0.55, 3 / 16), (0.8, 1 / 4), (1.7, 1 / 12)):
        om = 1 / tau
        om_m = 1 / (lam / (tau - 0.5) + 0.5)
        f = t * (1 + 0.05 * rng.standard_normal(Q))
        out = oracle.collide_node(lattice, f, tau, trt_lambda=lam)
        assert abs(out.sum() - f.sum()) < 1e-15
        assert np.abs(E.T @ out - E.T @ f).max() < 1e-15
        feq = oracle.equilibrium(lattice, f.sum(), (E.T @ f)[:d])
        assert np.abs(oracle.collide_node(lattice, feq, tau, trt_lambda=lam) - feq).max() < 1e-15
        # moments of the non-equilibrium part (F = 0): parity of the total
        # power decides the rate
        for pw in [(1, 1, 0), (2, 0, 0), (0, 2, 0), (1, 2, 0), (2, 1, 0), (2, 2, 0), (3, 0, 0),
                   (1, 0, 0), (0, 1, 0)] + ([(1, 1, 1), (0, 1, 2), (1, 0, 2)] if d == 3 else []):
            before = _moment(E, f - feq, pw)
            after = _moment(E, out - feq, pw)
            rate = om if sum(pw) % 2 == 0 else om_m
            assert abs(after - (1 - rate) * before) < 1e-15, (pw, after, before)
        F = 1e-4 * rng.standard_normal(d)
        outF = oracle.collide_node(lattice, f, tau, F=F, trt_lambda=lam)
        assert abs(outF.sum() - f.sum()) < 1e-15
        assert np.abs(E[:, :d].T @ outF - (E[:, :d].T @ f + F)).max() < 1e-15
        # BGK as the special case omega_m = omega
        bgk = oracle.collide_node(lattice, f, tau, F=F)
        same = oracle.collide_node(lattice, f, tau, F=F, trt_lambda=(tau - 0.5) ** 2)
        assert np.abs(bgk - same).max() < 1e-15


# --------------------------------------------------------------------------
# Whole scheme: invariants


@pytest.mark.parametrize("lattice,shape", [("d2q9", (12, 10, 1)), ("d3q19", (6, 5, 7)),
                                           ("d3q27", (5, 6, 4))])
@pytest.mark.parametrize("bc", ["cavity", "periodic", "channel"])
def test_rest_state_is_exact(lattice, shape, bc):
    """u = 0, no force, resting walls: every population stays at t_a (to round-off)."""
    nx, ny, nz = shape
    _, t, _ = oracle.tables(lattice)
    _, _, f0 = oracle.run(lattice, nx, ny, nz, 0.7, bc, 0, want_f=True)
    assert np.array_equal(f0, np.repeat(t[:, None], nx * ny * nz, axis=1))
    p, u, f = oracle.run(lattice, nx, ny, nz, 0.7, bc, 40, want_f=True)
    assert np.abs(f - f0).max() < 1e-15
    assert np.abs(u).max() < 1e-15


@pytest.mark.parametrize("lattice,shape", [("d2q9", (16, 12, 1)), ("d3q19", (8, 6, 7)),
                                           ("d3q27", (6, 7, 5))])
def test_periodic_conservation(lattice, shape):
    """Periodic streaming + collision conserve sum P and sum j to round-off."""
    nx, ny, nz = shape
    Q, d = oracle.dims(lattice)
    p0, u0 = W.random_smooth_state(nx, ny, nz, d, amp_u=0.05, amp_p=1e-3, seed=3)
    N = nx * ny * nz
    p, u = oracle.run(lattice, nx, ny, nz, 0.62, "periodic", 300, p0=p0, u0=u0)
    assert abs(p.sum() - p0.sum()) / N < 1e-14
    assert np.abs(u.sum(axis=1) - u0.sum(axis=1)).max() / N < 1e-14
    # something did happen
    assert np.abs(u - u0).max() > 1e-4


@pytest.mark.parametrize("lattice,shape", [("d2q9", (10, 8, 1)), ("d3q19", (6, 5, 4))])
def test_uniform_force_momentum_growth(lattice, shape):
    """Each step adds exactly F per node to the momentum of a periodic box."""
    nx, ny, nz = shape
    Q, d = oracle.dims(lattice)
    N = nx * ny * nz
    G = np.array([2e-5, -1e-5, 3e-5][:d])
    F = np.repeat(G[:, None], N, axis=1)
    for n in (1, 7, 30):
        p, u = oracle.run(lattice, nx, ny, nz, 0.9, "periodic", n, F=F)
        # rho0 u = j + F/2, with j = n F after n steps from rest
        assert np.abs(u.sum(axis=1) - (n + 0.5) * G * N).max() < 1e-16 * N * n + 1e-18
        assert abs(p.sum() - N / 3) < 1e-14 * N


@pytest.mark.parametrize("lattice,shape", [("d2q9", (12, 9, 1)), ("d3q19", (7, 6, 5)),
                                           ("d3q27", (5, 6, 4))])
def test_cavity_mass_conservation(lattice, shape):
    """A closed cavity with a tangential lid keeps its mass (corners included)."""
    nx, ny, nz = shape
    N = nx * ny * nz
    p, u = oracle.run(lattice, nx, ny, nz, 0.6, "cavity", 200, lid=[0.1, 0, 0])
    assert abs(p.sum() - N / 3) / N < 1e-14
    assert np.abs(u).max() > 1e-3


@pytest.mark.parametrize("lattice", ["d3q19", "d3q27"])
def test_cavity_mirror_symmetry(lattice):
    """Lid along +x: the flow is mirror-symmetric about the z mid-plane."""
    nx, ny, nz = 7, 6, 6
    p, u = oracle.run(lattice, nx, ny, nz, 0.6, "cavity", 150, lid=[0.1, 0, 0])
    P = p.reshape(nz, ny, nx)
    U = u.reshape(3, nz, ny, nx)
    assert np.abs(U[0] - U[0][::-1]).max() < 1e-15
    assert np.abs(U[1] - U[1][::-1]).max() < 1e-15
    assert np.abs(U[2] + U[2][::-1]).max() < 1e-15
    assert np.abs(P - P[::-1]).max() < 1e-15
    assert np.abs(U[2]).max() > 1e-5


def test_pressure_gauge_invariance():
    """Incompressible model: shifting P0 by a constant leaves u unchanged."""
    nx, ny, nz = 8, 7, 6
    _, u0 = W.random_smooth_state(nx, ny, nz, 3, seed=9)
    N = nx * ny * nz
    pa, ua = oracle.run("d3q19", nx, ny, nz, 0.7, "cavity", 60, lid=[0.05, 0, 0],
                        p0=np.full(N, 1 / 3), u0=u0)
    pb, ub = oracle.run("d3q19", nx, ny, nz, 0.7, "cavity", 60, lid=[0.05, 0, 0],
                        p0=np.zeros(N), u0=u0)
    assert np.abs(ua - ub).max() < 1e-15
    assert np.abs((pa - pb) - 1 / 3).max() < 1e-14


# --------------------------------------------------------------------------
# Whole scheme: analytic flows


def _tg_amplitude(u, n):
    x, y, _ = W.grid(n, n, 1)
    k = 2 * math.pi / n
    mode = -np.cos(k * x) * np.sin(k * y)
    return (u[0] * mode).sum() / (mode * mode).sum()


@pytest.mark.parametrize("compressible", [False, True])
def test_taylor_green_decay(compressible):
    """Velocity amplitude decays at nu (kx^2 + ky^2), nu = (tau - 1/2)/3 (within 1%)."""
    n, tau = 96, 0.8
    p0, u0 = W.taylor_green_2d(n, n, 0.05)
    amps = []
    for T in (100, 900):
        _, u = oracle.run("d2q9", n, n, 1, tau, "periodic", T, p0=p0, u0=u0,
                          compressible=compressible)
        amps.append(_tg_amplitude(u, n))
    rate = -math.log(amps[1] / amps[0]) / 800
    assert abs(rate / W.taylor_green_rate(n, n, tau) - 1) < 0.01


@pytest.mark.parametrize("lattice", ["d2q9", "d3q19", "d3q27"])
def test_poiseuille(lattice):
    """Body-force channel flow: exact parabola at (tau - 1/2)^2 = 3/16; else the
    same second differences (-G/nu) plus a constant wall slip."""
    ny, G = 14, 1e-6
    Q, d = oracle.dims(lattice)
    for tau in (0.5 + math.sqrt(3 / 16), 0.8):
        nu = W.viscosity(tau)
        F = np.zeros((d, ny))
        F[0] = G
        steps = int(25 * ny * ny / nu)
        _, u = oracle.run(lattice, 1, ny, 1, tau, "channel", steps, F=F)
        ux = u[0]
        y = np.arange(ny)
        parabola = G / (2 * nu) * (y + 0.5) * (ny - 0.5 - y)
        d2 = ux[2:] - 2 * ux[1:-1] + ux[:-2]
        assert np.abs(d2 * nu / G + 1).max() < 1e-8
        slip = ux - parabola
        assert np.abs(slip - slip.mean()).max() < 1e-9 * parabola.max()
        if tau < 0.9:
            assert abs(slip.mean()) > 1e-4 * parabola.max()
        else:
            assert np.abs(slip).max() < 1e-9 * parabola.max()
        assert np.abs(u[1:]).max() < 1e-10 * parabola.max()


@pytest.mark.parametrize("lattice", ["d2q9", "d3q19", "d3q27"])
def test_trt_poiseuille_exact_for_any_tau(lattice):
    """With Lambda = 3/16 half-way bounce-back puts the walls exactly half a
    link out for any tau (Ginzburg's TRT result): the steady body-force channel
    profile is the parabola to rounding, while BGK at the same tau is not."""
    ny, G = 12, 1e-5
    Q, d = oracle.dims(lattice)
    y = np.arange(ny)
    for tau in (0.8, 1.5, 3.0):
        nu = W.viscosity(tau)
        F = np.zeros((d, ny))
        F[0] = G
        steps = int(30 * ny * ny / nu)
        parabola = G / (2 * nu) * (y + 0.5) * (ny - 0.5 - y)
        _, u = oracle.run(lattice, 1, ny, 1, tau, "channel", steps, F=F, trt_lambda=3 / 16)
        assert np.abs(u[0] - parabola).max() < 1e-10 * parabola.max(), tau
        assert np.abs(u[1:]).max() < 1e-10 * parabola.max()
        _, ub = oracle.run(lattice, 1, ny, 1, tau, "channel", steps, F=F)
        assert np.abs(ub[0] - parabola).max() > 1e-3 * parabola.max(), tau


@pytest.mark.parametrize("lam", [1 / 4, 3 / 16, 1 / 12])
def test_trt_shear_viscosity_set_by_omega(lam):
    """TRT: the shear-wave decay rate is nu (kx^2 + ky^2) with nu = (tau - 1/2)/3
    from the even rate alone, whatever Lambda (within 1 %)."""
    n, tau = 96, 0.8
    p0, u0 = W.taylor_green_2d(n, n, 0.05)
    amps = []
    for T in (100, 900):
        _, u = oracle.run("d2q9", n, n, 1, tau, "periodic", T, p0=p0, u0=u0, trt_lambda=lam)
        amps.append(_tg_amplitude(u, n))
    rate = -math.log(amps[1] / amps[0]) / 800
    assert abs(rate / W.taylor_green_rate(n, n, tau) - 1) < 0.01


@pytest.mark.parametrize("lattice", LATTICES)
def test_mrt_reduces_to_bgk_and_trt(lattice):
    """Multiple-relaxation-time collision: with every rate equal to omega it is
    BGK, and with the even moments at omega and the odd ones at omega_m it is
    TRT of the same Lambda (both pinned on their own elsewhere)."""
    rng = np.random.default_rng(21)
    e, t, _ = oracle.tables(lattice)
    Q, d = oracle.dims(lattice)
    for tau, lam in ((0.55, 3 / 16), (0.8, 1 / 4), (1.7, 1 / 12)):
        om = 1 / tau
        om_m = 1 / (lam / (tau - 0.5) + 0.5)
        f = t * (1 + 0.05 * rng.standard_normal(Q))
        F = 1e-4 * rng.standard_normal(d)
        for Fx in (None, F):
            bgk = oracle.collide_node(lattice, f, tau, F=Fx)
            trt = oracle.collide_node(lattice, f, tau, F=Fx, trt_lambda=lam)
            assert np.abs(oracle.collide_node(lattice, f, tau, F=Fx, mrt=(om, om, om)) -
                          bgk).max() < 1e-15
            assert np.abs(oracle.collide_node(lattice, f, tau, F=Fx, mrt=(om, om, om_m)) -
                          trt).max() < 1e-15


@pytest.mark.parametrize("lattice", LATTICES)
def test_mrt_moments_relax_by_class(lattice):
    """MRT keeps P and j (the force adds F), leaves feq fixed, relaxes the
    non-equilibrium stress moments (e_x e_y, e_x^2 - e_y^2) at omega, the bulk
    moment (|e|^2 minus its mean over the set) at s_bulk and odd third-order
    moments (e_x e_y^2) at s_odd, whatever the other rates."""
    rng = np.random.default_rng(22)
    e, t, _ = oracle.tables(lattice)
    Q, d = oracle.dims(lattice)
    E = np.zeros((Q, 3))
    E[:, :d] = e[:, :d]
    c2 = (E ** 2).sum(axis=1)
    for tau, rates in ((0.6, (1.5, 1.2, 1.1)), (1.3, (0.7, 1.9, 1.6))):
        om = 1 / tau
        sb, se, so = rates
        f = t * (1 + 0.05 * rng.standard_normal(Q))
        out = oracle.collide_node(lattice, f, tau, mrt=rates)
        assert abs(out.sum() - f.sum()) < 1e-15
        assert np.abs(E.T @ out - E.T @ f).max() < 1e-15
        feq = oracle.equilibrium(lattice, f.sum(), (E.T @ f)[:d])
        assert np.abs(oracle.collide_node(lattice, feq, tau, mrt=rates) - feq).max() < 1e-15
        n, nout = f - feq, out - feq
        for w, rate in ((E[:, 0] * E[:, 1], om), (E[:, 0] ** 2 - E[:, 1] ** 2, om),
                        (c2 - c2.mean(), sb), (E[:, 0] * E[:, 1] ** 2, so)):
            assert abs(w @ nout - (1 - rate) * (w @ n)) < 1e-15
        F = 1e-4 * rng.standard_normal(d)
        outF = oracle.collide_node(lattice, f, tau, F=F, mrt=rates)
        assert abs(outF.sum() - f.sum()) < 1e-15
        assert np.abs(E[:, :d].T @ outF - (E[:, :d].T @ f + F)).max() < 1e-15


def test_mrt_shear_viscosity_set_by_omega():
    """MRT: the shear-wave decay rate is nu (kx^2 + ky^2), nu = (tau - 1/2)/3,
    from the stress rate alone, whatever the bulk and ghost rates (within 1 %)."""
    n, tau = 96, 0.8
    p0, u0 = W.taylor_green_2d(n, n, 0.05)
    for rates in ((1.5, 1.2, 1.1), (0.9, 1.8, 1.4)):
        amps = []
        for T in (100, 900):
            _, u = oracle.run("d2q9", n, n, 1, tau, "periodic", T, p0=p0, u0=u0, mrt=rates)
            amps.append(_tg_amplitude(u, n))
        rate = -math.log(amps[1] / amps[0]) / 800
        assert abs(rate / W.taylor_green_rate(n, n, tau) - 1) < 0.01, rates


def test_mrt_conserves_mass_and_momentum_on_periodic_box():
    """Distinct MRT rates, D3Q19 periodic box: total mass and momentum stay
    constant to rounding over 200 steps."""
    nx, ny, nz = 12, 10, 8
    p0, u0 = W.random_smooth_state(nx, ny, nz, 3, amp_u=0.04, seed=5)
    _, _, f0 = oracle.run("d3q19", nx, ny, nz, 0.7, "periodic", 0, p0=p0, u0=u0.ravel(),
                          want_f=True)
    _, _, f1 = oracle.run("d3q19", nx, ny, nz, 0.7, "periodic", 200, p0=p0, u0=u0.ravel(),
                          want_f=True, mrt=(1.4, 1.2, 1.1))
    e, _, _ = oracle.tables("d3q19")
    assert abs(f1.sum() - f0.sum()) < 1e-12 * f0.sum()
    assert np.abs(e[:, :3].T @ f1.sum(axis=1) - e[:, :3].T @ f0.sum(axis=1)).max() < 1e-12


def test_mrt_rates_are_checked():
    f = oracle.equilibrium("d2q9", 1.0, [0.0, 0.0])
    for bad in ((0.0, 1.0, 1.0), (1.0, 2.0, 1.0), (1.0, 1.0, float("nan"))):
        with pytest.raises(AssertionError):
            oracle.collide_node("d2q9", f, 0.8, mrt=bad)


@pytest.mark.parametrize("lattice", ["d2q9", "d3q19"])
def test_couette(lattice):
    """Moving top wall, no force: linear profile U (y + 1/2)/ny for any tau."""
    ny, U = 12, 0.02
    for tau in (0.6, 1.3):
        nu = W.viscosity(tau)
        _, u = oracle.run(lattice, 1, ny, 1, tau, "channel", int(25 * ny * ny / nu),
                          lid=[U, 0, 0])
        y = np.arange(ny)
        assert np.abs(u[0] - U * (y + 0.5) / ny).max() < 1e-10 * U


# --------------------------------------------------------------------------
# Adjoint: central finite differences of the forward run


def _J(lattice, shape, tau, bc, T, lid, F):
    nx, ny, nz = shape
    _, u = oracle.run(lattice, nx, ny, nz, tau, bc, T, lid=lid, F=F)
    return 0.5 * float((u * u).sum())


@pytest.mark.parametrize("lattice,shape,bc", [("d3q19", (4, 5, 3), "cavity"),
                                              ("d2q9", (6, 5, 1), "channel"),
                                              ("d3q27", (3, 4, 3), "periodic")])
def test_adjoint_matches_finite_differences(lattice, shape, bc):
    nx, ny, nz = shape
    Q, d = oracle.dims(lattice)
    N = nx * ny * nz
    tau, T, K = 0.7, 7, 3
    lid = [0.05, 0.0, 0.01] if bc != "periodic" else None
    F = W.fourier_force(nx, ny, nz, amplitude=1e-3, seed=4, dims=d, dtype=np.float64)
    J, gF, gU = oracle.adjoint(lattice, nx, ny, nz, tau, bc, T, K, lid=lid, F=F)
    assert abs(J - _J(lattice, shape, tau, bc, T, lid, F)) < 1e-15
    rng = np.random.default_rng(1)
    for _ in range(2):
        v = rng.standard_normal((d, N))
        h = 1e-3 * np.abs(F).max()
        fd = (_J(lattice, shape, tau, bc, T, lid, F + h * v)
              - _J(lattice, shape, tau, bc, T, lid, F - h * v)) / (2 * h)
        assert abs(fd - (gF * v).sum()) <= 1e-7 * abs(fd)
    if lid is not None:
        for k in (0, 2):
            h = 1e-4
            lp = list(lid); lm = list(lid)
            lp[k] += h; lm[k] -= h
            fd = (_J(lattice, shape, tau, bc, T, lp, F) - _J(lattice, shape, tau, bc, T, lm, F)) / (2 * h)
            assert abs(fd - gU[k]) <= 1e-6 * abs(fd) + 1e-14
    else:
        assert np.all(gU == 0)


def test_adjoint_checkpoint_interval_invariance():
    """Recomputing between checkpoints gives the same gradient for any K."""
    args = ("d3q19", 4, 4, 3, 0.75, "cavity", 9)
    F = W.fourier_force(4, 4, 3, amplitude=1e-3, seed=2, dtype=np.float64)
    ref = oracle.adjoint(*args, 1, lid=[0.05, 0, 0], F=F)
    for K in (2, 4, 9, 20):
        got = oracle.adjoint(*args, K, lid=[0.05, 0, 0], F=F)
        assert got[0] == ref[0]
        assert np.array_equal(got[1], ref[1])
        assert np.array_equal(got[2], ref[2])


# --------------------------------------------------------------------------
# Per-face boundaries and obstacles (Sec. 4-5 workloads)

CHANNEL_FACES = ["periodic", "periodic", "wall", "wall", "periodic", "periodic"]


@pytest.mark.parametrize("lattice", ["d3q19", "d3q27"])
def test_symmetry_face_equals_mirrored_domain(lattice):
    """A free-slip symmetry face half a link above the last row gives exactly
    the lower half of the flow on the doubled, mirror-symmetric domain."""
    nx, m, nz = 9, 6, 5
    ny = 2 * m
    p0h, u0h = W.random_smooth_state(nx, m, nz, 3, amp_u=0.04, seed=3)
    p0h = p0h.reshape(nz, m, nx)
    u0h = u0h.reshape(3, nz, m, nx)
    p0 = np.concatenate([p0h, p0h[:, ::-1]], axis=1).ravel()
    u0 = np.concatenate([u0h, u0h[:, :, ::-1]], axis=2)
    u0[1, :, m:] *= -1
    F = np.zeros((3, nz, ny, nx))
    F[0] = 1e-5
    F[2] = -4e-6
    pf, uf = oracle.run(lattice, nx, ny, nz, 0.7, CHANNEL_FACES, 30, p0=p0,
                        u0=u0.reshape(3, -1), F=F.reshape(3, -1))
    half = ["periodic", "periodic", "wall", "symmetry", "periodic", "periodic"]
    ph, uh = oracle.run(lattice, nx, m, nz, 0.7, half, 30, p0=p0h.ravel(),
                        u0=u0h.reshape(3, -1), F=np.ascontiguousarray(F[:, :, :m]).reshape(3, -1))
    assert np.abs(uf.reshape(3, nz, ny, nx)[:, :, :m].reshape(3, -1) - uh).max() < 1e-15
    assert np.abs(pf.reshape(nz, ny, nx)[:, :m].ravel() - ph).max() < 1e-15


def test_solid_rows_equal_walls():
    """Rows of solid nodes bounce exactly like the walled faces of a channel."""
    nx, ny, nz = 7, 8, 5
    p0, u0 = W.random_smooth_state(nx, ny, nz, 3, amp_u=0.04, seed=4)
    F = W.fourier_force(nx, ny, nz, amplitude=1e-5, seed=2, dims=3)
    _, uw = oracle.run("d3q19", nx, ny, nz, 0.7, "channel", 25, p0=p0, u0=u0, F=F)
    P = np.full((nz, ny + 2, nx), 1 / 3)
    P[:, 1:-1] = p0.reshape(nz, ny, nx)
    U = np.zeros((3, nz, ny + 2, nx))
    U[:, :, 1:-1] = u0.reshape(3, nz, ny, nx)
    Fs = np.zeros((3, nz, ny + 2, nx))
    Fs[:, :, 1:-1] = F.reshape(3, nz, ny, nx)
    sol = np.zeros((nz, ny + 2, nx), np.uint8)
    sol[:, 0] = sol[:, -1] = 1
    ps, us = oracle.run("d3q19", nx, ny + 2, nz, 0.7, "periodic", 25, p0=P.ravel(),
                        u0=U.reshape(3, -1), F=Fs.reshape(3, -1), solid=sol)
    assert np.abs(us.reshape(3, nz, ny + 2, nx)[:, :, 1:-1].reshape(3, -1) - uw).max() < 1e-16
    # solid nodes report zero
    assert np.all(ps.reshape(nz, ny + 2, nx)[:, 0] == 0) and np.all(us[:, sol.ravel() != 0] == 0)


@pytest.mark.parametrize("lattice", ["d2q9", "d3q19", "d3q27"])
def test_obstacle_force_balances_momentum(lattice):
    """Momentum-exchange force: per step, the change of the fluid's total
    momentum equals the body force on the fluid minus the force on the
    obstacle (exactly, periodic box, stationary obstacle)."""
    Q, d = oracle.dims(lattice)
    nx, ny, nz = (16, 12, 1) if d == 2 else (12, 10, 8)
    sol = np.zeros((nz, ny, nx), np.uint8)
    if d == 2:
        sol[0, 4:7, 5:9] = 1
    else:
        sol[3:5, 4:7, 5:8] = 1
    fl = sol.ravel() == 0
    Fb = np.zeros((d, nx * ny * nz))
    Fb[0] = 1e-5
    Fb[1] = 3e-6
    p0, u0 = W.random_smooth_state(nx, ny, nz, d, amp_u=0.02, seed=5)
    u0[:, ~fl] = 0
    mom = []
    for k in (10, 11):
        _, u, Fo = oracle.run(lattice, nx, ny, nz, 0.8, "periodic", k, p0=p0, u0=u0, F=Fb,
                              solid=sol, want_force=True)
        mom.append(u[:, fl].sum(axis=1))
    change = mom[1] - mom[0]
    assert np.abs(change - (Fb[:, fl].sum(axis=1) - Fo[:d])).max() < 1e-14
    assert np.abs(Fo[:d]).max() > 1e-3  # the obstacle does take a force


@pytest.mark.parametrize("lattice", ["d2q9", "d3q19", "d3q27"])
def test_uniform_flow_through_open_faces_is_steady(lattice):
    """A uniform flow entering through a velocity inlet, leaving through a
    zero-gradient outflow, between free-slip planes, is an exact fixed point."""
    Q, d = oracle.dims(lattice)
    nx, ny, nz = (10, 6, 1) if d == 2 else (10, 6, 4)
    U0 = 0.05
    u0 = np.zeros((d, nx * ny * nz))
    u0[0] = U0
    inl = np.zeros((d, ny * nz))
    inl[0] = U0
    faces = ["inlet", "outflow", "symmetry", "symmetry", "periodic", "periodic"]
    p, u = oracle.run(lattice, nx, ny, nz, 0.7, faces, 20, u0=u0, inlet=inl)
    assert np.abs(u - u0).max() < 1e-15 and np.abs(p - 1 / 3).max() < 1e-15
    # a wrong inlet speed is not steady
    _, u = oracle.run(lattice, nx, ny, nz, 0.7, faces, 20, u0=u0, inlet=1.1 * inl)
    assert np.abs(u - u0).max() > 1e-4


def test_open_faces_are_axis_permutation_invariant():
    """The same inlet/outflow/wall/symmetry channel set up along x and along y
    (axes swapped, inlet profile re-indexed) gives the swapped fields."""
    nx, ny, nz = 14, 9, 6
    y, z = np.meshgrid(np.arange(ny), np.arange(nz), indexing="xy")
    prof = 0.04 * (y + 0.5) * (ny - 0.5 - y) / (ny / 2) ** 2 * (1 + 0.1 * np.sin(2 * np.pi * z / nz))
    inl = np.zeros((3, ny * nz))
    inl[0] = prof.ravel()
    fa = ["inlet", "outflow", "wall", "wall", "symmetry", "symmetry"]
    _, ua = oracle.run("d3q19", nx, ny, nz, 0.7, fa, 40, inlet=inl)
    # swapped: box (ny, nx, nz), inlet on -y, face nodes numbered (x, z)
    inl_b = np.zeros((3, ny * nz))
    inl_b[1] = prof.ravel()  # (x fastest, then z): x of b is y of a
    fb = ["wall", "wall", "inlet", "outflow", "symmetry", "symmetry"]
    _, ub = oracle.run("d3q19", ny, nx, nz, 0.7, fb, 40, inlet=inl_b)
    ua4 = ua.reshape(3, nz, ny, nx)
    ub4 = ub.reshape(3, nz, nx, ny)
    assert np.abs(ua4[0] - ub4[1].transpose(0, 2, 1)).max() < 1e-15
    assert np.abs(ua4[1] - ub4[0].transpose(0, 2, 1)).max() < 1e-15
    assert np.abs(ua4[2] - ub4[2].transpose(0, 2, 1)).max() < 1e-15
    assert np.abs(ua4[0]).max() > 0.01


def test_inflow_outflow_channel_develops_poiseuille():
    """Parabolic velocity inlet, pressure outlet, no-slip walls: the flux is
    the inlet's at every section, the mid-channel profile is the inlet
    parabola (within 1 %) and the pressure gradient is Poiseuille's,
    -dp/dx = 8 rho0 nu u_max / H^2 (within 2 %); the outlet holds p_out."""
    nx, ny, tau = 120, 16, 0.8
    nu = W.viscosity(tau)
    y = np.arange(ny)
    umax = 0.05
    prof = umax * (y + 0.5) * (ny - 0.5 - y) / (ny / 2) ** 2
    inl = np.zeros((2, ny))
    inl[0] = prof
    u0 = np.zeros((2, nx * ny))
    u0[0] = np.tile(prof[:, None], (1, nx)).ravel()
    faces = ["inlet", "outflow", "wall", "wall", "periodic", "periodic"]
    p, u = oracle.run("d2q9", nx, ny, 1, tau, faces, 8000, u0=u0, inlet=inl, p_outflow=0.33)
    U = u.reshape(2, ny, nx)
    P = p.reshape(ny, nx)
    flux = U[0].sum(axis=0)
    assert np.abs(flux / prof.sum() - 1).max() < 1e-4
    assert np.abs(U[0, :, nx // 2] - prof).max() < 0.01 * umax
    assert np.abs(U[1, :, nx // 2]).max() < 1e-3 * umax
    slope = (P[:, 40] - P[:, 80]).mean() / 40
    assert abs(slope / (8 * nu * umax / ny ** 2) - 1) < 0.02
    assert abs(P[:, -1].mean() - 0.33) < 0.01 * (P[:, 0].mean() - 0.33)


# --------------------------------------------------------------------------
# Sec. 2.2: the paper's modified nodal bounce-back (walls on the nodes)

NODAL_CHANNEL = ["periodic", "periodic", "nodal", "nodal", "periodic", "periodic"]


@pytest.mark.parametrize("lattice", ["d2q9", "d3q19", "d3q27"])
def test_nodal_couette_walls_on_the_nodes(lattice):
    """Moving top wall: the linear profile U y/(ny - 1) with u = 0 on the
    bottom row of nodes and u = U on the top row, for any tau (half-way
    bounce-back puts the walls half a link out instead)."""
    ny, U = 12, 0.02
    y = np.arange(ny)
    for tau in (0.6, 1.3):
        nu = W.viscosity(tau)
        _, u = oracle.run(lattice, 1, ny, 1, tau, NODAL_CHANNEL, int(30 * ny * ny / nu),
                          lid=[U, 0, 0])
        assert np.abs(u[0] - U * y / (ny - 1)).max() < 1e-10 * U
        assert np.abs(u[1:]).max() < 1e-12 * U


@pytest.mark.parametrize("lattice", ["d2q9", "d3q19"])
def test_nodal_poiseuille(lattice):
    """Body-force channel between nodal walls: exact second differences -G/nu
    and a parabola through the wall nodes up to a constant slip that depends
    on tau (as for BGK half-way bounce-back, but a different slip)."""
    ny, G = 14, 1e-6
    Q, d = oracle.dims(lattice)
    y = np.arange(ny)
    slips = []
    for tau in (0.6, 0.8, 1.2):
        nu = W.viscosity(tau)
        F = np.zeros((d, ny))
        F[0] = G
        _, u = oracle.run(lattice, 1, ny, 1, tau, NODAL_CHANNEL, int(30 * ny * ny / nu), F=F)
        ux = u[0]
        d2 = ux[2:] - 2 * ux[1:-1] + ux[:-2]
        assert np.abs(d2 * nu / G + 1).max() < 1e-8
        par = G / (2 * nu) * y * (ny - 1 - y)
        slip = ux - par
        assert np.abs(slip - slip.mean()).max() < 1e-9 * par.max()
        slips.append(slip.mean() / par.max())
        _, uh = oracle.run(lattice, 1, ny, 1, tau, "channel", int(30 * ny * ny / nu), F=F)
        assert np.abs(uh[0] - ux).max() > 1e-3 * par.max()  # not half-way bounce-back
    assert 0 < slips[0] < slips[1] < slips[2] < 0.05


def test_nodal_wall_with_symmetry_equals_mirrored_channel():
    """A nodal wall below and a symmetry face above give the lower half of the
    nodal channel of twice the height (mirror plane half a link above)."""
    nx, m, nz = 7, 6, 5
    ny = 2 * m
    p0h, u0h = W.random_smooth_state(nx, m, nz, 3, amp_u=0.03, seed=6)
    p0h = p0h.reshape(nz, m, nx)
    u0h = u0h.reshape(3, nz, m, nx)
    p0 = np.concatenate([p0h, p0h[:, ::-1]], axis=1).ravel()
    u0 = np.concatenate([u0h, u0h[:, :, ::-1]], axis=2)
    u0[1, :, m:] *= -1
    _, uf = oracle.run("d3q19", nx, ny, nz, 0.7, NODAL_CHANNEL, 25, p0=p0, u0=u0.reshape(3, -1))
    half = ["periodic", "periodic", "nodal", "symmetry", "periodic", "periodic"]
    _, uh = oracle.run("d3q19", nx, m, nz, 0.7, half, 25, p0=p0h.ravel(), u0=u0h.reshape(3, -1))
    assert np.abs(uf.reshape(3, nz, ny, nx)[:, :, :m].reshape(3, -1) - uh).max() < 1e-15
