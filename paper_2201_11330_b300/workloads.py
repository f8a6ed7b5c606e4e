"""Seeded synthetic inputs for the lattice-Boltzmann hot path.

This module holds workload definitions only: initial pressure/velocity
fields, body-force fields and case parameters.  It contains none of the
method's arithmetic (no equilibrium, collision, streaming or moments), so the
CUDA path and the FP64 oracle can both be fed from it.  Everything is numpy
FP64, structure of arrays (component-major), node index n = x + nx*(y + ny*z).

Workloads (all synthetic; the paper's own geometries are out of scope):
  * lid-driven cavity: uniform rest state p = 1/3 (P = sum f = 1), u = 0, lid
    on the +y face moving in +x; tau from Re = U L / nu with nu = (tau - 1/2)/3.
  * 2D Taylor-Green vortex on a periodic box.
  * periodic box driven by a smooth seeded body force built from the four
    lowest Fourier modes per axis.
  * random smooth perturbations for parity tests.
"""
from __future__ import annotations

import math

import numpy as np

CS2 = 1.0 / 3.0


def tau_from_re(re: float, u: float, length: float) -> float:
    """Standard BGK relaxation time for Reynolds number re = u*length/nu."""
    nu = u * length / re
    return nu / CS2 + 0.5


def tau_from_paper(tau_paper: float) -> float:
    """The paper's tau (omega = 1/(tau + 1/2)) expressed as the standard tau."""
    return tau_paper + 0.5


def viscosity(tau: float) -> float:
    """Kinematic viscosity nu = c_s^2 (tau - 1/2) of the standard tau."""
    return CS2 * (tau - 0.5)


def grid(nx: int, ny: int, nz: int = 1):
    """Node coordinates (x, y, z) as flat FP64 arrays in node order."""
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    return x.ravel(), y.ravel(), z.ravel()


def taylor_green_2d(nx: int, ny: int, u0: float, rho0: float = 1.0, P0: float = 1.0):
    """Initial (p, u) of the 2D Taylor-Green vortex on a periodic nx x ny box.

    u_x = -u0 cos(kx x) sin(ky y), u_y = u0 (kx/ky) sin(kx x) cos(ky y),
    p = c_s^2 P0 - rho0 u0^2/4 (cos 2 kx x + (kx/ky)^2 cos 2 ky y).
    Returns p shape (N,), u shape (2, N).
    """
    kx, ky = 2 * math.pi / nx, 2 * math.pi / ny
    x, y, _ = grid(nx, ny, 1)
    ux = -u0 * np.cos(kx * x) * np.sin(ky * y)
    uy = u0 * (kx / ky) * np.sin(kx * x) * np.cos(ky * y)
    p = CS2 * P0 - rho0 * u0 * u0 / 4.0 * (np.cos(2 * kx * x) + (kx / ky) ** 2 * np.cos(2 * ky * y))
    return p, np.stack([ux, uy])


def taylor_green_rate(nx: int, ny: int, tau: float) -> float:
    """Analytic decay rate of the Taylor-Green velocity amplitude, nu (kx^2 + ky^2)."""
    kx, ky = 2 * math.pi / nx, 2 * math.pi / ny
    return viscosity(tau) * (kx * kx + ky * ky)


def fourier_force(nx: int, ny: int, nz: int, amplitude: float = 1e-5, seed: int = 2201,
                  modes: int = 4, dims: int = 3, dtype=np.float32):
    """Smooth periodic body force from the `modes` lowest Fourier modes per axis.

    F_c = A * sum_{m=1..modes} sum_{axis} [a cos(2 pi m x_axis/L) + b sin(...)],
    a, b ~ N(0, 1) from numpy.random.default_rng(seed), rescaled so that
    max |F_c| over the box and components equals `amplitude`.  Returned in
    `dtype` (FP32 by default, the force field's storage type) as shape (dims, N).
    """
    rng = np.random.default_rng(seed)
    x, y, z = grid(nx, ny, nz)
    coords = (x, y, z)
    lengths = (nx, ny, nz)
    out = np.zeros((dims, nx * ny * nz))
    for c in range(dims):
        for m in range(1, modes + 1):
            for ax in range(3 if nz > 1 else 2):
                a, b = rng.standard_normal(2)
                ph = 2 * math.pi * m * coords[ax] / lengths[ax]
                out[c] += a * np.cos(ph) + b * np.sin(ph)
    scale = np.abs(out).max()
    if scale > 0:
        out *= amplitude / scale
    return out.astype(dtype)


def random_smooth_state(nx: int, ny: int, nz: int, dims: int, amp_u: float = 0.05,
                        amp_p: float = 1e-3, seed: int = 7):
    """Random smooth (p, u) fields for parity tests: low Fourier modes, seeded."""
    rng = np.random.default_rng(seed)
    x, y, z = grid(nx, ny, nz)
    coords = (x, y, z)
    lengths = (nx, ny, nz)
    axes = 3 if nz > 1 else 2

    def field():
        acc = np.zeros(nx * ny * nz)
        for m in range(1, 3):
            for ax in range(axes):
                a, b = rng.standard_normal(2)
                ph = 2 * math.pi * m * coords[ax] / lengths[ax]
                acc += a * np.cos(ph) + b * np.sin(ph)
        return acc / max(np.abs(acc).max(), 1e-300)

    u = np.stack([amp_u * field() for _ in range(dims)])
    p = CS2 + amp_p * field()
    return p, u


def cavity_params(n: int, re: float, lid_u: float = 0.1):
    """Lid-driven cavity of side n (walls half a spacing outside the nodes)."""
    return {"tau": tau_from_re(re, lid_u, n), "lid": (lid_u, 0.0, 0.0)}
