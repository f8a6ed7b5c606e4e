"""FP64 CPU oracle for the IMEXLBM per-step update (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path never does: the CUDA
library and its Python binding share no code with it.

``oracle.c`` holds the arithmetic (see its header for the paper sections it
follows); this module only compiles it with gcc and marshals numpy arrays
through ctypes.  Every array crossing the interface is FP64, structure of
arrays (component-major), node index ``n = x + nx*(y + ny*z)``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

D2Q9, D3Q19, D3Q27 = 0, 1, 2
BC_PERIODIC, BC_CAVITY, BC_CHANNEL = 0, 1, 2
_LATTICE_NAMES = {"d2q9": D2Q9, "d3q19": D3Q19, "d3q27": D3Q27}
_BC_NAMES = {"periodic": BC_PERIODIC, "cavity": BC_CAVITY, "channel": BC_CHANNEL}
FACE_PERIODIC, FACE_WALL, FACE_INLET, FACE_OUTFLOW, FACE_SYMMETRY, FACE_NODAL = 0, 1, 2, 3, 4, 5
_FACE_NAMES = {"periodic": FACE_PERIODIC, "wall": FACE_WALL, "inlet": FACE_INLET,
               "outflow": FACE_OUTFLOW, "symmetry": FACE_SYMMETRY, "nodal": FACE_NODAL}

_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", _LIB, _SRC, "-lm"]
        subprocess.check_call(cmd)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.or_tables.argtypes = [ctypes.c_int, ip, ip, ip, dp, ip]
        lib.or_equilibrium.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_double, dp, dp]
        lib.or_collide_node.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                        ctypes.c_double, dp, dp, dp, ctypes.c_double, dp]
        lib.or_run.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                               ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                               dp, dp, dp, dp, ctypes.c_long, dp, dp, dp, ctypes.c_int,
                               ctypes.c_double, dp]
        lib.or_adjoint.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_double, ctypes.c_int, ctypes.c_double, dp, dp, dp,
                                   dp, ctypes.c_long, ctypes.c_long, dp, dp, dp, ctypes.c_int]
        up = ctypes.POINTER(ctypes.c_ubyte)
        lib.or_run_faces.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_double, ip, ctypes.c_int, ctypes.c_double,
                                     dp, dp, up, dp, dp, dp, ctypes.c_double, ctypes.c_long,
                                     dp, dp, dp, dp, ctypes.c_int, ctypes.c_double, dp]
        for f in (lib.or_tables, lib.or_equilibrium, lib.or_collide_node, lib.or_run,
                  lib.or_adjoint, lib.or_run_faces):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, n=None):
    if a is None:
        return None
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def _lat(lattice):
    return _LATTICE_NAMES[lattice] if isinstance(lattice, str) else int(lattice)


def _bc(bc):
    return _BC_NAMES[bc] if isinstance(bc, str) else int(bc)


def dims(lattice) -> tuple[int, int]:
    """(Q, d) of a velocity set."""
    lat = _lat(lattice)
    return {D2Q9: (9, 2), D3Q19: (19, 3), D3Q27: (27, 3)}[lat]


def tables(lattice):
    """Velocity set (Sec. 2.1): e (Q x 3 ints), t (Q), opposite index (Q)."""
    lib = _load()
    Q, d = ctypes.c_int(), ctypes.c_int()
    e = np.zeros(27 * 3, dtype=np.int32)
    t = np.zeros(27)
    opp = np.zeros(27, dtype=np.int32)
    rc = lib.or_tables(_lat(lattice), ctypes.byref(Q), ctypes.byref(d),
                       e.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(t),
                       opp.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    if rc != 0:
        raise ValueError("bad lattice")
    q = Q.value
    return e[: 3 * q].reshape(q, 3).copy(), t[:q].copy(), opp[:q].copy()


def equilibrium(lattice, P, u, rho0=1.0, compressible=False):
    """One node's equilibrium, Eq. (incompressible_feq) or Eq. (feq)."""
    lib = _load()
    Q, _ = dims(lattice)
    out = np.zeros(Q)
    u3 = np.zeros(3)
    u3[: len(u)] = u
    rc = lib.or_equilibrium(_lat(lattice), int(bool(compressible)), float(rho0), float(P),
                            _dp(u3), _dp(out))
    assert rc == 0
    return out


def _mrt3(mrt):
    """(s_bulk, s_even, s_odd) of the multiple-relaxation-time collision, or None."""
    if mrt is None:
        return None
    return _f64(np.asarray(mrt, float), 3)


def collide_node(lattice, f, tau, rho0=1.0, compressible=False, F=None, trt_lambda=None,
                 mrt=None):
    """Eq. (collision) at one node (with the Guo source when F is given).

    ``trt_lambda`` selects the two-relaxation-time collision with that magic
    parameter instead of BGK; ``mrt = (s_bulk, s_even, s_odd)`` the
    multiple-relaxation-time collision (stress moments at 1/tau)."""
    lib = _load()
    Q, _ = dims(lattice)
    f = _f64(f, Q)
    out = np.zeros(Q)
    F3 = None
    if F is not None:
        F3 = np.zeros(3)
        F3[: len(F)] = F
    rc = lib.or_collide_node(_lat(lattice), float(tau), int(bool(compressible)), float(rho0),
                             _dp(f), _dp(F3), _dp(out), float(trt_lambda or 0.0),
                             _dp(_mrt3(mrt)))
    assert rc == 0
    return out


def faces_of(bc):
    """Six face types (-x, +x, -y, +y, -z, +z) from names or ints."""
    out = [(_FACE_NAMES[f] if isinstance(f, str) else int(f)) for f in bc]
    if len(out) != 6:
        raise ValueError("six face types expected")
    return out


def run(lattice, nx, ny, nz, tau, bc, steps, *, rho0=1.0, compressible=False, lid=None,
        F=None, p0=None, u0=None, want_f=False, threads=0, trt_lambda=None, solid=None,
        inlet=None, want_force=False, p_outflow=1.0 / 3.0, mrt=None):
    """Forward run of Sec. 3.1's loop for ``steps`` steps.

    Returns ``(p, u)`` (or ``(p, u, f)``): p shape (N,), u shape (d, N),
    f shape (Q, N) post-propagation.  ``threads=0`` leaves OpenMP's default.
    ``trt_lambda`` selects the two-relaxation-time collision, ``mrt = (s_bulk,
    s_even, s_odd)`` the multiple-relaxation-time collision.

    ``bc`` is "periodic", "cavity", "channel" or a sequence of six face
    types ("periodic", "wall", "inlet", "outflow", "symmetry", "nodal"; order -x, +x,
    -y, +y, -z, +z).  ``solid``: N bytes, nonzero = obstacle node.
    ``inlet``: inlet velocity, shape (d, face nodes), the face's nodes
    numbered by its two remaining axes, lower axis fastest.  ``p_outflow``:
    the pressure p = c_s^2 P held at outflow faces.  With
    ``want_force`` the momentum-exchange force on the obstacles during the
    last step (3,) is appended to the result.
    """
    if not isinstance(bc, str) or solid is not None or inlet is not None or want_force:
        return _run_faces(lattice, nx, ny, nz, tau, bc, steps, rho0=rho0,
                          compressible=compressible, lid=lid, F=F, p0=p0, u0=u0, want_f=want_f,
                          threads=threads, trt_lambda=trt_lambda, solid=solid, inlet=inlet,
                          want_force=want_force, p_outflow=p_outflow, mrt=mrt)
    lib = _load()
    Q, d = dims(lattice)
    N = nx * ny * nz
    lid3 = None if lid is None else _f64(np.pad(np.asarray(lid, float), (0, 3 - len(lid))))
    F = _f64(F, d * N)
    p0 = _f64(p0, N)
    u0 = _f64(u0, d * N)
    p = np.zeros(N)
    u = np.zeros(d * N)
    f = np.zeros(Q * N) if want_f else None
    rc = lib.or_run(_lat(lattice), nx, ny, nz, float(tau), _bc(bc), int(bool(compressible)),
                    float(rho0), _dp(lid3), _dp(F), _dp(p0), _dp(u0), int(steps), _dp(p),
                    _dp(u), _dp(f), int(threads), float(trt_lambda or 0.0), _dp(_mrt3(mrt)))
    if rc != 0:
        raise ValueError(f"or_run failed with status {rc}")
    u = u.reshape(d, N)
    if want_f:
        return p, u, f.reshape(Q, N)
    return p, u


def _run_faces(lattice, nx, ny, nz, tau, bc, steps, *, rho0, compressible, lid, F, p0, u0,
               want_f, threads, trt_lambda, solid, inlet, want_force, p_outflow, mrt=None):
    lib = _load()
    Q, d = dims(lattice)
    N = nx * ny * nz
    if isinstance(bc, str):
        named = {"periodic": ["periodic"] * 6, "cavity": ["wall"] * 6,
                 "channel": ["periodic", "periodic", "wall", "wall", "periodic", "periodic"]}
        bc = named[bc]
    faces = (ctypes.c_int * 6)(*faces_of(bc))
    lid3 = None if lid is None else _f64(np.pad(np.asarray(lid, float), (0, 3 - len(lid))))
    F = _f64(F, d * N)
    p0 = _f64(p0, N)
    u0 = _f64(u0, d * N)
    sol = None
    if solid is not None:
        sol = np.ascontiguousarray(np.asarray(solid).ravel() != 0, dtype=np.uint8)
        if sol.size != N:
            raise ValueError("solid needs N values")
    inl = None if inlet is None else np.ascontiguousarray(np.asarray(inlet, np.float64).ravel())
    p = np.zeros(N)
    u = np.zeros(d * N)
    f = np.zeros(Q * N) if want_f else None
    force = np.zeros(3) if want_force else None
    rc = lib.or_run_faces(_lat(lattice), nx, ny, nz, float(tau), faces, int(bool(compressible)),
                          float(rho0), _dp(lid3), _dp(F),
                          None if sol is None else sol.ctypes.data_as(
                              ctypes.POINTER(ctypes.c_ubyte)),
                          _dp(inl), _dp(p0), _dp(u0), float(p_outflow), int(steps), _dp(p),
                          _dp(u), _dp(f),
                          _dp(force), int(threads), float(trt_lambda or 0.0), _dp(_mrt3(mrt)))
    if rc != 0:
        raise ValueError(f"or_run_faces failed with status {rc}")
    out = [p, u.reshape(d, N)]
    if want_f:
        out.append(f.reshape(Q, N))
    if want_force:
        out.append(force)
    return tuple(out)


def adjoint(lattice, nx, ny, nz, tau, bc, T, K, *, rho0=1.0, lid=None, F=None, p0=None,
            u0=None, threads=0):
    """J = rho0/2 sum |u(T)|^2 and its gradients (dJ/dF shape (d, N), dJ/dU shape (3,))."""
    lib = _load()
    Q, d = dims(lattice)
    N = nx * ny * nz
    lid3 = None if lid is None else _f64(np.pad(np.asarray(lid, float), (0, 3 - len(lid))))
    F = _f64(F, d * N)
    p0 = _f64(p0, N)
    u0 = _f64(u0, d * N)
    J = np.zeros(1)
    gF = np.zeros(d * N)
    gU = np.zeros(3)
    rc = lib.or_adjoint(_lat(lattice), nx, ny, nz, float(tau), _bc(bc), float(rho0), _dp(lid3),
                        _dp(F), _dp(p0), _dp(u0), int(T), int(K), _dp(J), _dp(gF), _dp(gU),
                        int(threads))
    if rc != 0:
        raise ValueError(f"or_adjoint failed with status {rc}")
    return float(J[0]), gF.reshape(d, N), gU
