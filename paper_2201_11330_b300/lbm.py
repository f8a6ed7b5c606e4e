"""Python binding of the C ABI in include/lbm.h (ctypes, argument marshalling only).

Every step of the hot path runs in liblbm.so's CUDA kernels; this module only
converts arguments.  PyTorch provides device memory (the workspace and the
field tensors) and the current CUDA stream.  There is no CPU fallback: if the
library is missing or no GPU is present, the calls raise.

Two layers:
  * module functions with the C names (lbm_create, lbm_init, lbm_step, ...),
    taking plain ints / pointers, and
  * ``Lattice``, a small owner object that allocates the workspace with torch
    and calls those functions.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbm.so")

LBM_OK, LBM_ERR_ARG, LBM_ERR_CUDA, LBM_ERR_UNSTABLE, LBM_ERR_STATE, LBM_ERR_NOMEM = 0, -1, -2, -3, -4, -5
LBM_D2Q9, LBM_D3Q19, LBM_D3Q27 = 0, 1, 2
LBM_BC_PERIODIC, LBM_BC_CAVITY, LBM_BC_CHANNEL, LBM_BC_FACES = 0, 1, 2, 3
LBM_FACE_PERIODIC, LBM_FACE_WALL, LBM_FACE_INLET, LBM_FACE_OUTFLOW = 0, 1, 2, 3
LBM_FACE_SYMMETRY, LBM_FACE_NODAL = 4, 5
FACES = {"periodic": LBM_FACE_PERIODIC, "wall": LBM_FACE_WALL, "inlet": LBM_FACE_INLET,
         "outflow": LBM_FACE_OUTFLOW, "symmetry": LBM_FACE_SYMMETRY, "nodal": LBM_FACE_NODAL}
LBM_F64, LBM_F32, LBM_F16S, LBM_BF16S = 0, 1, 2, 3
LBM_COLL_BGK, LBM_COLL_TRT, LBM_COLL_MRT = 0, 1, 2
LBM_KERNEL_AUTO, LBM_KERNEL_PLAIN, LBM_KERNEL_PAIRED = 0, 1, 3
KERNELS = {"auto": LBM_KERNEL_AUTO, "plain": LBM_KERNEL_PLAIN,
           "paired": LBM_KERNEL_PAIRED}

LATTICES = {"d2q9": LBM_D2Q9, "d3q19": LBM_D3Q19, "d3q27": LBM_D3Q27}
BCS = {"periodic": LBM_BC_PERIODIC, "cavity": LBM_BC_CAVITY, "channel": LBM_BC_CHANNEL}
STORAGES = {"f64": LBM_F64, "f32": LBM_F32, "f16s": LBM_F16S, "bf16s": LBM_BF16S}
QD = {LBM_D2Q9: (9, 2), LBM_D3Q19: (19, 3), LBM_D3Q27: (27, 3)}

# Every extern "C" symbol include/lbm.h declares.
EXPORTS = [
    "lbm_default_opts", "lbm_tau_from_paper", "lbm_workspace_bytes", "lbm_create",
    "lbm_set_stream", "lbm_init", "lbm_init_f32", "lbm_set_force", "lbm_set_lid", "lbm_set_geometry",
    "lbm_set_inlet", "lbm_step_force", "lbm_set_graph_steps", "lbm_step",
    "lbm_step_count", "lbm_set_kernel_variant", "lbm_kernel_variant_in_use",
    "lbm_step_reduce", "lbm_macroscopic", "lbm_reduce", "lbm_state_bytes", "lbm_get_state",
    "lbm_set_state", "lbm_adjoint_workspace_bytes", "lbm_adjoint_forward",
    "lbm_adjoint_backward", "lbm_adjoint", "lbm_reduce_state_noalloc", "lbm_error_string",
    "lbm_destroy",
]


class lbm_opts(ctypes.Structure):
    _fields_ = [("storage", ctypes.c_int), ("aa", ctypes.c_int), ("compressible", ctypes.c_int),
                ("f32_unshifted", ctypes.c_int), ("rho0", ctypes.c_double),
                ("lid_u", ctypes.c_double * 3), ("has_force", ctypes.c_int),
                ("collision", ctypes.c_int), ("trt_lambda", ctypes.c_double),
                ("faces", ctypes.c_int * 6), ("geometry", ctypes.c_int),
                ("p_outflow", ctypes.c_double), ("mrt_bulk", ctypes.c_double),
                ("mrt_even", ctypes.c_double), ("mrt_odd", ctypes.c_double)]


class LBMError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {lbm_error_string(status)} (status {status})")
        self.status = status


_lib = None
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_i64 = ctypes.c_int64
_sz = ctypes.c_size_t


def load():
    """Load liblbm.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"{LIB_PATH} is missing: build it with `python -m paper_2201_11330_b300.build`")
    lib = ctypes.CDLL(LIB_PATH)
    ip = ctypes.c_int
    op = ctypes.POINTER(lbm_opts)
    sig = {
        "lbm_default_opts": (None, [op]),
        "lbm_tau_from_paper": (ctypes.c_double, [ctypes.c_double]),
        "lbm_workspace_bytes": (_sz, [ip, ip, ip, ip, op]),
        "lbm_create": (ip, [ip, ip, ip, ip, ctypes.c_double, ip, op, _vp, _sz, _vp,
                            ctypes.POINTER(_vp)]),
        "lbm_set_stream": (ip, [_vp, _vp]),
        "lbm_init": (ip, [_vp, _vp, _vp]),
        "lbm_init_f32": (ip, [_vp, _vp, _vp]),
        "lbm_set_force": (ip, [_vp, _vp]),
        "lbm_set_lid": (ip, [_vp, _dp]),
        "lbm_set_geometry": (ip, [_vp, _vp]),
        "lbm_set_inlet": (ip, [_vp, _vp]),
        "lbm_step_force": (ip, [_vp, _i64, _dp]),
        "lbm_set_graph_steps": (ip, [_vp, ip]),
        "lbm_step": (ip, [_vp, _i64]),
        "lbm_step_count": (_i64, [_vp]),
        "lbm_set_kernel_variant": (ip, [_vp, ip]),
        "lbm_kernel_variant_in_use": (ip, [_vp]),
        "lbm_macroscopic": (ip, [_vp, _vp, _vp, ip]),
        "lbm_reduce": (ip, [_vp, _dp]),
        "lbm_step_reduce": (ip, [_vp, _i64, _dp]),
        "lbm_state_bytes": (_sz, [_vp]),
        "lbm_get_state": (ip, [_vp, _vp, ctypes.POINTER(_i64)]),
        "lbm_set_state": (ip, [_vp, _vp, _i64]),
        "lbm_adjoint_workspace_bytes": (_sz, [_vp, _i64, _i64]),
        "lbm_adjoint_forward": (ip, [_vp, _i64, _i64, _vp, _sz, _dp]),
        "lbm_adjoint_backward": (ip, [_vp, _vp, _sz, _vp, _dp]),
        "lbm_adjoint": (ip, [_vp, _i64, _i64, _vp, _sz, _dp, _vp, _dp]),
        "lbm_reduce_state_noalloc": (ip, [ip, ip, ip, ip, ip, op, _vp, _i64, _vp, _vp, _dp]),
        "lbm_error_string": (ctypes.c_char_p, [ip]),
        "lbm_destroy": (None, [_vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


# ---- C names, marshalling only -------------------------------------------------

def lbm_default_opts() -> lbm_opts:
    o = lbm_opts()
    load().lbm_default_opts(ctypes.byref(o))
    return o


def lbm_tau_from_paper(tau_paper: float) -> float:
    return load().lbm_tau_from_paper(tau_paper)


def lbm_workspace_bytes(lattice: int, nx: int, ny: int, nz: int, opts: lbm_opts) -> int:
    return load().lbm_workspace_bytes(lattice, nx, ny, nz, ctypes.byref(opts))


def lbm_create(lattice, nx, ny, nz, tau, bc, opts, workspace_ptr, nbytes, stream_ptr):
    ctx = _vp()
    rc = load().lbm_create(lattice, nx, ny, nz, tau, bc, ctypes.byref(opts), workspace_ptr,
                           nbytes, stream_ptr, ctypes.byref(ctx))
    _check(rc, "lbm_create")
    return ctx


def lbm_set_stream(ctx, stream_ptr):
    _check(load().lbm_set_stream(ctx, stream_ptr), "lbm_set_stream")


def lbm_init(ctx, p_ptr, u_ptr):
    _check(load().lbm_init(ctx, p_ptr, u_ptr), "lbm_init")


def lbm_init_f32(ctx, p_ptr, u_ptr):
    _check(load().lbm_init_f32(ctx, p_ptr, u_ptr), "lbm_init_f32")


def lbm_set_force(ctx, force_ptr):
    _check(load().lbm_set_force(ctx, force_ptr), "lbm_set_force")


def lbm_set_lid(ctx, lid3):
    arr = (ctypes.c_double * 3)(*[float(v) for v in lid3])
    _check(load().lbm_set_lid(ctx, arr), "lbm_set_lid")


def lbm_set_geometry(ctx, solid_ptr):
    _check(load().lbm_set_geometry(ctx, solid_ptr), "lbm_set_geometry")


def lbm_set_inlet(ctx, u_ptr):
    _check(load().lbm_set_inlet(ctx, u_ptr), "lbm_set_inlet")


def lbm_step_force(ctx, n: int):
    out = (ctypes.c_double * 3)()
    _check(load().lbm_step_force(ctx, int(n), out), "lbm_step_force")
    return list(out)


def lbm_set_graph_steps(ctx, steps: int):
    _check(load().lbm_set_graph_steps(ctx, int(steps)), "lbm_set_graph_steps")


def lbm_step(ctx, n: int):
    _check(load().lbm_step(ctx, int(n)), "lbm_step")


def lbm_step_count(ctx) -> int:
    return load().lbm_step_count(ctx)


def lbm_set_kernel_variant(ctx, variant: int):
    _check(load().lbm_set_kernel_variant(ctx, int(variant)), "lbm_set_kernel_variant")


def lbm_kernel_variant_in_use(ctx) -> int:
    return load().lbm_kernel_variant_in_use(ctx)


def lbm_macroscopic(ctx, p_ptr, u_ptr, out_dtype: int):
    _check(load().lbm_macroscopic(ctx, p_ptr, u_ptr, out_dtype), "lbm_macroscopic")


def lbm_reduce(ctx):
    out = (ctypes.c_double * 6)()
    _check(load().lbm_reduce(ctx, out), "lbm_reduce")
    return list(out)


def lbm_step_reduce(ctx, n: int):
    out = (ctypes.c_double * 6)()
    _check(load().lbm_step_reduce(ctx, int(n), out), "lbm_step_reduce")
    return list(out)


def lbm_state_bytes(ctx) -> int:
    return load().lbm_state_bytes(ctx)


def lbm_get_state(ctx, dst_ptr) -> int:
    step = _i64()
    _check(load().lbm_get_state(ctx, dst_ptr, ctypes.byref(step)), "lbm_get_state")
    return step.value


def lbm_set_state(ctx, src_ptr, step: int):
    _check(load().lbm_set_state(ctx, src_ptr, int(step)), "lbm_set_state")


def lbm_adjoint_workspace_bytes(ctx, T: int, K: int) -> int:
    return load().lbm_adjoint_workspace_bytes(ctx, int(T), int(K))


def lbm_adjoint_forward(ctx, T, K, ws_ptr, nbytes) -> float:
    J = ctypes.c_double()
    _check(load().lbm_adjoint_forward(ctx, int(T), int(K), ws_ptr, nbytes, ctypes.byref(J)),
           "lbm_adjoint_forward")
    return J.value


def lbm_adjoint_backward(ctx, ws_ptr, nbytes, dJdF_ptr):
    gU = (ctypes.c_double * 3)()
    _check(load().lbm_adjoint_backward(ctx, ws_ptr, nbytes, dJdF_ptr, gU), "lbm_adjoint_backward")
    return list(gU)


def lbm_adjoint(ctx, T, K, ws_ptr, nbytes, dJdF_ptr):
    J = ctypes.c_double()
    gU = (ctypes.c_double * 3)()
    _check(load().lbm_adjoint(ctx, int(T), int(K), ws_ptr, nbytes, ctypes.byref(J), dJdF_ptr, gU),
           "lbm_adjoint")
    return J.value, list(gU)


def lbm_reduce_state_noalloc(lattice, nx, ny, nz, bc, opts, state_ptr, step, force_ptr,
                             stream_ptr):
    """Monitor reduction of a state buffer without any device allocation
    (for callers that may not allocate; see include/lbm.h)."""
    out = (ctypes.c_double * 6)()
    _check(load().lbm_reduce_state_noalloc(lattice, nx, ny, nz, bc, ctypes.byref(opts), state_ptr,
                                           int(step), force_ptr, stream_ptr, out),
           "lbm_reduce_state_noalloc")
    return list(out)


def lbm_error_string(status: int) -> str:
    return load().lbm_error_string(int(status)).decode()


def lbm_destroy(ctx):
    load().lbm_destroy(ctx)


def _check(rc: int, where: str):
    if rc != LBM_OK:
        raise LBMError(rc, where)


# ---- owner object ----------------------------------------------------------------

def _key(table, v):
    return table[v] if isinstance(v, str) else int(v)


class Lattice:
    """A simulation context whose workspace is a torch tensor on `device`.

    Fields exchanged with it are torch tensors on the same device: pressure
    (N,), velocity (d, N) in FP64 (or FP32 for outputs on request), force
    (d, N) in FP32.  Calls launch on torch's current stream.

    ``bc`` is "periodic", "cavity", "channel" or six face types ("periodic",
    "wall", "inlet", "outflow", "symmetry", "nodal"; order -x, +x, -y, +y,
    -z, +z).
    ``obstacles=True`` reserves the link words for ``set_geometry``.
    ``mrt=(s_bulk, s_even, s_odd)`` selects the multiple-relaxation-time
    collision with those rates (0 = 1/tau).
    """

    def __init__(self, lattice, nx, ny, nz, tau, bc, *, storage="f32", aa=False,
                 compressible=False, f32_unshifted=False, rho0=1.0, lid=(0.0, 0.0, 0.0),
                 has_force=False, kernel="auto", trt_lambda=None, obstacles=False,
                 p_outflow=1.0 / 3.0, mrt=None, device="cuda"):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the LBM library needs a CUDA device")
        self.torch = torch
        self.lattice = _key(LATTICES, lattice)
        self.Q, self.d = QD[self.lattice]
        self.shape = (int(nx), int(ny), int(nz))
        self.N = int(nx) * int(ny) * int(nz)
        self.tau = float(tau)
        o = lbm_default_opts()
        if isinstance(bc, (str, int)):
            self.bc = _key(BCS, bc)
        else:  # six face types
            faces = [_key(FACES, f) for f in bc]
            if len(faces) != 6:
                raise ValueError("six face types expected")
            for i, f in enumerate(faces):
                o.faces[i] = f
            self.bc = LBM_BC_FACES
        self.faces = [o.faces[i] for i in range(6)]
        o.geometry = int(bool(obstacles))
        o.p_outflow = float(p_outflow)
        self.device = torch.device(device)
        o.storage = _key(STORAGES, storage)
        o.aa = int(bool(aa))
        o.compressible = int(bool(compressible))
        o.f32_unshifted = int(bool(f32_unshifted))
        o.rho0 = float(rho0)
        lid = list(lid) + [0.0] * (3 - len(lid))
        for k in range(3):
            o.lid_u[k] = float(lid[k])
        o.has_force = int(bool(has_force))
        if trt_lambda is not None:  # two-relaxation-time collision
            o.collision = LBM_COLL_TRT
            o.trt_lambda = float(trt_lambda)
        if mrt is not None:  # multiple relaxation times: (bulk, even, odd) rates
            o.collision = LBM_COLL_MRT
            o.mrt_bulk, o.mrt_even, o.mrt_odd = (float(r) for r in mrt)
        self.opts = o
        nbytes = lbm_workspace_bytes(self.lattice, nx, ny, nz, o)
        if nbytes == 0:
            raise LBMError(LBM_ERR_ARG, "lbm_workspace_bytes")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.ctx = lbm_create(self.lattice, nx, ny, nz, self.tau, self.bc, o,
                              self.workspace.data_ptr(), nbytes, self._stream())
        self._force = None
        self._inlet = None
        self._adj_ws = None
        if kernel != "auto":
            self.set_kernel(kernel)

    def _stream(self):
        return self.torch.cuda.current_stream(self.device).cuda_stream

    def _sync_stream(self):
        lbm_set_stream(self.ctx, self._stream())

    def _dev(self, t, dtype, numel):
        torch = self.torch
        t = torch.as_tensor(t, dtype=dtype, device=self.device).contiguous()
        if t.numel() != numel:
            raise ValueError(f"expected {numel} values, got {t.numel()}")
        return t

    def init(self, p=None, u=None):
        """f = feq(p, u) (Sec. 2.2); p (N,) and u (d, N), None = 1/3 and 0.
        FP32 tensors (both, or the one given) go through lbm_init_f32, anything
        else is taken as FP64."""
        torch = self.torch
        self._sync_stream()
        given = [t for t in (p, u) if t is not None]
        f32 = bool(given) and all(isinstance(t, torch.Tensor) and t.dtype == torch.float32
                                  for t in given)
        dt = torch.float32 if f32 else torch.float64
        pt = None if p is None else self._dev(p, dt, self.N)
        ut = None if u is None else self._dev(u, dt, self.d * self.N)
        (lbm_init_f32 if f32 else lbm_init)(self.ctx, None if pt is None else pt.data_ptr(),
                                            None if ut is None else ut.data_ptr())
        # keep the inputs alive until the init kernel has consumed them
        self._init_inputs = (pt, ut)
        return self

    def set_force(self, F):
        """Body force (d, N) FP32 on the device (None removes it)."""
        torch = self.torch
        if F is None:
            lbm_set_force(self.ctx, None)
            self._force = None
            return self
        Ft = self._dev(F, torch.float32, self.d * self.N)
        lbm_set_force(self.ctx, Ft.data_ptr())
        self._force = Ft
        return self

    def set_lid(self, lid):
        lbm_set_lid(self.ctx, list(lid) + [0.0] * (3 - len(lid)))
        return self

    def set_geometry(self, solid):
        """Solid obstacles: N values, nonzero = solid (copied into link words).
        The state must be initialised again afterwards."""
        torch = self.torch
        self._sync_stream()
        st = torch.as_tensor(solid, device=self.device).reshape(-1).ne(0).to(torch.uint8)
        if st.numel() != self.N:
            raise ValueError(f"expected {self.N} values, got {st.numel()}")
        lbm_set_geometry(self.ctx, st.data_ptr())
        return self

    def set_inlet(self, u):
        """Inlet velocity (d, face nodes) FP32 (see lbm_set_inlet; None = at rest)."""
        torch = self.torch
        if u is None:
            lbm_set_inlet(self.ctx, None)
            self._inlet = None
            return self
        face = self.faces.index(LBM_FACE_INLET) if LBM_FACE_INLET in self.faces else 0
        nx, ny, nz = self.shape
        nf = {0: ny * nz, 1: nx * nz, 2: nx * ny}[face // 2]
        ut = self._dev(u, torch.float32, self.d * nf)
        lbm_set_inlet(self.ctx, ut.data_ptr())
        self._inlet = ut
        return self

    def step_force(self, n=1):
        """step(n); returns the momentum-exchange force on the obstacles (3,)
        during the last step."""
        self._sync_stream()
        return lbm_step_force(self.ctx, n)

    def step(self, n=1):
        self._sync_stream()
        lbm_step(self.ctx, n)
        return self

    def set_graph_steps(self, steps):
        """CUDA-graph replays of `steps` steps in step() (0 off, -1 automatic)."""
        lbm_set_graph_steps(self.ctx, steps)
        return self

    @property
    def step_count(self):
        return lbm_step_count(self.ctx)

    def set_kernel(self, variant):
        """'auto', 'plain' or 'paired' (see lbm_set_kernel_variant)."""
        lbm_set_kernel_variant(self.ctx, _key(KERNELS, variant))
        return self

    @property
    def kernel(self):
        v = lbm_kernel_variant_in_use(self.ctx)
        return {LBM_KERNEL_PLAIN: "plain", LBM_KERNEL_PAIRED: "paired"}[v]

    def macroscopic(self, dtype=None):
        """(p (N,), u (d, N)) of the current step."""
        torch = self.torch
        dtype = dtype or torch.float64
        self._sync_stream()
        p = torch.empty(self.N, dtype=dtype, device=self.device)
        u = torch.empty((self.d, self.N), dtype=dtype, device=self.device)
        lbm_macroscopic(self.ctx, p.data_ptr(), u.data_ptr(), 1 if dtype == torch.float32 else 0)
        return p, u

    def macroscopic_into(self, p, u):
        """Write p and u of the current step into preallocated tensors."""
        torch = self.torch
        self._sync_stream()
        dt = (p if p is not None else u).dtype
        lbm_macroscopic(self.ctx, None if p is None else p.data_ptr(),
                        None if u is None else u.data_ptr(), 1 if dt == torch.float32 else 0)

    def reduce(self):
        """dict(mass, momentum (3,), kinetic_energy, max_speed), FP64."""
        self._sync_stream()
        r = lbm_reduce(self.ctx)
        return {"mass": r[0], "momentum": r[1:4], "kinetic_energy": r[4], "max_speed": r[5]}

    def step_reduce(self, n=1):
        """step(n) with the last step also returning the Monitor values (as reduce())."""
        self._sync_stream()
        r = lbm_step_reduce(self.ctx, n)
        return {"mass": r[0], "momentum": r[1:4], "kinetic_energy": r[4], "max_speed": r[5]}

    def state_bytes(self):
        return lbm_state_bytes(self.ctx)

    def get_state(self):
        torch = self.torch
        self._sync_stream()
        buf = torch.empty(self.state_bytes(), dtype=torch.uint8, device=self.device)
        step = lbm_get_state(self.ctx, buf.data_ptr())
        return buf, step

    def set_state(self, buf, step):
        self._sync_stream()
        lbm_set_state(self.ctx, buf.data_ptr(), step)
        return self

    def adjoint_workspace(self, T, K):
        torch = self.torch
        nbytes = lbm_adjoint_workspace_bytes(self.ctx, T, K)
        if nbytes == 0:
            raise LBMError(LBM_ERR_ARG, "lbm_adjoint_workspace_bytes")
        if self._adj_ws is None or self._adj_ws.numel() < nbytes:
            self._adj_ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        return self._adj_ws

    def adjoint_forward(self, T, K):
        ws = self.adjoint_workspace(T, K)
        self._sync_stream()
        return lbm_adjoint_forward(self.ctx, T, K, ws.data_ptr(), ws.numel())

    def adjoint_backward(self):
        torch = self.torch
        self._sync_stream()
        g = torch.empty((self.d, self.N), dtype=torch.float64, device=self.device)
        gU = lbm_adjoint_backward(self.ctx, self._adj_ws.data_ptr(), self._adj_ws.numel(),
                                  g.data_ptr())
        return g, torch.tensor(gU, dtype=torch.float64)

    def adjoint(self, T, K):
        """(J, dJ/dF (d, N) FP64 on device, dJ/dU (3,) FP64 on host)."""
        torch = self.torch
        ws = self.adjoint_workspace(T, K)
        self._sync_stream()
        g = torch.empty((self.d, self.N), dtype=torch.float64, device=self.device)
        J, gU = lbm_adjoint(self.ctx, T, K, ws.data_ptr(), ws.numel(), g.data_ptr())
        return J, g, torch.tensor(gU, dtype=torch.float64)

    def close(self):
        if getattr(self, "ctx", None):
            lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
