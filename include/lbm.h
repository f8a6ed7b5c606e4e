/*
 * lbm.h -- C ABI of the B300 (sm_103a) lattice-Boltzmann hot path.
 *
 * One time step is the IMEXLBM update of arxiv 2201.11330: the local BGK
 * collision of Eq. (collision) with the paper's time discretisation
 * (omega = 1/(tau_paper + 1/2)), the incompressible equilibrium of Eq.
 * (incompressible_feq) (or Eq. (feq) on request), fused with propagation
 * Eq. (propagation) and the boundary conditions of Sec. 2.2 (half-way
 * bounce-back Eq. (bb)), a moving lid and periodic faces.  Steps run in the
 * order Collision -> BoundaryCondition -> Propagation -> PostProcessing of
 * Sec. 3.1, fused into one kernel launch per step.
 *
 * Conventions shared by every call
 *   - tau is the STANDARD BGK relaxation time tau_std = tau_paper + 1/2, so
 *     omega = 1/tau and nu = (tau - 1/2)/3.  lbm_tau_from_paper() converts.
 *   - Lattice units: c = 1, c_s^2 = 1/3, dt = 1.  Pressure p = c_s^2 sum f.
 *   - Grids are nx * ny * nz nodes, node index n = x + nx*(y + ny*z);
 *     2D (D2Q9) uses nz = 1.  N = nx*ny*nz must be below 2^31.
 *   - Field arrays are structure of arrays: a d-component field is d
 *     consecutive blocks of N values (component-major).
 *   - Walls sit half a spacing outside the first and last node of a walled
 *     axis.  LBM_BC_CAVITY walls every face and moves the +y face ("lid");
 *     LBM_BC_CHANNEL walls the y faces only (the +y wall may move) with x and
 *     z periodic; LBM_BC_PERIODIC wraps every axis.  A link crossing the
 *     moving wall (upstream y >= ny, corners included) gains
 *     2 t_a rho0 (e_a . U)/c_s^2.
 *
 * Memory and streams
 *   - The library never allocates device memory.  The caller passes one
 *     device workspace of lbm_workspace_bytes() bytes (any allocator, e.g. a
 *     torch uint8 tensor), 256-byte aligned, that must outlive the context.
 *     Every other device pointer is borrowed for the duration of the call
 *     only, except the force field of lbm_set_force, which is borrowed until
 *     it is replaced or the context is destroyed.
 *   - Every kernel is launched on the context's stream (a cudaStream_t passed
 *     as void*, NULL = legacy default stream).  Calls are asynchronous unless
 *     they return host values (lbm_reduce, lbm_adjoint*), which synchronise
 *     that stream.
 *
 * Errors: every call returns an lbm_status.  Argument errors are found on the
 * host before anything is launched and leave the context unchanged.  No call
 * aborts, throws or prints.  lbm_error_string() gives a static description.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = -1,      /* invalid argument (sizes, tau <= 1/2, NULL, enum) */
    LBM_ERR_CUDA = -2,     /* a CUDA launch or copy failed */
    LBM_ERR_UNSTABLE = -3, /* a reduction saw a non-finite value */
    LBM_ERR_STATE = -4,    /* call not valid in the context's current state */
    LBM_ERR_NOMEM = -5     /* workspace smaller than required */
} lbm_status;

typedef enum { LBM_D2Q9 = 0, LBM_D3Q19 = 1, LBM_D3Q27 = 2 } lbm_lattice;

/* Box types.  LBM_BC_FACES takes one lbm_face per face from lbm_opts.faces. */
typedef enum {
    LBM_BC_PERIODIC = 0,
    LBM_BC_CAVITY = 1,
    LBM_BC_CHANNEL = 2,
    LBM_BC_FACES = 3
} lbm_bc;

/* Per-face boundary conditions (the workloads of Sec. 4-5: channel flow past
 * a cylinder with a parabolic inlet and an outflow, flow past a sphere with
 * symmetry planes).  For the population entering node x along e_a the
 * upstream node x - e_a is fixed, coordinate by coordinate, by the face each
 * coordinate leaves through:
 *   LBM_FACE_PERIODIC  wraps (both faces of an axis must be periodic);
 *   LBM_FACE_WALL      half-way bounce-back, f_a(x) = f*_abar(x); the +y wall
 *                      adds the lid term 2 t_a rho0 (e_a . U)/c_s^2;
 *   LBM_FACE_INLET     half-way bounce-back with the term of the inlet
 *                      velocity (lbm_set_inlet) at x; at most one inlet face;
 *   LBM_FACE_OUTFLOW   pressure outlet by anti-bounce-back,
 *                      f_a(x) = -f*_abar(x) + 2 feq+_a(P_out, u(x)), feq+ the
 *                      even half of the equilibrium at P_out =
 *                      opts.p_outflow / c_s^2, u(x) the node's velocity from
 *                      its post-collision populations (the paper names a
 *                      convective outflow without printing it; behind a
 *                      velocity inlet an outlet must fix the pressure level);
 *   LBM_FACE_SYMMETRY  specular reflection (free slip): the coordinate stays
 *                      that of x and the direction's normal component flips;
 *   LBM_FACE_NODAL     the paper's "second-order modified nodal bounce back"
 *                      (Sec. 2.2, Eq. (bb)): the wall lies ON the boundary
 *                      nodes, which collide like the bulk; a population
 *                      entering one from outside is the opposite one that has
 *                      just arrived from inside, f_a(x) = f_abar(x) (plus the
 *                      lid term on +y; the node's own f*_abar(x) where that
 *                      one also comes from outside, as at corners).
 * A link crossing a wall or inlet bounces whatever else it crosses; then
 * nodal, then outflow win over symmetry and periodic.  The inlet term wins over the lid
 * term on a link crossing both.  Faces are ordered -x, +x, -y, +y, -z, +z;
 * D2Q9 ignores the z faces. */
typedef enum {
    LBM_FACE_PERIODIC = 0,
    LBM_FACE_WALL = 1,
    LBM_FACE_INLET = 2,
    LBM_FACE_OUTFLOW = 3,
    LBM_FACE_SYMMETRY = 4,
    LBM_FACE_NODAL = 5
} lbm_face;

/* Storage of the distributions in HBM.  Arithmetic is FP64 for LBM_F64 and
 * FP32 otherwise.  The "shifted" forms store f_a - t_a (t_a the lattice
 * weight), which the incompressible update leaves invariant up to rounding. */
typedef enum {
    LBM_F64 = 0,   /* FP64, unshifted */
    LBM_F32 = 1,   /* FP32, shifted (unshifted with lbm_opts.f32_unshifted) */
    LBM_F16S = 2,  /* IEEE binary16 of f - t, round to nearest even */
    LBM_BF16S = 3  /* bfloat16 of f - t, round to nearest even */
} lbm_storage;

/* Collision operator.  BGK is the paper's (Eq. (collision)); TRT (two
 * relaxation times, not in the paper) relaxes the symmetric part of each
 * opposite pair at omega = 1/tau and the antisymmetric part at omega_m set
 * by the "magic" parameter Lambda = (tau - 1/2)(1/omega_m - 1/2); with
 * Lambda = 3/16 half-way bounce-back places Poiseuille walls exactly for
 * any tau, and Lambda = (tau - 1/2)^2 is BGK.  TRT is available with the
 * incompressible equilibrium only (compressible + TRT is LBM_ERR_ARG) and
 * has no adjoint.
 * MRT (multiple relaxation times, not in the paper; d'Humieres et al. 2002)
 * relaxes the non-equilibrium part in an orthogonal moment basis (the
 * monomials e_x^i e_y^j e_z^k, i, j, k <= 2, by degree with |e|^2 first
 * among degree two, orthogonalised over the velocity set), with the Guo
 * source transformed the same way: the traceless stress at omega = 1/tau
 * (shear viscosity), the bulk moment (|e|^2) at mrt_bulk, the higher
 * moments at mrt_even / mrt_odd by the parity of their degree; density and
 * momentum are conserved (the force adds F).  A rate of 0 means omega, so
 * the defaults are BGK.  MRT runs with the incompressible equilibrium and
 * FP64 or FP32 storage (16-bit storage, compressible + MRT: LBM_ERR_ARG) and
 * has no adjoint. */
typedef enum { LBM_COLL_BGK = 0, LBM_COLL_TRT = 1, LBM_COLL_MRT = 2 } lbm_collision;

typedef struct {
    int storage;        /* lbm_storage */
    int aa;             /* 0: two-lattice pull scheme; 1: single-lattice AA pattern */
    int compressible;   /* 0: Eq. (incompressible_feq); 1: Eq. (feq) with rho = sum f */
    int f32_unshifted;  /* LBM_F32 only: store f itself instead of f - t */
    double rho0;        /* constant density of the incompressible model (> 0) */
    double lid_u[3];    /* moving-wall velocity (ignored for LBM_BC_PERIODIC) */
    int has_force;      /* 1: a body-force field will be set with lbm_set_force */
    int collision;      /* lbm_collision (default BGK) */
    double trt_lambda;  /* TRT magic parameter (> 0), e.g. 3/16 */
    int faces[6];       /* lbm_face per face (-x, +x, -y, +y, -z, +z), LBM_BC_FACES only */
    int geometry;       /* 1: solid obstacles will be set with lbm_set_geometry */
    double p_outflow;   /* pressure held at outflow faces (> 0, default 1/3) */
    double mrt_bulk;    /* LBM_COLL_MRT: rate of the bulk moment, (0, 2), or 0 = omega */
    double mrt_even;    /* LBM_COLL_MRT: rate of the even higher moments, (0, 2) or 0 */
    double mrt_odd;     /* LBM_COLL_MRT: rate of the odd higher moments, (0, 2) or 0 */
} lbm_opts;

typedef struct lbm_ctx lbm_ctx;

/* Defaults: LBM_F32, pull scheme, incompressible, BGK, shifted, rho0 = 1,
 * lid 0, trt_lambda 3/16 (used only with LBM_COLL_TRT), MRT rates 0 (= omega),
 * all faces periodic (used only with LBM_BC_FACES), no obstacles, p_outflow
 * 1/3. */
void lbm_default_opts(lbm_opts *opts);

/* tau_std = tau_paper + 1/2 (Sec. 3.3: "ome = 1/(tau+0.5)"). */
double lbm_tau_from_paper(double tau_paper);

/* Bytes of device workspace a context of this shape needs (0 on bad
 * arguments): the distributions (two lattices for the pull scheme, one for
 * AA) plus reduction scratch. */
size_t lbm_workspace_bytes(int lattice, int nx, int ny, int nz, const lbm_opts *opts);

/* Create a context (host memory only).  Sec. 3.3 DataInput/AllocateArrays:
 * the case is fixed here.  dev_workspace: caller-owned device memory of
 * `bytes` >= lbm_workspace_bytes(); cuda_stream: cudaStream_t or NULL.
 * Errors: LBM_ERR_ARG (bad lattice/bc/storage, sizes < 1, nz != 1 for D2Q9,
 * tau <= 1/2, rho0 <= 0, N >= 2^31, misaligned workspace; with LBM_BC_FACES
 * or opts.geometry: an unpaired periodic face, more than one inlet, or the
 * AA scheme, which supports the three named box types only), LBM_ERR_NOMEM
 * (workspace too small).  LBM_BC_FACES and obstacles run the pull scheme:
 * the plain (16-bit storage: paired) kernel on the nodes that touch only
 * walls, the lid and periodic faces, and the general kernel, one node per
 * thread, on a list of the rest. */
int lbm_create(int lattice, int nx, int ny, int nz, double tau, int bc, const lbm_opts *opts,
               void *dev_workspace, size_t bytes, void *cuda_stream, lbm_ctx **out);

/* Change the stream later calls launch on. */
int lbm_set_stream(lbm_ctx *ctx, void *cuda_stream);

/* Sec. 2.2 / Sec. 3.3 InitUP + Sec. 3.4 InitPDF: f = feq(p, u) at every node.
 * p: device FP64 pressure field (N values) or NULL for p = 1/3 everywhere;
 * u: device FP64 velocity field (d*N, component-major) or NULL for u = 0.
 * Resets the step counter to 0.  When a force is set, the stored state also
 * holds the first collision (the state is always post-collision). */
int lbm_init(lbm_ctx *ctx, const double *p, const double *u);
/* lbm_init with FP32 fields (half the bytes to bring to the device). */
int lbm_init_f32(lbm_ctx *ctx, const float *p, const float *u);

/* Body force (Guo form, trapezoidal): device FP32 field of d*N values,
 * component-major, borrowed until replaced; NULL removes the force.
 * Requires opts.has_force = 1 at creation (LBM_ERR_STATE otherwise). */
int lbm_set_force(lbm_ctx *ctx, const float *force);

/* Moving-wall velocity U (3 values, host).  Takes effect at the next step. */
int lbm_set_lid(lbm_ctx *ctx, const double *lid_u3);

/* Solid obstacles (Sec. 4-5 geometries; the paper's geo mask): solid is a
 * device array of N bytes, nonzero = solid node.  Requires opts.geometry = 1
 * at creation (LBM_ERR_STATE otherwise).  Builds one 32-bit link word per
 * node in the workspace (which of the node's incoming links start on a
 * solid node) and counts the fluid nodes; the mask itself is not kept.
 * Solid nodes are never updated, lbm_macroscopic reports p = 0 and u = 0
 * there, and lbm_reduce / lbm_step_reduce sum over fluid nodes only.
 * Invalidates the state: call lbm_init (or lbm_set_state) afterwards.
 * Synchronises the stream. */
int lbm_set_geometry(lbm_ctx *ctx, const uint8_t *solid);

/* Inlet velocity of the LBM_FACE_INLET face: device FP32, d * (face nodes)
 * values, component-major, the face's nodes numbered by its two remaining
 * axes with the lower axis fastest (face -x/+x: y + ny*z; -y/+y: x + nx*z;
 * -z/+z: x + nx*y).  Borrowed until replaced; NULL (the initial state) is an
 * inlet at rest.  LBM_ERR_STATE without an inlet face. */
int lbm_set_inlet(lbm_ctx *ctx, const float *u_in);

/* lbm_step(n), n >= 1, whose last step also sums the momentum exchange on
 * the solid nodes (Sec. 5, Ladd): over fluid nodes x and links whose source
 * is solid, 2 f*_abar(x) e_abar, the population that leaves x towards the
 * obstacle and comes back reversed.  out: host, 3 doubles (force on the
 * obstacles during that step, lattice units; z = 0 in 2D).  Per-block sums
 * in the kernel's arithmetic, then FP64 in a fixed order.  Requires
 * obstacles (LBM_ERR_STATE otherwise).  Synchronises the stream. */
int lbm_step_force(lbm_ctx *ctx, int64_t n, double *out);

/* Advance n >= 0 time steps (Sec. 3.1 main loop body), one fused kernel
 * launch per step. */
int lbm_step(lbm_ctx *ctx, int64_t n);

/* CUDA graphs for lbm_step: with steps = G (even, >= 2) lbm_step(n) for
 * n >= 2G runs its launches as replays of a G-step graph (captured once on a
 * private stream the context creates, replayed into the context's stream,
 * re-captured after any change of the launch parameters); the results are
 * those of direct launches, bit for bit.  Pays where a step's kernels are
 * shorter than their launch overhead.  steps = 0: direct launches only;
 * -1 (the default): G = 32 for states up to 256 MB, else direct.  Never used
 * while the context's stream is itself being captured.  LBM_ERR_ARG for
 * other values. */
int lbm_set_graph_steps(lbm_ctx *ctx, int steps);

/* Steps taken since lbm_init (or the value given to lbm_set_state). */
int64_t lbm_step_count(const lbm_ctx *ctx);

/* Which kernel runs the step (all compute the same arithmetic and give
 * bitwise identical results):
 *   LBM_KERNEL_PLAIN  one node per thread, Q populations straight from HBM;
 *   LBM_KERNEL_PAIRED 16-bit storage only, nx even: two adjacent nodes per
 *                     thread, one 32-bit word per slot, e_x = +-1 directions
 *                     realigned with warp shuffles;
 *   LBM_KERNEL_AUTO   the library's measured choice for the storage type
 *                     (PAIRED where eligible, else PLAIN).
 * The adjoint's recompute always uses the plain kernel.  LBM_ERR_ARG for an
 * unknown variant (2 is not used: it numbered a shared-memory staged
 * variant that measured slower than PLAIN everywhere and was removed) or
 * PAIRED on an ineligible context. */
typedef enum {
    LBM_KERNEL_AUTO = 0,
    LBM_KERNEL_PLAIN = 1,
    LBM_KERNEL_PAIRED = 3
} lbm_kernel_variant;
int lbm_set_kernel_variant(lbm_ctx *ctx, int variant);
/* The variant lbm_step currently launches (PLAIN or PAIRED). */
int lbm_kernel_variant_in_use(const lbm_ctx *ctx);

/* lbm_step(n) whose last step also computes the Monitor values of
 * lbm_reduce (same definitions, out: host, 6 doubles) inside the step
 * kernel: per-block sums written by the step itself, then a fixed-order
 * FP64 reduction of those (deterministic).  Saves the separate read of the
 * whole state that lbm_reduce needs.  n >= 1.  Synchronises the stream.
 * Errors as lbm_step and lbm_reduce. */
int lbm_step_reduce(lbm_ctx *ctx, int64_t n, double *out);

/* Sec. 3.4 PostProcessing: p = c_s^2 sum f and u = (sum e f + F/2)/rho of
 * the current step.  p_out: device, N values, or NULL; u_out: device, d*N
 * values component-major, or NULL.  out_dtype: 0 = FP64, 1 = FP32. */
int lbm_macroscopic(lbm_ctx *ctx, void *p_out, void *u_out, int out_dtype);

/* Sec. 3.4 Monitor (global part done on the GPU): out[0] = sum_x P (mass,
 * P = sum_a f_a), out[1..3] = sum_x rho u (momentum), out[4] = sum_x
 * rho |u|^2 / 2 (kinetic energy), out[5] = max_x |u|.  Per-node terms in the
 * kernel's arithmetic, cross-block sums in FP64.  out: host, 6 doubles.
 * Synchronises the stream.  LBM_ERR_UNSTABLE if any result is not finite. */
int lbm_reduce(lbm_ctx *ctx, double *out);

/* Checkpoint / resume.  The state is the encoded distributions of
 * lbm_state_bytes() bytes (layout private to the library, stable for a
 * given shape and options).  dst/src: device. */
size_t lbm_state_bytes(const lbm_ctx *ctx);
int lbm_get_state(lbm_ctx *ctx, void *dst, int64_t *step);
int lbm_set_state(lbm_ctx *ctx, const void *src, int64_t step);

/* Adjoint (not in the paper): gradients of J = rho0/2 sum_x |u(x, T)|^2
 * after T steps from the current state, with respect to the force field and
 * the moving-wall velocity.  States are checkpointed every K steps and
 * recomputed in between.  Incompressible model, BGK and pull scheme only.
 * adj_workspace: device, lbm_adjoint_workspace_bytes(ctx, T, K) bytes.
 * lbm_adjoint_forward runs the T forward steps (the context ends at step
 * T) and returns J; lbm_adjoint_backward then fills dJdF (device FP64, d*N,
 * component-major; may be NULL) and dJdU (host, 3 doubles; may be NULL).
 * lbm_adjoint does both.  All three synchronise the stream. */
size_t lbm_adjoint_workspace_bytes(const lbm_ctx *ctx, int64_t T, int64_t K);
int lbm_adjoint_forward(lbm_ctx *ctx, int64_t T, int64_t K, void *adj_workspace, size_t bytes,
                        double *J);
int lbm_adjoint_backward(lbm_ctx *ctx, void *adj_workspace, size_t bytes, double *dJdF,
                         double *dJdU);
int lbm_adjoint(lbm_ctx *ctx, int64_t T, int64_t K, void *adj_workspace, size_t bytes,
                double *J, double *dJdF, double *dJdU);

/* Allocation-free monitor reduction (the paper has no counterpart).
 *
 * Same six values as lbm_reduce, computed from a distribution buffer the
 * caller passes, for callers that hold such a buffer (for example a
 * checkpoint from lbm_get_state) but may not allocate device memory: code
 * running under an allocator that is frozen after start-up, inside a host
 * callback, or a tool that only inspects buffers it is handed.  It needs no
 * context and no workspace, and calls no cudaMalloc/cudaFree or other
 * allocating routine.
 *
 * Scratch: a fixed device array inside the library holding
 * LBM_NOALLOC_MAX_PARTIALS partial sums (8 doubles each) plus the result,
 * about 512 KB, present on every GPU that loads the library until the
 * process exits.  The call needs at least ceil(nx/256) * nz partials
 * (x-segments of at most 256 nodes times z-planes; the rows of each are
 * split over further blocks as far as the array allows) and returns
 * LBM_ERR_NOMEM, launching nothing, when that exceeds
 * LBM_NOALLOC_MAX_PARTIALS.  Every partial a call uses is rewritten by it,
 * so nothing needs clearing; but all calls on a device share the array, so
 * calls that overlap on the GPU (different streams or threads) race and must
 * be serialised by the caller.  Every call looks up the array's device
 * address on the current device with cudaGetSymbolAddress (so the address is
 * never stale, even after a device reset); the first call on a device also
 * loads the library's device code there, so make it before any stream
 * capture.
 *
 * Arguments: lattice, nx, ny, nz, bc and *opts as given to lbm_create for
 * the context that produced the buffer (one of the three named box types,
 * no obstacles; LBM_ERR_ARG otherwise); state: device buffer of
 * lbm_state_bytes() bytes in that context's layout; step: the step count
 * lbm_get_state reported (it selects the AA layout); force: the device FP32
 * force field (d*N) the context used, or NULL; cuda_stream: stream to run
 * on (NULL = default); out: host, 6 doubles as for lbm_reduce.
 * Synchronises the stream.  Errors: LBM_ERR_ARG (bad arguments),
 * LBM_ERR_NOMEM (scratch too small for the shape), LBM_ERR_CUDA,
 * LBM_ERR_UNSTABLE (a non-finite result). */
#define LBM_NOALLOC_MAX_PARTIALS 8192
int lbm_reduce_state_noalloc(int lattice, int nx, int ny, int nz, int bc, const lbm_opts *opts,
                             const void *state, int64_t step, const float *force,
                             void *cuda_stream, double *out);

/* Static description of a status code. */
const char *lbm_error_string(int status);

/* Free the host-side context and its graphs, if any (after the context's
 * stream has finished their replays; the workspace stays the caller's). */
void lbm_destroy(lbm_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
