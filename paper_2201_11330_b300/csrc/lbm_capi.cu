// lbm_capi.cu -- the C ABI declared in include/lbm.h (host side).
//
// Owns no device memory: every buffer is carved out of the caller's
// workspace.  All launches go to the context's stream.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "lbm.h"
#include "lbm_capi_internal.h"
#include "lbm_geo.cuh"
#include "lbm_pair.cuh"
#include "lbm_kernels.cuh"

// bytes of every row next to an open x face that the node-list launch takes
#ifndef LBM_XMARGIN_BYTES
#define LBM_XMARGIN_BYTES 32
#endif

using namespace lbm;

namespace {

constexpr int kMaxReduceBlocks = 1184;  // 8 per SM on 148 SMs
constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

int lattice_q(int lattice) { return lattice == LBM_D2Q9 ? 9 : lattice == LBM_D3Q19 ? 19 : 27; }
int lattice_d(int lattice) { return lattice == LBM_D2Q9 ? 2 : 3; }
size_t storage_elem(int s) { return s == LBM_F64 ? 8 : s == LBM_F32 ? 4 : 2; }

int default_block(int nx)
{
    int b = (nx + 31) / 32 * 32;
    return b > 256 ? 256 : b;
}

bool valid_shape(int lattice, int nx, int ny, int nz)
{
    if (lattice < LBM_D2Q9 || lattice > LBM_D3Q27)
        return false;
    if (nx < 1 || ny < 1 || nz < 1 || ny > 65535 || nz > 65535)
        return false;
    if (lattice == LBM_D2Q9 && nz != 1)
        return false;
    const long long N = (long long)nx * ny * nz;
    return N < (1LL << 31);
}

bool valid_opts(const lbm_opts &o)
{
    if (o.storage < LBM_F64 || o.storage > LBM_BF16S)
        return false;
    if (o.collision != LBM_COLL_BGK && o.collision != LBM_COLL_TRT &&
        o.collision != LBM_COLL_MRT)
        return false;
    if (o.collision == LBM_COLL_TRT &&
        (o.compressible || !(o.trt_lambda > 0.0 && isfinite(o.trt_lambda))))
        return false;
    if (o.collision == LBM_COLL_MRT) {
        // incompressible model, FP64 / FP32 storage; each rate 0 (= omega) or in (0, 2)
        if (o.compressible || (o.storage != LBM_F64 && o.storage != LBM_F32))
            return false;
        for (const double r : {o.mrt_bulk, o.mrt_even, o.mrt_odd})
            if (!(r == 0.0 || (r > 0.0 && r < 2.0)))
                return false;
    }
    if (!(o.rho0 > 0.0) || !isfinite(o.rho0))
        return false;
    if (o.geometry != 0 && o.geometry != 1)
        return false;
    if (!(o.p_outflow > 0.0) || !isfinite(o.p_outflow))
        return false;
    for (int k = 0; k < 3; ++k)
        if (!isfinite(o.lid_u[k]))
            return false;
    return true;
}

// Face types of a box: the named types, or opts.faces for LBM_BC_FACES
// (validated: known types, periodic faces in pairs, at most one inlet; D2Q9
// z faces periodic).
bool resolve_faces(int lattice, int bc, const lbm_opts &o, int face[6])
{
    if (bc == LBM_BC_FACES) {
        for (int i = 0; i < 6; ++i)
            face[i] = o.faces[i];
    } else if (bc >= LBM_BC_PERIODIC && bc <= LBM_BC_CHANNEL) {
        for (int k = 0; k < 3; ++k) {
            const bool periodic = k == 1 ? bc == LBM_BC_PERIODIC : bc != LBM_BC_CAVITY;
            face[2 * k] = face[2 * k + 1] = periodic ? LBM_FACE_PERIODIC : LBM_FACE_WALL;
        }
    } else {
        return false;
    }
    if (lattice == LBM_D2Q9)
        face[4] = face[5] = LBM_FACE_PERIODIC;
    int ninlet = 0;
    for (int i = 0; i < 6; ++i) {
        if (face[i] < LBM_FACE_PERIODIC || face[i] > LBM_FACE_NODAL)
            return false;
        if ((face[i] == LBM_FACE_PERIODIC) != (face[i ^ 1] == LBM_FACE_PERIODIC))
            return false;
        ninlet += face[i] == LBM_FACE_INLET;
    }
    return ninlet <= 1;
}

// Boxes that may have open faces or obstacles keep a list of the nodes the
// plain kernel cannot update (the general kernel takes those).
bool wants_node_list(const lbm_opts &o)
{
    bool open = o.geometry != 0;
    for (int i = 0; i < 6; ++i)
        open = open || o.faces[i] != LBM_FACE_PERIODIC;
    return open;
}

struct Layout {
    size_t state_bytes, f_off[2], partial_off, result_off, step_partial_off, links_off, total;
    size_t flags_off, nlist_off;
    int nred;
    long long step_blocks;
};

Layout layout_for(int lattice, int nx, int ny, int nz, const lbm_opts &o)
{
    Layout L;
    const size_t N = (size_t)nx * ny * nz;
    L.state_bytes = (size_t)lattice_q(lattice) * N * storage_elem(o.storage);
    size_t off = 0;
    L.f_off[0] = off;
    off += align_up(L.state_bytes);
    L.f_off[1] = off;
    if (!o.aa)
        off += align_up(L.state_bytes);
    const int bx = default_block(nx);
    const long long nseg = (long long)((nx + bx - 1) / bx) * ny * nz;
    L.nred = (int)(nseg < kMaxReduceBlocks ? nseg : kMaxReduceBlocks);
    L.partial_off = off;
    off += align_up((size_t)L.nred * kPartialStride * sizeof(double));
    L.result_off = off;
    off += kAlign;
    // one monitor partial per block of a step launch (the plain kernel has the
    // most blocks of all step kernels)
    L.step_blocks = nseg;
    long long parts = nseg;
    if (wants_node_list(o))  // plus the general kernel's node-list blocks
        parts += ((long long)N + 255) / 256;
    L.step_partial_off = off;
    off += align_up((size_t)parts * kPartialStride * sizeof(double));
    L.links_off = off;
    if (o.geometry)
        off += align_up(N * sizeof(unsigned));
    L.flags_off = off;
    L.nlist_off = off;
    if (wants_node_list(o)) {
        off += align_up(N);
        L.nlist_off = off;
        off += align_up(N * sizeof(int));
    }
    L.total = off;
    return L;
}

cudaError_t dispatch(int lattice, const Launch &l)
{
    switch (lattice) {
    case LBM_D2Q9:
        return launch_d2q9(l);
    case LBM_D3Q19:
        return launch_d3q19(l);
    default:
        return launch_d3q27(l);
    }
}

template <class L>
void fill_lid_terms(lbm_ctx *c)
{
    for (int a = 0; a < L::Q; ++a) {
        const double eU = L::e(a, 0) * c->opts.lid_u[0] + L::e(a, 1) * c->opts.lid_u[1] +
                          L::e(a, 2) * c->opts.lid_u[2];
        const double v = 2.0 * L::w(a) * c->opts.rho0 * eU * 3.0;
        c->sp.cd.lid[a] = v;
        c->sp.cf.lid[a] = (float)v;
    }
}

template <class L>
void fill_row_offsets(lbm_ctx *c)
{
    const long long N = c->N, sy = c->nx, sz = (long long)c->nx * c->ny;
    for (int a = 0; a < kMaxQ; ++a)
        c->sp.pull_off[a] = c->sp.push_off[a] = c->sp.push_st[a] = 0;
    for (int a = 0; a < L::Q; ++a) {
        const long long shift = L::e(a, 1) * sy + L::e(a, 2) * sz;
        c->sp.pull_off[a] = a * N - shift;
        c->sp.push_off[a] = c->sp.push_st[a] = a * N + shift;
    }
}

void fill_params(lbm_ctx *c)
{
    ++c->param_version;
    StepParams &p = c->sp;
    p.nx = c->nx;
    p.ny = c->ny;
    p.nz = c->nz;
    p.N = (int)c->N;
    p.periodic = 0;
    for (int k = 0; k < 3; ++k)
        if (c->face[2 * k] == LBM_FACE_PERIODIC)
            p.periodic |= 1 << k;
    p.nlist = nullptr;
    p.nlist_len = 0;
    p.part_base = 0;
    p.open_faces = 0;
    // An open x face's nodes lie one per row: the node list takes whole DRAM
    // sectors of them (and the plain kernel leaves those sectors alone)
    p.xm = std::max(1, LBM_XMARGIN_BYTES / (int)storage_elem(c->opts.storage));
    for (int i = 0; i < 6; ++i)
        if (c->face[i] == LBM_FACE_INLET || c->face[i] == LBM_FACE_OUTFLOW ||
            c->face[i] == LBM_FACE_SYMMETRY || c->face[i] == LBM_FACE_NODAL)
            p.open_faces |= 1 << i;
    p.lid_on = c->face[3] == LBM_FACE_WALL || c->face[3] == LBM_FACE_NODAL;
    p.inlet_face = -1;
    for (int i = 0; i < 6; ++i) {
        p.face[i] = c->face[i];
        if (c->face[i] == LBM_FACE_INLET)
            p.inlet_face = i;
    }
    p.links = c->links_ready ? c->links : nullptr;
    const double omega = 1.0 / c->tau;
    const double sigma = c->shifted ? 1.0 : 0.0;
    // TRT: Lambda = (1/omega - 1/2)(1/omega_m - 1/2); BGK: omega_m = omega
    const double omega_m =
        c->opts.collision == LBM_COLL_TRT ? 1.0 / (c->opts.trt_lambda / (c->tau - 0.5) + 0.5) : omega;
    p.cd.omega_m = omega_m;
    p.cd.kf_m = (1.0 - 0.5 * omega_m) / omega_m;
    p.cf.omega_m = (float)omega_m;
    p.cf.kf_m = (float)p.cd.kf_m;
    // MRT rates of the bulk, even and odd higher moments (0: omega)
    const double mrt[3] = {c->opts.mrt_bulk, c->opts.mrt_even, c->opts.mrt_odd};
    for (int k = 0; k < 3; ++k) {
        p.cd.mrt[k] = mrt[k] > 0.0 ? mrt[k] : omega;
        p.cf.mrt[k] = (float)p.cd.mrt[k];
    }
    p.cd.omega = omega;
    p.cd.rho0 = c->opts.rho0;
    p.cd.inv_rho0 = 1.0 / c->opts.rho0;
    p.cd.sigma = sigma;
    p.cd.kf = (1.0 - 0.5 * omega) / omega;
    p.cf.omega = (float)omega;
    p.cf.rho0 = (float)c->opts.rho0;
    p.cf.inv_rho0 = (float)(1.0 / c->opts.rho0);
    p.cf.sigma = (float)sigma;
    p.cf.kf = (float)p.cd.kf;
    // pressure outlet: 2 feq+ - 2 sigma t = t [2 (P_out - sigma)] + 2 t r (...)
    const double P_out = c->opts.p_outflow * 3.0;
    p.cd.pout2 = 2.0 * (P_out - sigma);
    p.cd.pout_r = c->opts.compressible ? P_out : c->opts.rho0;
    p.cf.pout2 = (float)p.cd.pout2;
    p.cf.pout_r = (float)p.cd.pout_r;
    for (int a = 0; a < kMaxQ; ++a) {
        p.cd.lid[a] = 0.0;
        p.cf.lid[a] = 0.0f;
    }
    if (c->lattice == LBM_D2Q9)
        fill_lid_terms<D2Q9>(c);
    else if (c->lattice == LBM_D3Q19)
        fill_lid_terms<D3Q19>(c);
    else
        fill_lid_terms<D3Q27>(c);
    if (c->lattice == LBM_D2Q9)
        fill_row_offsets<D2Q9>(c);
    else if (c->lattice == LBM_D3Q19)
        fill_row_offsets<D3Q19>(c);
    else
        fill_row_offsets<D3Q27>(c);
    p.F = c->force;
    p.u_out = nullptr;
}

// p.inlet survives fill_params (which lbm_set_lid calls)
void keep_inlet(lbm_ctx *c, const float *inlet) { c->sp.inlet = inlet; }

// The paired kernel moves two 16-bit values per thread and slot.
bool pair_eligible(const lbm_ctx *c)
{
    return (c->opts.storage == LBM_F16S || c->opts.storage == LBM_BF16S) && c->nx % 2 == 0;
}

bool use_pair(const lbm_ctx *c, int pattern = PAT_PULL)
{
    if (!pair_eligible(c))
        return false;
    if (c->kernel_variant == LBM_KERNEL_PAIRED)
        return true;
    if (c->kernel_variant != LBM_KERNEL_AUTO)
        return false;
    // automatic choice (measured on B300): paired for 16-bit storage (the
    // D3Q27 AA gather half 3.33 ms vs 3.58 ms plain at 512^3)
    (void)pattern;
    return true;
}

Launch base_launch(const lbm_ctx *c, int kind)
{
    Launch l;
    memset(&l, 0, sizeof(l));
    l.kind = kind;
    l.storage = c->opts.storage;
    l.comp = c->opts.compressible != 0;
    l.model = l.comp                                   ? M_COMP
              : c->opts.collision == LBM_COLL_TRT      ? M_TRT
              : c->opts.collision == LBM_COLL_MRT      ? M_MRT
                                                       : M_INC;
    l.force = c->force != nullptr;
    l.uout = false;
    l.sp = c->sp;
    l.block = dim3(c->bx, 1, 1);
    l.grid = dim3((c->nx + c->bx - 1) / c->bx, c->ny, c->nz);
    l.stream = c->stream;
    return l;
}

}  // namespace

// ---- internal helpers shared with the adjoint driver ------------------------
namespace lbm {

bool ctx_opts_valid(const lbm_opts &o) { return valid_opts(o); }

Launch ctx_base_launch(const lbm_ctx *c, int kind) { return base_launch(c, kind); }

// Lists the nodes the plain kernel cannot update (solid, obstacle links,
// open faces).  Once per geometry; synchronises.
int build_node_list(lbm_ctx *c)
{
    const size_t N = (size_t)c->N;
    Launch l = base_launch(c, K_FLAGS);
    l.storage = LBM_F32;  // the flag kernel is instantiated once per lattice
    l.flags = c->nflags;
    l.pair = use_pair(c, PAT_PULL);  // the paired kernel updates whole pairs
    c->list_pairs = l.pair;
    if (dispatch(c->lattice, l) != cudaSuccess)
        return LBM_ERR_CUDA;
    std::vector<unsigned char> flags(N);
    if (cudaMemcpyAsync(flags.data(), c->nflags, N, cudaMemcpyDeviceToHost, c->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        return LBM_ERR_CUDA;
    std::vector<int> list;
    for (size_t n = 0; n < N; ++n)
        if (flags[n])
            list.push_back((int)n);
    if (!list.empty() &&
        (cudaMemcpyAsync(c->nlist, list.data(), list.size() * sizeof(int), cudaMemcpyHostToDevice,
                         c->stream) != cudaSuccess ||
         cudaStreamSynchronize(c->stream) != cudaSuccess))
        return LBM_ERR_CUDA;
    c->n_general = (long long)list.size();
    c->list_ready = true;
    ++c->param_version;  // the general kernel's grid changed
    return LBM_OK;
}

cudaError_t ctx_dispatch(const lbm_ctx *c, const Launch &l) { return dispatch(c->lattice, l); }

int ctx_launch_step(lbm_ctx *c, const void *src, void *dst, int pattern, void *u_out,
                    long long *reduce_blocks, bool obstacle_force)
{
    Launch l = base_launch(c, K_STEP);
    l.pattern = pattern;
    l.src = src;
    l.dst = dst;
    if (reduce_blocks)
        l.sp.partials = c->step_partials;
    if (c->geo) {
        // pull scheme: the plain kernel (two nodes per thread for 16-bit
        // storage) on every node it can update (walls, lid, periodic faces;
        // same arithmetic, bitwise equal results), the general kernel, one
        // node per thread, on the listed rest
        const int mon = reduce_blocks ? (obstacle_force ? 2 : 1) : 0;
        const long long grid_blocks = (long long)l.grid.x * l.grid.y * l.grid.z;
        if (!c->nflags) {
            l.geo = true;
            l.mon = mon;
            if (reduce_blocks)
                *reduce_blocks = grid_blocks;
            return dispatch(c->lattice, l) == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
        }
        if (!c->list_ready || c->list_pairs != use_pair(c, PAT_PULL)) {
            const int rc = build_node_list(c);
            if (rc != LBM_OK)
                return rc;
        }
        // the plain (or paired) kernel on the nodes it can update; its
        // reduction partials come first, the general kernel's after them
        Launch ls = l;
        ls.skip = true;
        ls.mon = mon;
        ls.pair = c->list_pairs;
        if (ls.pair)
            ls.grid = dim3((c->nx + 2 * kPairThreads - 1) / (2 * kPairThreads), c->ny, c->nz);
        const long long skip_blocks = (long long)ls.grid.x * ls.grid.y * ls.grid.z;
        const long long gblocks = (c->n_general + 255) / 256;
        if (gblocks > 0) {
            Launch lg = l;
            lg.geo = true;
            lg.mon = mon;
            lg.sp.nlist = c->nlist;
            lg.sp.nlist_len = (int)c->n_general;
            lg.sp.part_base = skip_blocks;
            lg.grid = dim3((unsigned)gblocks, 1, 1);
            lg.block = dim3(256, 1, 1);
            if (dispatch(c->lattice, lg) != cudaSuccess)
                return LBM_ERR_CUDA;
        }
        if (dispatch(c->lattice, ls) != cudaSuccess)
            return LBM_ERR_CUDA;
        if (reduce_blocks)
            *reduce_blocks = skip_blocks + gblocks;
        return LBM_OK;
    }
    if (u_out) {
        l.uout = true;
        l.sp.u_out = u_out;
    } else if (use_pair(c, pattern)) {
        l.pair = true;
        if (reduce_blocks)
            *reduce_blocks = (long long)((c->nx + 2 * kPairThreads - 1) / (2 * kPairThreads)) *
                             c->ny * c->nz;
    }
    if (reduce_blocks && !l.pair)
        *reduce_blocks = (long long)l.grid.x * l.grid.y * l.grid.z;
    return dispatch(c->lattice, l) == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

int ctx_launch_moments(lbm_ctx *c, const void *src, int form, void *p_out, void *u_out,
                       int out_f32, double *partials)
{
    Launch l = base_launch(c, K_MOMENTS);
    l.pattern = form;
    l.src = src;
    l.mp.p_out = p_out;
    l.mp.u_out = u_out;
    l.mp.out_f32 = out_f32;
    l.mp.partials = partials;
    l.mp.xseg = (c->nx + c->bx - 1) / c->bx;
    l.mp.nseg = l.mp.xseg * c->ny * c->nz;
    l.mp.links = c->sp.links;
    // persistent blocks, grid-stride over the row segments (measured faster
    // than one segment per block with a chunked reduction of the partials)
    l.grid = dim3(c->nred, 1, 1);
    return dispatch(c->lattice, l) == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

int ctx_reduce_state(lbm_ctx *c, const void *src, int form, double r[6])
{
    int rc = ctx_launch_moments(c, src, form, nullptr, nullptr, 0, c->partials);
    if (rc != LBM_OK)
        return rc;
    if (launch_finish(c->partials, c->nred, c->result, c->stream) != cudaSuccess)
        return LBM_ERR_CUDA;
    if (cudaMemcpyAsync(r, c->result, kReduceVals * sizeof(double), cudaMemcpyDeviceToHost,
                        c->stream) != cudaSuccess)
        return LBM_ERR_CUDA;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess)
        return LBM_ERR_CUDA;
    return LBM_OK;
}

int ctx_current_form(const lbm_ctx *c)
{
    if (!c->opts.aa)
        return FORM_LOCAL;
    return (c->step % 2 == 0) ? FORM_SWAPPED : FORM_STREAMED;
}

const void *ctx_state(const lbm_ctx *c) { return c->opts.aa ? c->f[0] : c->f[c->cur]; }

}  // namespace lbm

// ---- C ABI -------------------------------------------------------------------
extern "C" {

void lbm_default_opts(lbm_opts *o)
{
    if (!o)
        return;
    memset(o, 0, sizeof(*o));
    o->storage = LBM_F32;
    o->rho0 = 1.0;
    o->collision = LBM_COLL_BGK;
    o->trt_lambda = 3.0 / 16.0;
    o->p_outflow = 1.0 / 3.0;
}

double lbm_tau_from_paper(double tau_paper) { return tau_paper + 0.5; }

size_t lbm_workspace_bytes(int lattice, int nx, int ny, int nz, const lbm_opts *opts)
{
    lbm_opts o;
    if (opts)
        o = *opts;
    else
        lbm_default_opts(&o);
    if (!valid_shape(lattice, nx, ny, nz) || !valid_opts(o))
        return 0;
    return layout_for(lattice, nx, ny, nz, o).total;
}

int lbm_create(int lattice, int nx, int ny, int nz, double tau, int bc, const lbm_opts *opts,
               void *dev_workspace, size_t bytes, void *cuda_stream, lbm_ctx **out)
{
    if (!out)
        return LBM_ERR_ARG;
    *out = nullptr;
    lbm_opts o;
    if (opts)
        o = *opts;
    else
        lbm_default_opts(&o);
    if (!valid_shape(lattice, nx, ny, nz) || !valid_opts(o))
        return LBM_ERR_ARG;
    if (!(tau > 0.5) || !isfinite(tau))
        return LBM_ERR_ARG;
    int face[6];
    if (!resolve_faces(lattice, bc, o, face))
        return LBM_ERR_ARG;
    const bool geo = bc == LBM_BC_FACES || o.geometry;
    if (geo && o.aa)
        return LBM_ERR_ARG;
    if (!dev_workspace || ((uintptr_t)dev_workspace % kAlign) != 0)
        return LBM_ERR_ARG;
    const Layout L = layout_for(lattice, nx, ny, nz, o);
    if (bytes < L.total)
        return LBM_ERR_NOMEM;
    lbm_ctx *c = new (std::nothrow) lbm_ctx;
    if (!c)
        return LBM_ERR_NOMEM;
    memset(c, 0, sizeof(*c));
    c->lattice = lattice;
    c->Q = lattice_q(lattice);
    c->d = lattice_d(lattice);
    c->nx = nx;
    c->ny = ny;
    c->nz = nz;
    c->N = (int64_t)nx * ny * nz;
    c->tau = tau;
    c->bc = bc;
    c->opts = o;
    if (bc == LBM_BC_PERIODIC)
        for (int k = 0; k < 3; ++k)
            c->opts.lid_u[k] = 0.0;
    c->shifted = o.storage != LBM_F64 && !(o.storage == LBM_F32 && o.f32_unshifted);
    c->ws = (char *)dev_workspace;
    c->ws_bytes = bytes;
    c->state_bytes = L.state_bytes;
    c->f[0] = c->ws + L.f_off[0];
    c->f[1] = o.aa ? c->f[0] : c->ws + L.f_off[1];
    c->cur = 0;
    c->nred = L.nred;
    c->partials = (double *)(c->ws + L.partial_off);
    c->result = (double *)(c->ws + L.result_off);
    c->step_partials = (double *)(c->ws + L.step_partial_off);
    c->step_blocks = L.step_blocks;
    c->stream = (cudaStream_t)cuda_stream;
    c->force = nullptr;
    c->step = 0;
    c->bx = default_block(nx);
    c->initialized = false;
    c->kernel_variant = LBM_KERNEL_AUTO;
    c->geo = geo;
    for (int i = 0; i < 6; ++i)
        c->face[i] = face[i];
    c->links = o.geometry ? (unsigned *)(c->ws + L.links_off) : nullptr;
    c->links_ready = false;
    c->count = (unsigned long long *)((char *)c->result + 128);
    c->n_fluid = c->N;
    c->nflags = wants_node_list(o) ? (unsigned char *)(c->ws + L.flags_off) : nullptr;
    c->nlist = wants_node_list(o) ? (int *)(c->ws + L.nlist_off) : nullptr;
    c->list_ready = false;
    c->graph_mode = -1;  // automatic; graphs and their stream are made on first use
    fill_params(c);
    c->sp.inlet = nullptr;
    *out = c;
    return LBM_OK;
}

int lbm_set_stream(lbm_ctx *c, void *cuda_stream)
{
    if (!c)
        return LBM_ERR_ARG;
    c->stream = (cudaStream_t)cuda_stream;
    return LBM_OK;
}

namespace {
int init_from(lbm_ctx *c, const void *p, const void *u, bool in_f32)
{
    if (!c)
        return LBM_ERR_ARG;
    Launch l = base_launch(c, K_INIT);
    l.pattern = c->opts.aa ? 1 : 0;
    l.p0 = p;
    l.u0 = u;
    l.in_f32 = in_f32;
    c->cur = 0;
    l.dst = c->f[0];
    c->step = 0;
    if (dispatch(c->lattice, l) != cudaSuccess)
        return LBM_ERR_CUDA;
    c->initialized = true;
    return LBM_OK;
}
}  // namespace

int lbm_init(lbm_ctx *c, const double *p, const double *u) { return init_from(c, p, u, false); }

int lbm_init_f32(lbm_ctx *c, const float *p, const float *u) { return init_from(c, p, u, true); }

int lbm_set_force(lbm_ctx *c, const float *force)
{
    if (c)
        ++c->param_version;
    if (!c)
        return LBM_ERR_ARG;
    if (!c->opts.has_force)
        return LBM_ERR_STATE;
    c->force = force;
    c->sp.F = force;
    return LBM_OK;
}

int lbm_set_lid(lbm_ctx *c, const double *lid_u3)
{
    if (!c || !lid_u3)
        return LBM_ERR_ARG;
    for (int k = 0; k < 3; ++k)
        if (!isfinite(lid_u3[k]))
            return LBM_ERR_ARG;
    if (c->bc == LBM_BC_PERIODIC)
        return LBM_OK;
    for (int k = 0; k < 3; ++k)
        c->opts.lid_u[k] = lid_u3[k];
    const float *inlet = c->sp.inlet;
    fill_params(c);
    keep_inlet(c, inlet);
    return LBM_OK;
}

int lbm_set_geometry(lbm_ctx *c, const uint8_t *solid)
{
    if (!c || !solid)
        return LBM_ERR_ARG;
    if (!c->opts.geometry)
        return LBM_ERR_STATE;
    if (cudaMemsetAsync(c->count, 0, sizeof(unsigned long long), c->stream) != cudaSuccess)
        return LBM_ERR_CUDA;
    Launch l = base_launch(c, K_LINKS);
    l.storage = LBM_F32;  // the link kernel is instantiated once per lattice
    l.solid = solid;
    l.links = c->links;
    l.nsolid = c->count;
    if (dispatch(c->lattice, l) != cudaSuccess)
        return LBM_ERR_CUDA;
    unsigned long long nsolid = 0;
    if (cudaMemcpyAsync(&nsolid, c->count, sizeof(nsolid), cudaMemcpyDeviceToHost, c->stream) !=
        cudaSuccess)
        return LBM_ERR_CUDA;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess)
        return LBM_ERR_CUDA;
    c->n_fluid = c->N - (int64_t)nsolid;
    c->links_ready = true;
    c->sp.links = c->links;
    c->list_ready = false;  // the general kernel's nodes change with the obstacles
    ++c->param_version;
    c->initialized = false;
    return LBM_OK;
}

int lbm_set_inlet(lbm_ctx *c, const float *u_in)
{
    if (!c)
        return LBM_ERR_ARG;
    if (c->sp.inlet_face < 0)
        return LBM_ERR_STATE;
    keep_inlet(c, u_in);
    ++c->param_version;
    return LBM_OK;
}

namespace {

// The launches of time step `step` with the pull lattices in `cur`.
int launch_one_step(lbm_ctx *c, int64_t step, int cur)
{
    if (c->opts.aa) {
        const int pat = (step % 2 == 0) ? PAT_GATHER : PAT_LOCAL;
        return ctx_launch_step(c, c->f[0], c->f[0], pat, nullptr);
    }
    return ctx_launch_step(c, c->f[cur], c->f[1 - cur], PAT_PULL, nullptr);
}

int step_direct(lbm_ctx *c, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) {
        const int rc = launch_one_step(c, c->step, c->cur);
        if (rc != LBM_OK)
            return rc;
        if (!c->opts.aa)
            c->cur = 1 - c->cur;
        ++c->step;
    }
    return LBM_OK;
}

// Steps per graph: graphs pay where a step's kernels are shorter than their
// launches (the automatic choice: states up to 256 MB).
int graph_steps(const lbm_ctx *c)
{
    if (c->graph_mode >= 0)
        return c->graph_mode;
    return c->state_bytes <= ((size_t)256 << 20) ? 32 : 0;
}

void drop_graphs(lbm_ctx *c)
{
    for (int k = 0; k < 2; ++k) {
        if (c->graph[k])
            cudaGraphExecDestroy(c->graph[k]);
        c->graph[k] = nullptr;
    }
}

// Captures G steps starting from the context's current step and lattice on
// the private stream (nothing runs) and instantiates them as graph[key].
int capture_graph(lbm_ctx *c, int key, int G)
{
    if (c->graph[key]) {
        cudaGraphExecDestroy(c->graph[key]);
        c->graph[key] = nullptr;
    }
    if (!c->cap_stream &&
        cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return LBM_ERR_CUDA;
    cudaStream_t user = c->stream;
    if (cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return LBM_ERR_CUDA;
    c->stream = c->cap_stream;
    int rc = LBM_OK, cur = c->cur;
    for (int i = 0; i < G && rc == LBM_OK; ++i) {
        rc = launch_one_step(c, c->step + i, cur);
        cur = 1 - cur;
    }
    c->stream = user;
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
    if (rc != LBM_OK || e != cudaSuccess || !g) {
        if (g)
            cudaGraphDestroy(g);
        (void)cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    const cudaError_t ei = cudaGraphInstantiate(&c->graph[key], g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
        c->graph[key] = nullptr;
        (void)cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    c->graph_version[key] = c->param_version;
    c->graph_len[key] = G;
    return LBM_OK;
}

}  // namespace

int lbm_set_graph_steps(lbm_ctx *c, int steps)
{
    if (!c || steps < -1 || (steps > 0 && steps % 2 != 0))
        return LBM_ERR_ARG;
    c->graph_mode = steps;
    return LBM_OK;
}

int lbm_step(lbm_ctx *c, int64_t n)
{
    if (!c || n < 0)
        return LBM_ERR_ARG;
    if (!c->initialized)
        return LBM_ERR_STATE;
    const int G = graph_steps(c);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const bool capturing = cudaStreamIsCapturing(c->stream, &cs) != cudaSuccess ||
                           cs != cudaStreamCaptureStatusNone;
    if (capturing)
        (void)cudaGetLastError();
    if (G >= 2 && n >= 2 * (int64_t)G && !capturing) {
        // a first direct step does the lazy set-up (node lists, occupancy
        // queries), which cannot run under capture
        int rc = step_direct(c, 1);
        if (rc != LBM_OK)
            return rc;
        n -= 1;
        // the G-step sequence (G even) repeats from the same AA parity or
        // pull lattice: one cached graph per starting parity / lattice
        const int key = c->opts.aa ? (int)(c->step % 2) : c->cur;
        bool ok = c->graph[key] && c->graph_version[key] == c->param_version &&
                  c->graph_len[key] == G;
        if (!ok)
            ok = capture_graph(c, key, G) == LBM_OK;
        if (ok) {
            while (n >= G) {
                if (cudaGraphLaunch(c->graph[key], c->stream) != cudaSuccess)
                    return LBM_ERR_CUDA;
                c->step += G;
                n -= G;
            }
        }
    }
    return step_direct(c, n);
}

int64_t lbm_step_count(const lbm_ctx *c) { return c ? c->step : -1; }

int lbm_set_kernel_variant(lbm_ctx *c, int variant)
{
    if (!c || (variant != LBM_KERNEL_AUTO && variant != LBM_KERNEL_PLAIN &&
               variant != LBM_KERNEL_PAIRED))
        return LBM_ERR_ARG;
    if (variant == LBM_KERNEL_PAIRED && !pair_eligible(c))
        return LBM_ERR_ARG;
    c->kernel_variant = variant;
    ++c->param_version;
    return LBM_OK;
}

int lbm_kernel_variant_in_use(const lbm_ctx *c)
{
    if (!c)
        return LBM_ERR_ARG;
    return use_pair(c) ? LBM_KERNEL_PAIRED : LBM_KERNEL_PLAIN;
}

int lbm_step_reduce(lbm_ctx *c, int64_t n, double *out)
{
    if (!c || n < 1 || !out)
        return LBM_ERR_ARG;
    if (!c->initialized)
        return LBM_ERR_STATE;
    int rc = lbm_step(c, n - 1);
    if (rc != LBM_OK)
        return rc;
    long long nb = 0;
    if (c->opts.aa) {
        const int pat = (c->step % 2 == 0) ? PAT_GATHER : PAT_LOCAL;
        rc = ctx_launch_step(c, c->f[0], c->f[0], pat, nullptr, &nb);
    } else {
        rc = ctx_launch_step(c, c->f[c->cur], c->f[1 - c->cur], PAT_PULL, nullptr, &nb);
        if (rc == LBM_OK)
            c->cur = 1 - c->cur;
    }
    if (rc != LBM_OK)
        return rc;
    ++c->step;
    const int nout = (int)(nb < c->nred ? nb : c->nred);
    if (launch_chunks(c->step_partials, nb, c->partials, nout, c->stream) != cudaSuccess)
        return LBM_ERR_CUDA;
    if (launch_finish(c->partials, nout, c->result, c->stream) != cudaSuccess)
        return LBM_ERR_CUDA;
    double r[kReduceVals];
    if (cudaMemcpyAsync(r, c->result, sizeof(r), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        return LBM_ERR_CUDA;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess)
        return LBM_ERR_CUDA;
    out[0] = r[0] + (c->shifted ? (double)c->n_fluid : 0.0);
    for (int k = 1; k < 5; ++k)
        out[k] = r[k];
    out[5] = sqrt(r[5]);
    for (int k = 0; k < kReduceVals; ++k)
        if (!isfinite(out[k]))
            return LBM_ERR_UNSTABLE;
    return LBM_OK;
}

int lbm_step_force(lbm_ctx *c, int64_t n, double *out)
{
    if (!c || n < 1 || !out)
        return LBM_ERR_ARG;
    if (!c->initialized)
        return LBM_ERR_STATE;
    if (!c->links_ready)
        return LBM_ERR_STATE;
    int rc = lbm_step(c, n - 1);
    if (rc != LBM_OK)
        return rc;
    long long nb = 0;
    rc = ctx_launch_step(c, c->f[c->cur], c->f[1 - c->cur], PAT_PULL, nullptr, &nb, true);
    if (rc != LBM_OK)
        return rc;
    c->cur = 1 - c->cur;
    ++c->step;
    const int nout = (int)(nb < c->nred ? nb : c->nred);
    if (launch_chunks(c->step_partials, nb, c->partials, nout, c->stream) != cudaSuccess)
        return LBM_ERR_CUDA;
    if (launch_finish(c->partials, nout, c->result, c->stream) != cudaSuccess)
        return LBM_ERR_CUDA;
    double r[3];
    if (cudaMemcpyAsync(r, c->result, sizeof(r), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        return LBM_ERR_CUDA;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess)
        return LBM_ERR_CUDA;
    for (int k = 0; k < 3; ++k) {
        out[k] = r[k];
        if (!isfinite(out[k]))
            return LBM_ERR_UNSTABLE;
    }
    return LBM_OK;
}

int lbm_macroscopic(lbm_ctx *c, void *p_out, void *u_out, int out_dtype)
{
    if (!c || (out_dtype != 0 && out_dtype != 1))
        return LBM_ERR_ARG;
    if (!c->initialized)
        return LBM_ERR_STATE;
    if (!p_out && !u_out)
        return LBM_OK;
    return ctx_launch_moments(c, ctx_state(c), ctx_current_form(c), p_out, u_out, out_dtype,
                              nullptr);
}

int lbm_reduce(lbm_ctx *c, double *out)
{
    if (!c || !out)
        return LBM_ERR_ARG;
    if (!c->initialized)
        return LBM_ERR_STATE;
    double r[kReduceVals];
    const int rc = ctx_reduce_state(c, ctx_state(c), ctx_current_form(c), r);
    if (rc != LBM_OK)
        return rc;
    out[0] = r[0] + (c->shifted ? (double)c->n_fluid : 0.0);
    out[1] = r[1];
    out[2] = r[2];
    out[3] = r[3];
    out[4] = r[4];
    out[5] = sqrt(r[5]);
    for (int k = 0; k < kReduceVals; ++k)
        if (!isfinite(out[k]))
            return LBM_ERR_UNSTABLE;
    return LBM_OK;
}

size_t lbm_state_bytes(const lbm_ctx *c) { return c ? c->state_bytes : 0; }

int lbm_get_state(lbm_ctx *c, void *dst, int64_t *step)
{
    if (!c || !dst)
        return LBM_ERR_ARG;
    if (!c->initialized)
        return LBM_ERR_STATE;
    if (cudaMemcpyAsync(dst, ctx_state(c), c->state_bytes, cudaMemcpyDeviceToDevice,
                        c->stream) != cudaSuccess)
        return LBM_ERR_CUDA;
    if (step)
        *step = c->step;
    return LBM_OK;
}

int lbm_set_state(lbm_ctx *c, const void *src, int64_t step)
{
    if (!c || !src || step < 0)
        return LBM_ERR_ARG;
    if (cudaMemcpyAsync((void *)ctx_state(c), src, c->state_bytes, cudaMemcpyDeviceToDevice,
                        c->stream) != cudaSuccess)
        return LBM_ERR_CUDA;
    c->step = step;
    c->initialized = true;
    return LBM_OK;
}

const char *lbm_error_string(int status)
{
    switch (status) {
    case LBM_OK:
        return "ok";
    case LBM_ERR_ARG:
        return "invalid argument";
    case LBM_ERR_CUDA:
        return "CUDA launch or copy failed";
    case LBM_ERR_UNSTABLE:
        return "non-finite value in the state (unstable run)";
    case LBM_ERR_STATE:
        return "call not valid in the current state";
    case LBM_ERR_NOMEM:
        return "workspace too small";
    }
    return "unknown status";
}

void lbm_destroy(lbm_ctx *c)
{
    if (!c)
        return;
    if (c->graph[0] || c->graph[1])  // no replay may still be running
        cudaStreamSynchronize(c->stream);
    drop_graphs(c);
    if (c->cap_stream)
        cudaStreamDestroy(c->cap_stream);
    delete c;
}

}  // extern "C"

namespace lbm {
cudaError_t launch_finish(const double *partials, int nblocks, double *out, cudaStream_t s)
{
    k_reduce_finish<<<1, 256, 0, s>>>(partials, nblocks, out);
    return cudaGetLastError();
}

cudaError_t launch_chunks(const double *in, long long nin, double *out, int nout, cudaStream_t s)
{
    const long long chunk = (nin + nout - 1) / nout;
    k_reduce_chunks<<<nout, 256, 0, s>>>(in, nin, chunk, out);
    return cudaGetLastError();
}
}  // namespace lbm
