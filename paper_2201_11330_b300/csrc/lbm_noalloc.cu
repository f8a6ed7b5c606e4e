// lbm_noalloc.cu -- lbm_reduce_state_noalloc: the monitor reduction (mass,
// momentum, kinetic energy, max |u|) of a distribution buffer, for callers
// that cannot allocate device memory.
//
// The context-based lbm_reduce keeps its per-block partial sums in the
// caller's workspace.  Some callers hold a state buffer (for example a
// checkpoint taken with lbm_get_state) but may not call cudaMalloc at all:
// code running under an allocator that is frozen after start-up (a fixed
// memory pool), in a host callback, or a tool that only inspects buffers it
// is handed.  This entry point needs no workspace and no context: its scratch
// is a file-scope device array of fixed size that every GPU loading the
// library holds until the process exits.
#include <math.h>
#include <algorithm>
#include <string.h>


#include "lbm.h"
#include "lbm_capi_internal.h"
#include "lbm_kernels.cuh"

using namespace lbm;

namespace {

constexpr int kStaticPartials = LBM_NOALLOC_MAX_PARTIALS;

// One partial (kPartialStride doubles) per block, then the 6-double result.
// Shared by every call on a device.
static __device__ __align__(256) double g_noalloc_scratch[kStaticPartials * kPartialStride + 8];

// Device address of the scratch array on the current device.  In host code
// g_noalloc_scratch is only a stand-in symbol; the address is looked up on
// every call (cheap once the module is loaded), so it is never stale, even
// after the device's primary context was reset.
cudaError_t scratch_for_current_device(double **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess)
        return e;
    *out = (double *)p;
    return cudaSuccess;
}

// grid (xseg, nz, ychunks): block (xs, z, c) walks the rows y = c, c +
// ychunks, ... of its z-plane segment and writes one FP64 partial.  The
// per-node values are those of k_moments (node_moments, monitor_values),
// bit for bit, and so are the warp sums of a row segment; only the order in
// which the FP64 partials are added differs.
template <class L, int S, int FORM, bool COMP, bool FORCE>
__global__ void __launch_bounds__(256) k_moments_noalloc(const typename Sto<S>::T *src,
                                                         const StepParams p, double *partials,
                                                         int xseg)
{
    using R = typename Sto<S>::R;
    const int xs = blockIdx.x, z = blockIdx.y, c0 = blockIdx.z;
    const int x = xs * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    // lane k < 5 keeps the FP64 running sum of value k (one FP64 add per warp
    // and row, as k_moments); the maximum stays in the kernel's arithmetic
    double acc = 0.0;
    R accmax = R(0);
    for (int y = c0; y < p.ny; y += gridDim.z) {
        R vals[kReduceVals] = {R(0), R(0), R(0), R(0), R(0), R(0)};
        if (x < p.nx) {
            const int n = x + p.nx * (y + p.ny * z);
            R s, rho, u[3];
            node_moments<L, S, FORM, COMP, FORCE>(src, p, x, y, z, n, s, rho, u);
            monitor_values(s, rho, u, vals);
        }
        R mine = R(0);
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const R w = warp_sum(vals[k]);
            mine = lane == k ? w : mine;
        }
        if (lane < 5)
            acc += double(mine);
        accmax = max(accmax, warp_max(vals[5]));
    }
    __shared__ double sh[8][kReduceVals];
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    if (lane < 5)
        sh[warp][lane] = acc;
    else if (lane == 5)
        sh[warp][5] = double(accmax);
    __syncthreads();
    if (threadIdx.x < kReduceVals) {
        const int k = threadIdx.x;
        double r = sh[0][k];
        for (int w = 1; w < nwarps; ++w)
            r = (k == 5) ? fmax(r, sh[w][k]) : r + sh[w][k];
        const size_t b = ((size_t)c0 * gridDim.y + z) * xseg + xs;
        partials[b * kPartialStride + k] = r;  // every slot of the launch rewritten
    }
}

template <class F>
cudaError_t pick(bool b, F &&f)
{
    return b ? f(std::true_type{}) : f(std::false_type{});
}

template <class L, int S>
cudaError_t launch_s(const void *state, int form, bool comp, bool force, const StepParams &p,
                     double *partials, int xseg, dim3 grid, dim3 block, cudaStream_t st)
{
    using T = typename Sto<S>::T;
    const T *src = (const T *)state;
    return pick(comp, [&](auto C) {
        return pick(force, [&](auto Fo) {
            constexpr bool c = decltype(C)::value, fo = decltype(Fo)::value;
            if (form == FORM_LOCAL)
                k_moments_noalloc<L, S, FORM_LOCAL, c, fo><<<grid, block, 0, st>>>(src, p, partials, xseg);
            else if (form == FORM_SWAPPED)
                k_moments_noalloc<L, S, FORM_SWAPPED, c, fo><<<grid, block, 0, st>>>(src, p, partials, xseg);
            else
                k_moments_noalloc<L, S, FORM_STREAMED, c, fo><<<grid, block, 0, st>>>(src, p, partials, xseg);
            return cudaGetLastError();
        });
    });
}

template <class L>
cudaError_t launch_l(int storage, const void *state, int form, bool comp, bool force,
                     const StepParams &p, double *partials, int xseg, dim3 grid, dim3 block,
                     cudaStream_t st)
{
    switch (storage) {
    case ST_F64:
        return launch_s<L, ST_F64>(state, form, comp, force, p, partials, xseg, grid, block, st);
    case ST_F32:
        return launch_s<L, ST_F32>(state, form, comp, force, p, partials, xseg, grid, block, st);
    case ST_F16S:
        return launch_s<L, ST_F16S>(state, form, comp, force, p, partials, xseg, grid, block, st);
    default:
        return launch_s<L, ST_BF16S>(state, form, comp, force, p, partials, xseg, grid, block, st);
    }
}

}  // namespace

extern "C" int lbm_reduce_state_noalloc(int lattice, int nx, int ny, int nz, int bc,
                                        const lbm_opts *opts, const void *state, int64_t step,
                                        const float *force, void *cuda_stream, double *out)
{
    if (!opts || !state || !out || step < 0)
        return LBM_ERR_ARG;
    if (lattice < LBM_D2Q9 || lattice > LBM_D3Q27 || bc < LBM_BC_PERIODIC || bc > LBM_BC_CHANNEL)
        return LBM_ERR_ARG;
    if (nx < 1 || ny < 1 || nz < 1 || nz > 65535 || (lattice == LBM_D2Q9 && nz != 1))
        return LBM_ERR_ARG;
    if ((long long)nx * ny * nz >= (1LL << 31))
        return LBM_ERR_ARG;
    const lbm_opts &o = *opts;
    if (!ctx_opts_valid(o))  // the options lbm_create accepts
        return LBM_ERR_ARG;
    if (o.geometry)  // solid nodes are known only to a context
        return LBM_ERR_ARG;
    // same row segments as the context path: x-segments of up to 256 nodes
    int bx = (nx + 31) / 32 * 32;
    if (bx > 256)
        bx = 256;
    const int xseg = (nx + bx - 1) / bx;
    if ((long long)xseg * nz > kStaticPartials)
        return LBM_ERR_NOMEM;  // the fixed scratch holds LBM_NOALLOC_MAX_PARTIALS partials
    // rows of a z-plane segment split over blocks, as far as the scratch allows
    const int ychunks = (int)std::min<long long>(ny, kStaticPartials / ((long long)xseg * nz));
    double *scratch = nullptr;
    if (scratch_for_current_device(&scratch) != cudaSuccess)
        return LBM_ERR_CUDA;
    double *partials = scratch;
    double *result = scratch + (size_t)kStaticPartials * kPartialStride;

    StepParams p;
    memset(&p, 0, sizeof(p));
    p.nx = nx;
    p.ny = ny;
    p.nz = nz;
    p.N = nx * ny * nz;
    p.periodic = bc == LBM_BC_PERIODIC ? 7 : bc == LBM_BC_CHANNEL ? 5 : 0;
    p.lid_on = bc != LBM_BC_PERIODIC;
    const bool shifted = o.storage != LBM_F64 && !(o.storage == LBM_F32 && o.f32_unshifted);
    const double sigma = shifted ? 1.0 : 0.0;
    p.cd.rho0 = o.rho0;
    p.cd.inv_rho0 = 1.0 / o.rho0;
    p.cd.sigma = sigma;
    p.cf.rho0 = (float)o.rho0;
    p.cf.inv_rho0 = (float)(1.0 / o.rho0);
    p.cf.sigma = (float)sigma;
    p.F = force;
    const int form = !o.aa ? FORM_LOCAL : (step % 2 == 0 ? FORM_SWAPPED : FORM_STREAMED);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const dim3 grid(xseg, nz, ychunks), block(bx, 1, 1);
    cudaError_t e;
    switch (lattice) {
    case LBM_D2Q9:
        e = launch_l<D2Q9>(o.storage, state, form, o.compressible != 0, force != nullptr, p,
                           partials, xseg, grid, block, st);
        break;
    case LBM_D3Q19:
        e = launch_l<D3Q19>(o.storage, state, form, o.compressible != 0, force != nullptr, p,
                            partials, xseg, grid, block, st);
        break;
    default:
        e = launch_l<D3Q27>(o.storage, state, form, o.compressible != 0, force != nullptr, p,
                            partials, xseg, grid, block, st);
        break;
    }
    if (e != cudaSuccess)
        return LBM_ERR_CUDA;
    k_reduce_finish<<<1, 256, 0, st>>>(partials, xseg * nz * ychunks, result);
    if (cudaGetLastError() != cudaSuccess)
        return LBM_ERR_CUDA;
    double r[kReduceVals];
    if (cudaMemcpyAsync(r, result, sizeof(r), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return LBM_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess)
        return LBM_ERR_CUDA;
    out[0] = r[0] + (shifted ? (double)p.N : 0.0);
    for (int k = 1; k < 5; ++k)
        out[k] = r[k];
    out[5] = sqrt(r[5]);
    for (int k = 0; k < kReduceVals; ++k)
        if (!isfinite(out[k]))
            return LBM_ERR_UNSTABLE;
    return LBM_OK;
}
