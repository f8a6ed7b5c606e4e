// lbm_adjoint.cu -- host driver of the adjoint (reverse) sweep with
// checkpointing: lbm_adjoint_forward / lbm_adjoint_backward / lbm_adjoint.
//
// Forward: T steps of the pull scheme from the current state, the state after
// every K-th step written straight into its checkpoint slot (no extra copy),
// then J and the seed lambda^T = e . u^T.  Backward, segment by segment from
// the last: recompute the K-1 intermediate steps from the segment's
// checkpoint while writing u^k of each step (the only field the transposed
// collision needs), run the K adjoint steps in reverse, and flush the
// segment's force gradient (kernel arithmetic) into the FP64 total.
#include <string.h>

#include "lbm_capi_internal.h"
#include "lbm_kernels.cuh"

using namespace lbm;

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct AdjLayout {
    int64_t nseg;
    size_t ckpt_off, ckpt_stride;
    size_t rec_off[2];
    size_t useg_off, useg_stride;
    size_t lam_off[2];
    size_t gF_off;
    size_t gU_off;
    int gU_n;
    size_t total;
    size_t real;  // bytes of the adjoint arithmetic type
};

bool adj_supported(const lbm_ctx *c)
{
    return !c->opts.aa && !c->opts.compressible && c->opts.collision == LBM_COLL_BGK && !c->geo;
}

AdjLayout adj_layout(const lbm_ctx *c, int64_t T, int64_t K)
{
    AdjLayout a;
    const size_t N = (size_t)c->N;
    a.real = c->opts.storage == LBM_F64 ? 8 : 4;
    a.nseg = (T + K - 1) / K;
    size_t off = 0;
    a.ckpt_off = off;
    a.ckpt_stride = align_up(c->state_bytes);
    off += a.ckpt_stride * (size_t)a.nseg;
    for (int i = 0; i < 2; ++i) {
        a.rec_off[i] = off;
        off += align_up(c->state_bytes);
    }
    a.useg_off = off;
    a.useg_stride = align_up((size_t)c->d * N * a.real);
    off += a.useg_stride * (size_t)K;
    for (int i = 0; i < 2; ++i) {
        a.lam_off[i] = off;
        off += align_up((size_t)c->Q * N * a.real);
    }
    a.gF_off = off;
    off += align_up((size_t)c->d * N * a.real);
    const int xseg = (c->nx + c->bx - 1) / c->bx;
    a.gU_n = xseg * c->nz;
    a.gU_off = off;
    off += align_up((size_t)a.gU_n * 4 * sizeof(double));
    off += kAlign;  // gU result
    a.total = off;
    return a;
}

__global__ void k_sum_columns(const double *part, int n, int stride, int ncols, double *out)
{
    __shared__ double sh[256][3];
    double acc[3] = {0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        for (int k = 0; k < ncols; ++k)
            acc[k] += part[(size_t)i * stride + k];
    for (int k = 0; k < 3; ++k)
        sh[threadIdx.x][k] = acc[k];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int k = 0; k < 3; ++k)
                sh[threadIdx.x][k] += sh[threadIdx.x + s][k];
        __syncthreads();
    }
    if (threadIdx.x < ncols)
        out[threadIdx.x] = sh[0][threadIdx.x];
}

char *at(void *ws, size_t off) { return (char *)ws + off; }

}  // namespace

extern "C" {

size_t lbm_adjoint_workspace_bytes(const lbm_ctx *c, int64_t T, int64_t K)
{
    if (!c || T < 1 || K < 1 || !adj_supported(c))
        return 0;
    return adj_layout(c, T, K).total;
}

int lbm_adjoint_forward(lbm_ctx *c, int64_t T, int64_t K, void *ws, size_t bytes, double *J)
{
    if (!c || T < 1 || K < 1 || !ws || ((uintptr_t)ws % kAlign) != 0)
        return LBM_ERR_ARG;
    if (!adj_supported(c))
        return LBM_ERR_ARG;
    if (!c->initialized)
        return LBM_ERR_STATE;
    const AdjLayout a = adj_layout(c, T, K);
    if (bytes < a.total)
        return LBM_ERR_NOMEM;
    c->adj_ready = false;
    if (cudaMemcpyAsync(at(ws, a.ckpt_off), c->f[c->cur], c->state_bytes,
                        cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
        return LBM_ERR_CUDA;
    const void *src = c->f[c->cur];
    for (int64_t k = 1; k <= T; ++k) {
        void *dst;
        if (k % K == 0 && k < T)
            dst = at(ws, a.ckpt_off + a.ckpt_stride * (size_t)(k / K));
        else
            dst = (src == c->f[0]) ? c->f[1] : c->f[0];
        const int rc = ctx_launch_step(c, src, dst, PAT_PULL, nullptr);
        if (rc != LBM_OK)
            return rc;
        src = dst;
    }
    c->cur = (src == c->f[0]) ? 0 : 1;
    c->step += T;
    double r[6];
    const int rc = lbm_reduce(c, r);
    if (rc != LBM_OK)
        return rc;
    if (J)
        *J = r[4];
    Launch l = ctx_base_launch(c, K_SEED);
    l.ap.state = c->f[c->cur];
    l.ap.lam_out = at(ws, a.lam_off[0]);
    l.ap.gF = at(ws, a.gF_off);
    if (ctx_dispatch(c, l) != cudaSuccess)
        return LBM_ERR_CUDA;
    c->adj_T = T;
    c->adj_K = K;
    c->adj_ws = ws;
    c->adj_bytes = bytes;
    c->adj_ready = true;
    return LBM_OK;
}

int lbm_adjoint_backward(lbm_ctx *c, void *ws, size_t bytes, double *dJdF, double *dJdU)
{
    if (!c || !ws)
        return LBM_ERR_ARG;
    if (!c->adj_ready || ws != c->adj_ws || bytes != c->adj_bytes)
        return LBM_ERR_STATE;
    const int64_t T = c->adj_T, K = c->adj_K;
    const AdjLayout a = adj_layout(c, T, K);
    const size_t N = (size_t)c->N;
    const size_t dN = (size_t)c->d * N;
    cudaStream_t s = c->stream;
    if (dJdF && cudaMemsetAsync(dJdF, 0, dN * sizeof(double), s) != cudaSuccess)
        return LBM_ERR_CUDA;
    double *gU_part = (double *)at(ws, a.gU_off);
    if (cudaMemsetAsync(gU_part, 0, (size_t)a.gU_n * 4 * sizeof(double), s) != cudaSuccess)
        return LBM_ERR_CUDA;
    const int out_f32 = a.real == 4 ? 1 : 0;
    int li = 0;
    for (int64_t sg = a.nseg - 1; sg >= 0; --sg) {
        const int64_t k0 = sg * K, k1 = (k0 + K < T) ? k0 + K : T;
        const void *ck = at(ws, a.ckpt_off + a.ckpt_stride * (size_t)sg);
        int rc = ctx_launch_moments(c, ck, FORM_LOCAL, nullptr, at(ws, a.useg_off), out_f32,
                                    nullptr);
        if (rc != LBM_OK)
            return rc;
        const void *src = ck;
        for (int64_t k = k0 + 1; k < k1; ++k) {
            void *dst = at(ws, a.rec_off[(k - k0 - 1) % 2]);
            rc = ctx_launch_step(c, src, dst, PAT_PULL,
                                 at(ws, a.useg_off + a.useg_stride * (size_t)(k - k0)));
            if (rc != LBM_OK)
                return rc;
            src = dst;
        }
        for (int64_t k = k1 - 1; k >= k0; --k) {
            Launch l = ctx_base_launch(c, K_ADJ);
            l.ap.lam_in = at(ws, a.lam_off[li]);
            l.ap.lam_out = at(ws, a.lam_off[1 - li]);
            l.ap.u_k = at(ws, a.useg_off + a.useg_stride * (size_t)(k - k0));
            l.ap.gF = at(ws, a.gF_off);
            l.ap.gU_part = gU_part;
            l.ap.xseg = (c->nx + c->bx - 1) / c->bx;
            if (ctx_dispatch(c, l) != cudaSuccess)
                return LBM_ERR_CUDA;
            li = 1 - li;
        }
        Launch f = ctx_base_launch(c, K_FLUSH);
        f.ap.gF = at(ws, a.gF_off);
        f.ap.dJdF = dJdF;
        f.count = dN;
        f.grid = dim3(1184, 1, 1);
        f.block = dim3(256, 1, 1);
        if (ctx_dispatch(c, f) != cudaSuccess)
            return LBM_ERR_CUDA;
    }
    double *gU = (double *)(at(ws, a.gU_off) + align_up((size_t)a.gU_n * 4 * sizeof(double)));
    k_sum_columns<<<1, 256, 0, s>>>(gU_part, a.gU_n, 4, 3, gU);
    if (cudaGetLastError() != cudaSuccess)
        return LBM_ERR_CUDA;
    double host[3];
    if (cudaMemcpyAsync(host, gU, sizeof(host), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return LBM_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess)
        return LBM_ERR_CUDA;
    if (dJdU)
        for (int k = 0; k < 3; ++k)
            dJdU[k] = host[k];
    c->adj_ready = false;  // the seed has been consumed
    return LBM_OK;
}

int lbm_adjoint(lbm_ctx *c, int64_t T, int64_t K, void *ws, size_t bytes, double *J,
                double *dJdF, double *dJdU)
{
    int rc = lbm_adjoint_forward(c, T, K, ws, bytes, J);
    if (rc != LBM_OK)
        return rc;
    return lbm_adjoint_backward(c, ws, bytes, dJdF, dJdU);
}

}  // extern "C"
