// lbm_capi_internal.h -- the context object and helpers shared by the host
// translation units (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm.h"
#include "lbm_kernels.cuh"

struct lbm_ctx {
    int lattice, Q, d;
    int nx, ny, nz;
    int64_t N;
    double tau;
    int bc;
    lbm_opts opts;
    bool shifted;
    char *ws;
    size_t ws_bytes;
    void *f[2];  // pull scheme: current state f[cur]; AA: f[0] only
    int cur;
    size_t state_bytes;
    int nred;  // moment-kernel blocks (reduction partials)
    double *partials;
    double *result;
    double *step_partials;  // per-block monitor sums of a reducing step
    long long step_blocks;  // capacity of step_partials (blocks)
    cudaStream_t stream;
    const float *force;
    int64_t step;
    int bx;  // threads per block along x
    bool initialized;
    int kernel_variant;  // lbm_kernel_variant
    // per-face boundaries and obstacles (the general step kernel)
    bool geo;                   // LBM_BC_FACES or obstacles
    int face[6];                // lbm_face per face
    unsigned *links;            // per-node link words (workspace), or NULL
    bool links_ready;           // lbm_set_geometry has run
    unsigned long long *count;  // solid-node counter (workspace)
    int64_t n_fluid;            // nodes that are not solid
    unsigned char *nflags;      // per-node "needs the general kernel" flags (workspace)
    int *nlist;                 // the nodes that need the general kernel (workspace)
    bool list_ready;
    bool list_pairs;            // the list was built for the paired kernel
    long long n_general;        // entries of nlist
    // CUDA graphs of lbm_step's launches (launch-bound small problems)
    int graph_mode;            // -1 automatic, 0 off, else steps per graph (even)
    long long param_version;   // bumped by every change of the launch parameters
    cudaStream_t cap_stream;   // private stream the graphs are captured on
    cudaGraphExec_t graph[2];  // by the starting AA parity / pull lattice
    long long graph_version[2];
    int graph_len[2];
    lbm::StepParams sp;
    // adjoint run recorded by lbm_adjoint_forward for lbm_adjoint_backward
    int64_t adj_T, adj_K;
    void *adj_ws;
    size_t adj_bytes;
    bool adj_ready;
};

namespace lbm {
// lbm_opts that lbm_create accepts (the option checks, without the shape)
bool ctx_opts_valid(const lbm_opts &o);
lbm::Launch ctx_base_launch(const lbm_ctx *c, int kind);
cudaError_t ctx_dispatch(const lbm_ctx *c, const lbm::Launch &l);
int ctx_launch_step(lbm_ctx *c, const void *src, void *dst, int pattern, void *u_out,
                    long long *reduce_blocks = nullptr, bool obstacle_force = false);
int ctx_launch_moments(lbm_ctx *c, const void *src, int form, void *p_out, void *u_out,
                       int out_f32, double *partials);
// the six monitor sums of a state (per-block FP64 partials of the moments
// kernel, then a fixed-order reduction); synchronises the stream
int ctx_reduce_state(lbm_ctx *c, const void *src, int form, double r[6]);
int ctx_current_form(const lbm_ctx *c);
const void *ctx_state(const lbm_ctx *c);
}  // namespace lbm
