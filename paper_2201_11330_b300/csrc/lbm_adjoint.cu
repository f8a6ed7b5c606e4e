// lbm_adjoint.cu -- placeholder until the adjoint kernels land.
#include "lbm_capi_internal.h"

extern "C" {
size_t lbm_adjoint_workspace_bytes(const lbm_ctx *, int64_t, int64_t) { return 0; }
int lbm_adjoint_forward(lbm_ctx *, int64_t, int64_t, void *, size_t, double *) { return LBM_ERR_STATE; }
int lbm_adjoint_backward(lbm_ctx *, void *, size_t, double *, double *) { return LBM_ERR_STATE; }
int lbm_adjoint(lbm_ctx *, int64_t, int64_t, void *, size_t, double *, double *, double *) { return LBM_ERR_STATE; }
}
