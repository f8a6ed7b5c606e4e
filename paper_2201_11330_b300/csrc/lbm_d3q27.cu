// lbm_d3q27.cu -- storage dispatch for the D3Q27 velocity set (Sec. 2.1); the
// kernels of each storage type are instantiated in lbm_d3q27_<storage>.cu.
#include "lbm_kernels.cuh"

namespace lbm {
cudaError_t launch_d3q27_f64(const Launch &l);
cudaError_t launch_d3q27_f32(const Launch &l);
cudaError_t launch_d3q27_f16s(const Launch &l);
cudaError_t launch_d3q27_bf16s(const Launch &l);

cudaError_t launch_d3q27(const Launch &l)
{
    switch (l.storage) {
    case ST_F64:
        return launch_d3q27_f64(l);
    case ST_F32:
        return launch_d3q27_f32(l);
    case ST_F16S:
        return launch_d3q27_f16s(l);
    case ST_BF16S:
        return launch_d3q27_bf16s(l);
    }
    return cudaErrorInvalidValue;
}
}  // namespace lbm
