// lbm_d3q27_f64.cu -- kernel instantiations for D3Q27 with F64 storage.
#include "lbm_launch.cuh"

namespace lbm {
cudaError_t launch_d3q27_f64(const Launch &l) { return launch_storage<D3Q27, ST_F64>(l); }
}  // namespace lbm
