// lbm_d3q19_f64.cu -- kernel instantiations for D3Q19 with F64 storage.
#include "lbm_launch.cuh"

namespace lbm {
cudaError_t launch_d3q19_f64(const Launch &l) { return launch_storage<D3Q19, ST_F64>(l); }
}  // namespace lbm
