// lbm_d3q19_f64.cu -- kernel instantiations for D3Q19 with F64 storage.
#include "lbm_launch.cuh"

namespace lbm {
// the MRT launches are instantiated in lbm_d3q19_f64_mrt.cu
extern template cudaError_t launch_mrt<D3Q19, ST_F64>(const Launch &);
cudaError_t launch_d3q19_f64(const Launch &l) { return launch_storage<D3Q19, ST_F64>(l); }
}  // namespace lbm
