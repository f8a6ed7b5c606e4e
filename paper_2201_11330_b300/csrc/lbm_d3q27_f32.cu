// lbm_d3q27_f32.cu -- kernel instantiations for D3Q27 with F32 storage.
#include "lbm_launch.cuh"

namespace lbm {
// the MRT launches are instantiated in lbm_d3q27_f32_mrt.cu
extern template cudaError_t launch_mrt<D3Q27, ST_F32>(const Launch &);
cudaError_t launch_d3q27_f32(const Launch &l) { return launch_storage<D3Q27, ST_F32>(l); }
}  // namespace lbm
