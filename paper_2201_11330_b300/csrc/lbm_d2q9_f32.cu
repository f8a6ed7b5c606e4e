// lbm_d2q9_f32.cu -- kernel instantiations for D2Q9 with F32 storage.
#include "lbm_launch.cuh"

namespace lbm {
// the MRT launches are instantiated in lbm_d2q9_f32_mrt.cu
extern template cudaError_t launch_mrt<D2Q9, ST_F32>(const Launch &);
cudaError_t launch_d2q9_f32(const Launch &l) { return launch_storage<D2Q9, ST_F32>(l); }
}  // namespace lbm
