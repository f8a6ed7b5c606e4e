// lbm_d3q19_f64_mrt.cu -- MRT kernel instantiations for D3Q19 with F64 storage
// (a unit of its own so that it compiles in parallel with lbm_d3q19_f64.cu).
#include "lbm_launch.cuh"

namespace lbm {
template cudaError_t launch_mrt<D3Q19, ST_F64>(const Launch &);
}  // namespace lbm
