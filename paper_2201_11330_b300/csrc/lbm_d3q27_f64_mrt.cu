// lbm_d3q27_f64_mrt.cu -- MRT kernel instantiations for D3Q27 with F64 storage
// (a unit of its own so that it compiles in parallel with lbm_d3q27_f64.cu).
#include "lbm_launch.cuh"

namespace lbm {
template cudaError_t launch_mrt<D3Q27, ST_F64>(const Launch &);
}  // namespace lbm
