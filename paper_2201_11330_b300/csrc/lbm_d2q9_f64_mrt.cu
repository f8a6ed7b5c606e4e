// lbm_d2q9_f64_mrt.cu -- MRT kernel instantiations for D2Q9 with F64 storage
// (a unit of its own so that it compiles in parallel with lbm_d2q9_f64.cu).
#include "lbm_launch.cuh"

namespace lbm {
template cudaError_t launch_mrt<D2Q9, ST_F64>(const Launch &);
}  // namespace lbm
