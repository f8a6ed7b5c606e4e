// lbm_d2q9.cu -- instantiation unit for the D2Q9 velocity set (Sec. 2.1).
#include "lbm_launch.cuh"

namespace lbm {
cudaError_t launch_d2q9(const Launch &l) { return launch_lattice<D2Q9>(l); }
}  // namespace lbm
