// lbm_d3q19.cu -- instantiation unit for the D3Q19 velocity set (Sec. 2.1).
#include "lbm_launch.cuh"

namespace lbm {
cudaError_t launch_d3q19(const Launch &l) { return launch_lattice<D3Q19>(l); }
}  // namespace lbm
