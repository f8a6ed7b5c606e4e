// lbm_d3q27.cu -- instantiation unit for the D3Q27 velocity set (Sec. 2.1).
#include "lbm_launch.cuh"

namespace lbm {
cudaError_t launch_d3q27(const Launch &l) { return launch_lattice<D3Q27>(l); }
}  // namespace lbm
