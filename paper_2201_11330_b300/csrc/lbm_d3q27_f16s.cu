// lbm_d3q27_f16s.cu -- kernel instantiations for D3Q27 with F16S storage.
#include "lbm_launch.cuh"

namespace lbm {
cudaError_t launch_d3q27_f16s(const Launch &l) { return launch_storage<D3Q27, ST_F16S>(l); }
}  // namespace lbm
