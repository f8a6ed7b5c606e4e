// lbm_d3q19_bf16s.cu -- kernel instantiations for D3Q19 with BF16S storage.
#include "lbm_launch.cuh"

namespace lbm {
cudaError_t launch_d3q19_bf16s(const Launch &l) { return launch_storage<D3Q19, ST_BF16S>(l); }
}  // namespace lbm
