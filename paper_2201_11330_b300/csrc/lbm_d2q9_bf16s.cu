// lbm_d2q9_bf16s.cu -- kernel instantiations for D2Q9 with BF16S storage.
#include "lbm_launch.cuh"

namespace lbm {
cudaError_t launch_d2q9_bf16s(const Launch &l) { return launch_storage<D2Q9, ST_BF16S>(l); }
}  // namespace lbm
