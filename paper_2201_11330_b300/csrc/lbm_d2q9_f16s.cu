// lbm_d2q9_f16s.cu -- kernel instantiations for D2Q9 with F16S storage.
#include "lbm_launch.cuh"

namespace lbm {
cudaError_t launch_d2q9_f16s(const Launch &l) { return launch_storage<D2Q9, ST_F16S>(l); }
}  // namespace lbm
