// One instantiation of the persistent sweep kernel (compiled separately so
// the four variants build in parallel).
#include "lrp_sweep_kernel.cuh"

namespace lrp {
template cudaError_t launch_sweep<double, 3, false>(const SweepParams&, cudaStream_t);
template int max_resident_teams<double, 3, false>(int, int, size_t, int);
}  // namespace lrp
