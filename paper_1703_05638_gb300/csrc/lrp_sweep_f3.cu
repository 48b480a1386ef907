// One instantiation of the persistent sweep kernel (compiled separately so
// the four variants build in parallel).
#include "lrp_sweep_kernel.cuh"

namespace lrp {
template cudaError_t launch_sweep<float, 3, true>(const SweepParams&, cudaStream_t);
template int max_resident_teams<float, 3, true>(int, int, size_t, int);
}  // namespace lrp
