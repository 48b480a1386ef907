// One instantiation of the persistent sweep kernel (compiled separately so
// the four variants build in parallel).
#include "lrp_sweep_kernel.cuh"

namespace lrp {
template cudaError_t launch_sweep<float, 3, true>(const SweepParams&, cudaStream_t);
}  // namespace lrp
