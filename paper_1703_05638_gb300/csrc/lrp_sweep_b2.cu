// One instantiation of the persistent sweep kernel: the mixed path with the
// multigrid vectors of the global-memory levels stored in BF16 (compiled
// separately so the variants build in parallel).
#include "lrp_sweep_kernel.cuh"

namespace lrp {
template cudaError_t launch_sweep<float, 2, true, __nv_bfloat16>(const SweepParams&, cudaStream_t);
template int max_resident_teams<float, 2, true, __nv_bfloat16>(int, int, size_t, int);
}  // namespace lrp
