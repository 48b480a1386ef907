// Launcher of the shared-memory-resident 2D sweep kernel (lrp_fast2d.cuh).
#include "lrp_fast2d.cuh"

namespace lrp {

static cudaError_t prepare_fast2d(size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(fast2d_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  const int cap = smem_dynamic_max(fast2d_kernel);  // one value for every launcher (see prepare_sweep)
  if ((long long)smem > cap) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(fast2d_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
}

cudaError_t launch_fast2d(const SweepParams& prm, cudaStream_t stream) {
  cudaError_t e = prepare_fast2d(prm.smem_bytes);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(prm.n_teams * prm.C);
  cfg.blockDim = dim3(prm.NT);
  cfg.dynamicSmemBytes = prm.smem_bytes;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  int na = 0;
  if (prm.C > 1) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = prm.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    na = 1;
  }
  cfg.attrs = attr;
  cfg.numAttrs = na;
  return cudaLaunchKernelEx(&cfg, fast2d_kernel, prm);
}

int fast2d_resident_teams(int C, int NT, size_t smem, int sm_count) {
  if (prepare_fast2d(smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (C == 1) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fast2d_kernel, NT, smem) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return per_sm * sm_count;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C * 64);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, fast2d_kernel, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

}  // namespace lrp
