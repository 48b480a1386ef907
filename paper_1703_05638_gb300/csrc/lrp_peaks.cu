// Device peak rates measured with the library's own kernels (no
// counterpart in the paper): the denominators of the roofline figures for
// the kernels whose bound is not HBM bandwidth.
//  * shared-memory bandwidth: every CTA streams 16-byte loads and stores
//    through its shared memory (no bank conflicts) for a fixed number of
//    rounds; bytes moved / time over all SMs;
//  * FP64 and FP32 FMA throughput: every thread runs 8 independent FMA
//    chains; 2 flops per FMA / time over all SMs.
// Each figure is the best of three timed launches (CUDA events), after one
// untimed launch.
#include <cuda_runtime.h>

#include "lrp_internal.h"

namespace lrp {
namespace {

constexpr int kSmemThreads = 512;
constexpr int kSmemFloat4 = 2048;  // 32 KB per CTA (static shared memory)

__device__ __forceinline__ float4 lds128(unsigned a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a)
               : "memory");
  return v;
}
__device__ __forceinline__ void sts128(unsigned a, float4 v) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
               : "memory");
}

__global__ void __launch_bounds__(kSmemThreads) k_smem_stream(int rounds, float* sink) {
  __shared__ float4 buf[kSmemFloat4];
  const int t = threadIdx.x;
  for (int i = t; i < kSmemFloat4; i += kSmemThreads) buf[i] = make_float4(i, 1.f, 2.f, 3.f);
  __syncthreads();
  const unsigned base = (unsigned)__cvta_generic_to_shared(buf);
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int r = 0; r < rounds; ++r) {
    // each thread loads 4 float4 and stores them back every round (volatile
    // shared-memory accesses: the compiler may not keep them in registers);
    // consecutive threads touch consecutive 16-byte words (conflict-free)
    float4 v[kSmemFloat4 / kSmemThreads];
#pragma unroll
    for (int j = 0; j < kSmemFloat4 / kSmemThreads; ++j) v[j] = lds128(base + 16u * (t + j * kSmemThreads));
#pragma unroll
    for (int j = 0; j < kSmemFloat4 / kSmemThreads; ++j) {
      acc.x += v[j].x;
      acc.y += v[j].y;
      v[j].z += 1.f;
      sts128(base + 16u * (t + j * kSmemThreads), v[j]);
    }
  }
  __syncthreads();
  if (acc.x + acc.y == -1.f) sink[blockIdx.x] = acc.x;  // never true; keeps the loads
}

template <typename T>
__global__ void __launch_bounds__(256) k_fma(int iters, T a, T b, T* sink) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = x[k] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == (T)-1) sink[blockIdx.x] = s;  // never true for these inputs
}

template <class Launch>
static cudaError_t best_ms(Launch launch, float* out_ms) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  float best = 1e30f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    e = cudaEventRecord(e0);
    if (e == cudaSuccess) {
      note_launch();
      launch();
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0) best = ms < best ? ms : best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *out_ms = best;
  return e;
}

}  // namespace
}  // namespace lrp

using namespace lrp;

extern "C" lrp_status lrp_measure_device_peaks(lrp_device_peaks* out) {
  if (!out) {
    set_error("lrp_measure_device_peaks: NULL argument");
    return LRP_EINVAL;
  }
  int dev = 0, sms = 0, mhz = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&mhz, cudaDevAttrClockRate, dev);
  if (e != cudaSuccess) return cuda_status(e, "lrp_measure_device_peaks: device query");
  float* sink = nullptr;
  e = dev_malloc(&sink, 4096 * sizeof(float));
  if (e != cudaSuccess) return cuda_status(e, "lrp_measure_device_peaks: sink");
  const int smem_blocks = sms * 4;  // several 32 KB CTAs per SM
  const int smem_rounds = 2000;
  float ms_smem = 0.f, ms_d = 0.f, ms_f = 0.f;
  e = best_ms([&] { k_smem_stream<<<smem_blocks, kSmemThreads>>>(smem_rounds, sink); }, &ms_smem);
  const int fma_blocks = sms * 8, fma_iters = 4096;
  if (e == cudaSuccess)
    e = best_ms([&] { k_fma<double><<<fma_blocks, 256>>>(fma_iters, 0.999999, 1e-7, (double*)sink); }, &ms_d);
  const int fma32_iters = 65536;
  if (e == cudaSuccess)
    e = best_ms([&] { k_fma<float><<<fma_blocks, 256>>>(fma32_iters, 0.999999f, 1e-7f, sink); }, &ms_f);
  cudaFree(sink);
  if (e != cudaSuccess) return cuda_status(e, "lrp_measure_device_peaks: timing");
  const double smem_bytes = (double)smem_blocks * smem_rounds * (kSmemFloat4 * 16.0) * 2.0;  // load + store
  const double fma_threads = (double)fma_blocks * 256 * 8;
  out->smem_gbs = smem_bytes / (ms_smem * 1e-3) / 1e9;
  out->fp64_fma_tflops = fma_threads * fma_iters * 2.0 / (ms_d * 1e-3) / 1e12;
  out->fp32_fma_tflops = fma_threads * fma32_iters * 2.0 / (ms_f * 1e-3) / 1e12;
  out->sm_count = sms;
  out->clock_mhz = mhz / 1000.0;
  return LRP_OK;
}
