// Allocation-free Hessian apply.
//
// Some callers cannot call cudaMalloc while they run: a serving process whose
// device memory is entirely reserved up front by another allocator (a
// framework's caching pool), or a latency-critical loop where a cudaMalloc
// would synchronise the device and stall other streams. For them this file
// provides lrp_hessian_apply_noalloc: the same computation as
// lrp_hessian_apply, but its solver workspace is a fixed array in device
// memory that exists from the moment the library is loaded, so the call
// itself allocates nothing. The problem handle (created earlier by
// lrp_setup_problem) and the caller's input and output arrays are used as
// they are.
#include <cuda_runtime.h>

#include <chrono>
#include <mutex>
#include <string>

#include "lrp_internal.h"

// The fixed workspace. Every GPU that loads this library holds it until the
// process exits.
#define LRP_NOALLOC_WS_BYTES (64u << 20)
static __device__ __align__(256) unsigned char g_noalloc_ws[LRP_NOALLOC_WS_BYTES];

namespace lrp {

// Device address of g_noalloc_ws, looked up once per device with that device
// current. In host code the array's name is only a host-side stand-in, so
// the kernels receive this looked-up address.
static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[64] = {};

static lrp_status noalloc_workspace(int device, void** out) {
  if (device < 0 || device >= 64) {
    set_error("device index out of range for the fixed workspace table");
    return LRP_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[device]) {
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetDevice");
    if (cur != device) {
      e = cudaSetDevice(device);
      if (e != cudaSuccess) return cuda_status(e, "cudaSetDevice");
    }
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_ws);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(g_noalloc_ws)");
    g_noalloc_addr[device] = p;
  }
  *out = g_noalloc_addr[device];
  return LRP_OK;
}

}  // namespace lrp

using namespace lrp;

extern "C" lrp_status lrp_hessian_apply_noalloc(lrp_problem* P, int nvec, const double* X, int ldx, double* Y,
                                                int ldy, lrp_apply_stats* st) {
  if (!P || !X || !Y) {
    set_error("lrp_hessian_apply_noalloc: NULL argument");
    return LRP_EINVAL;
  }
  if (nvec < 0 || ldx < P->nx || ldy < P->nx) {
    set_error("lrp_hessian_apply_noalloc: invalid nvec or leading dimension");
    return LRP_EINVAL;
  }
  if (nvec == 0) return LRP_OK;
  // host arrays would need staging buffers, i.e. an allocation
  if (!is_device_ptr(X) || !is_device_ptr(Y)) {
    set_error("lrp_hessian_apply_noalloc: X and Y must be device arrays");
    return LRP_EINVAL;
  }
  {
    lrp_status sd = check_on_device(P->device, X, "lrp_hessian_apply_noalloc X");
    if (sd == LRP_OK) sd = check_on_device(P->device, Y, "lrp_hessian_apply_noalloc Y");
    if (sd != LRP_OK) return sd;
  }
  auto t0 = std::chrono::steady_clock::now();
  cudaError_t e = cudaSetDevice(P->device);
  if (e != cudaSuccess) return cuda_status(e, "cudaSetDevice");
  void* ws = nullptr;
  lrp_status s = noalloc_workspace(P->device, &ws);
  if (s != LRP_OK) return s;
  // the sweep sizes its needs and rejects them if they exceed the array
  P->ws_fixed = (char*)ws;
  P->ws_fixed_bytes = LRP_NOALLOC_WS_BYTES;
  const unsigned stages = ST_LOAD_X | ST_PRIOR_IN | ST_FORWARD | ST_ADJOINT | ST_PRIOR_OUT | ST_STORE_Y;
  s = run_sweep(P, stages, nvec, X, ldx, Y, ldy, nullptr, 0, nullptr, 0, st, false);
  P->ws_fixed = nullptr;
  P->ws_fixed_bytes = 0;
  if (st) st->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return s;
}
