// FP64 helpers with short dependency chains. On this part a dependent FP64
// operation costs ~64 cycles and a library FP64 divide or square root ~650,
// so serial FP64 code (the QL rotation chase) is bound by these latencies.
#pragma once

#include <cuda_runtime.h>

namespace lrp {

// sqrt(t) and 1/sqrt(t) for a positive normal double t, from an FP32
// reciprocal-square-root seed refined by two steps of Goldschmidt's
// iteration (R. E. Goldschmidt, 1964): with g ~ sqrt(t) and h ~ 1/(2 sqrt(t)),
// r = 1/2 - g h, g <- g + g r, h <- h + h r; each step roughly squares the
// relative error (seed ~2^-22, so two steps reach rounding level). t is first
// scaled by an exact power of four into [1, 4), so the FP32 seed neither
// overflows nor underflows, and the results are scaled back exactly.
// Returns false (outputs untouched) for t <= 0, subnormal, infinite or NaN
// t: the caller then takes the library path.
__device__ __forceinline__ bool sqrt_rsqrt_gs(double t, double* sq, double* rs) {
  const int hi = __double2hiint(t);
  const int ex = (hi >> 20) & 0x7ff;  // biased exponent
  if (hi < 0 || ex == 0 || ex == 0x7ff) return false;
  const int k = (ex - 1023) >> 1;  // t = ts 4^k, ts in [1, 4)
  const double ts = __hiloint2double(hi - (k << 21), __double2loint(t));
  const double y0 = (double)rsqrtf(__double2float_rn(ts));
  double g = ts * y0;
  double h = 0.5 * y0;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const double r = fma(-g, h, 0.5);
    g = fma(g, r, g);
    h = fma(h, r, h);
  }
  // 2^k and 2^-k exactly (|k| <= 511)
  const double up = __hiloint2double((k + 1023) << 20, 0);
  const double dn = __hiloint2double((1023 - k) << 20, 0);
  *sq = g * up;
  *rs = 2.0 * h * dn;
  return true;
}

}  // namespace lrp
