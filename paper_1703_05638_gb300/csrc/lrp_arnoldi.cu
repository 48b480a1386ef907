// Arnoldi process of Sec. 4 Algorithm 1 (single vectors, modified
// Gram-Schmidt against every previous vector, Hessenberg matrix H), its
// Ritz values by the Francis double-shift QR iteration on H (real Schur
// form with Schur vectors), Ritz vectors by back substitution on the
// quasi-triangular factor, and a posterior built from the real Ritz pairs.
// The operator is either the exact Htilde or the truncated product of
// Algorithm 1 (LRP_LOWRANK_SOURCE), which is not exactly symmetric.
// Host code drives the iteration; every arithmetic step runs in kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "lrp_dense.h"
#include "lrp_internal.h"

namespace lrp {
namespace {

constexpr int kMgsThreads = 1024;

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();  // red[] is free (previous readers are done)
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < nw; ++i) s += red[i];  // same order in every thread
  return s;
}

// One Arnoldi orthogonalisation (Algorithm 1's inner loop, as printed): for
// i = 0..j, h_ij = v_i . w, w <- w - h_ij v_i (modified Gram-Schmidt, one
// vector at a time); h_{j+1,j} = ||w||, v_{j+1} = w / h_{j+1,j} (zero if w
// vanished). V: nx x (j+2) basis (ld nx), w: nx, H column j at Hcol (rows
// 0..j+1). One CTA; every thread owns the same entries of w throughout.
__global__ void __launch_bounds__(kMgsThreads) k_arnoldi_mgs(int nx, int j, double* V, double* w, double* Hcol) {
  __shared__ double red[32];
  for (int i = 0; i <= j; ++i) {
    const double* vi = V + (size_t)i * nx;
    double d = 0.0;
    for (int p = threadIdx.x; p < nx; p += blockDim.x) d += vi[p] * w[p];
    const double h = block_sum(d, red);
    for (int p = threadIdx.x; p < nx; p += blockDim.x) w[p] -= h * vi[p];
    if (threadIdx.x == 0) Hcol[i] = h;
  }
  double d = 0.0;
  for (int p = threadIdx.x; p < nx; p += blockDim.x) d += w[p] * w[p];
  const double nrm = sqrt(block_sum(d, red));
  if (threadIdx.x == 0) Hcol[j + 1] = nrm;
  double* vn = V + (size_t)(j + 1) * nx;
  const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
  for (int p = threadIdx.x; p < nx; p += blockDim.x) vn[p] = w[p] * inv;
}

// v <- v / ||v||
__global__ void __launch_bounds__(kMgsThreads) k_normalize(int nx, double* v) {
  __shared__ double red[32];
  double d = 0.0;
  for (int p = threadIdx.x; p < nx; p += blockDim.x) d += v[p] * v[p];
  const double nrm = sqrt(block_sum(d, red));
  const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
  for (int p = threadIdx.x; p < nx; p += blockDim.x) v[p] *= inv;
}

// ---------------------------------------------------------------------------
// Francis double-shift QR iteration (the implicitly shifted QR algorithm for
// a real upper Hessenberg matrix; e.g. Golub & Van Loan, Matrix
// Computations, Sec. 7.5): T is reduced in place to real Schur form
// (quasi-upper-triangular, 1x1 and 2x2 diagonal blocks) by orthogonal
// similarities, which are accumulated into Z (H = Z T Z^T). Deflation from
// the bottom: a subdiagonal entry below eps (|t_{l-1,l-1}| + |t_ll|) splits
// the active window; a 1x1 block is a real eigenvalue; a 2x2 block with real
// eigenvalues is triangularised by one reflector, one with complex
// eigenvalues is kept. Otherwise one double-shift step on the window
// (shifts: the eigenvalues of its trailing 2x2 block; an exceptional shift
// after every 10 iterations without deflation) chases a 3x3 bulge down by
// 3-vector Householder reflectors and ends with a 2-vector one.
// Thread 0 makes every decision and computes each reflector; all threads
// apply it (left to rows k..k+nv-1 from column c_lo on, right to columns
// k..k+nv-1 of rows 0..r_hi, and to Z). Column-major, ld m.
// status: 0 converged, 1 iteration cap (30 m double-shift steps) reached.
struct HqrState {
  int hi, l, k, its, total, phase;  // phase 0: search/deflate, 1: chasing
  double tr, det;
};

__device__ void householder(int nv, double x, double y, double z, double* v, double* beta) {
  const double nrm = sqrt(x * x + y * y + (nv == 3 ? z * z : 0.0));
  if (nrm == 0.0) {
    *beta = 0.0;
    v[0] = v[1] = v[2] = 0.0;
    return;
  }
  const double alpha = x >= 0.0 ? -nrm : nrm;
  v[0] = x - alpha;
  v[1] = y;
  v[2] = nv == 3 ? z : 0.0;
  const double vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  *beta = vv > 0.0 ? 2.0 / vv : 0.0;
}

__global__ void __launch_bounds__(256) k_hqr(int m, double* T, double* Z, double* wr, double* wi, int* status) {
  // command for the whole block: nv = 0 -> nothing to apply this round,
  // nv < 0 -> finished
  __shared__ double s_v[3];
  __shared__ double s_beta;
  __shared__ int s_k, s_nv, s_clo, s_rhi;
  const int tid = threadIdx.x, nth = blockDim.x;
  auto at = [&](int r, int c) -> double& { return T[(size_t)c * m + r]; };
  for (int e = tid; e < m * m; e += nth) Z[e] = (e % m == e / m) ? 1.0 : 0.0;
  HqrState st;
  st.hi = m - 1;
  st.l = 0;
  st.k = 0;
  st.its = 0;
  st.total = 0;
  st.phase = 0;
  st.tr = st.det = 0.0;
  double anorm = 0.0;
  if (tid == 0) {
    for (int c = 0; c < m; ++c)
      for (int r = 0; r <= min(c + 1, m - 1); ++r) anorm = fmax(anorm, fabs(at(r, c)));
    if (anorm == 0.0) anorm = 1.0;
    *status = 0;
  }
  __syncthreads();
  const double eps = 2.220446049250313e-16;
  for (;;) {
    if (tid == 0) {
      int nv = 0, k = 0, clo = 0, rhi = 0;
      double v[3] = {0.0, 0.0, 0.0}, beta = 0.0;
      bool decided = false;
      while (!decided) {
        if (st.hi < 0) {
          nv = -1;
          decided = true;
          break;
        }
        if (st.phase == 0) {
          // find the start l of the unreduced window ending at hi
          int l = st.hi;
          while (l > 0) {
            double s = fabs(at(l - 1, l - 1)) + fabs(at(l, l));
            if (s == 0.0) s = anorm;
            if (fabs(at(l, l - 1)) <= eps * s) {
              at(l, l - 1) = 0.0;
              break;
            }
            --l;
          }
          const int hi = st.hi;
          if (l == hi) {  // 1x1 block
            wr[hi] = at(hi, hi);
            wi[hi] = 0.0;
            st.hi -= 1;
            st.its = 0;
            continue;
          }
          if (l == hi - 1) {  // 2x2 block
            const double a = at(hi - 1, hi - 1), b = at(hi - 1, hi), c = at(hi, hi - 1), d = at(hi, hi);
            const double p = 0.5 * (a - d), disc = p * p + b * c;
            if (disc >= 0.0) {
              const double sq = sqrt(disc);
              const double zz = p + (p >= 0.0 ? sq : -sq);
              const double l1 = d + zz;
              const double l2 = zz != 0.0 ? d - b * c / zz : l1;
              // eigenvector of l1: the better conditioned of (b, l1 - a), (l1 - d, c)
              double u0 = b, u1 = l1 - a;
              const double w0 = l1 - d, w1 = c;
              if (w0 * w0 + w1 * w1 > u0 * u0 + u1 * u1) {
                u0 = w0;
                u1 = w1;
              }
              wr[hi - 1] = l1;
              wr[hi] = l2;
              wi[hi - 1] = wi[hi] = 0.0;
              householder(2, u0, u1, 0.0, v, &beta);
              nv = 2;
              k = hi - 1;
              clo = hi - 1;
              rhi = hi;
              st.phase = 2;  // zero the subdiagonal entry after the reflector
              decided = true;
            } else {
              wr[hi - 1] = wr[hi] = d + p;
              wi[hi - 1] = sqrt(-disc);
              wi[hi] = -sqrt(-disc);
              st.hi -= 2;
              st.its = 0;
            }
            continue;
          }
          // double-shift step on the window [l, hi]
          if (st.total >= 30 * m) {
            *status = 1;
            nv = -1;
            decided = true;
            break;
          }
          st.its += 1;
          st.total += 1;
          if (st.its % 10 == 0) {
            const double s = fabs(at(hi, hi - 1)) + fabs(at(hi - 1, hi - 2));
            st.tr = 1.5 * s;
            st.det = s * s;
          } else {
            const double a = at(hi - 1, hi - 1), b = at(hi - 1, hi), c = at(hi, hi - 1), d = at(hi, hi);
            st.tr = a + d;
            st.det = a * d - b * c;
          }
          st.l = l;
          const double h00 = at(l, l), h10 = at(l + 1, l), h01 = at(l, l + 1), h11 = at(l + 1, l + 1);
          const double h21 = at(l + 2, l + 1);
          const double x = h00 * h00 + h01 * h10 - st.tr * h00 + st.det;
          const double y = h10 * (h00 + h11 - st.tr);
          const double z = h10 * h21;
          householder(3, x, y, z, v, &beta);
          nv = 3;
          k = l;
          clo = l;
          rhi = min(l + 3, hi);
          st.k = l;
          st.phase = 1;
          decided = true;
        } else if (st.phase == 1) {
          // continue the chase: the bulge sits in column k-1 of the next rows
          const int hi = st.hi;
          const int k0 = st.k + 1;
          if (k0 > 1 + st.l) {
            // entries the previous reflector annihilated
            at(k0, k0 - 2) = 0.0;
            if (k0 + 1 <= hi) at(k0 + 1, k0 - 2) = 0.0;
          }
          if (k0 <= hi - 2) {
            householder(3, at(k0, k0 - 1), at(k0 + 1, k0 - 1), at(k0 + 2, k0 - 1), v, &beta);
            nv = 3;
            k = k0;
            clo = k0 - 1;
            rhi = min(k0 + 3, hi);
            st.k = k0;
            decided = true;
          } else if (k0 == hi - 1) {
            householder(2, at(k0, k0 - 1), at(k0 + 1, k0 - 1), 0.0, v, &beta);
            nv = 2;
            k = k0;
            clo = k0 - 1;
            rhi = hi;
            st.k = k0;
            decided = true;
          } else {
            // the step is complete
            at(hi, hi - 2) = 0.0;
            st.phase = 0;
          }
        } else {
          // after a 2x2 block's reflector: it is upper triangular now
          at(st.hi, st.hi - 1) = 0.0;
          st.hi -= 2;
          st.its = 0;
          st.phase = 0;
        }
      }
      s_v[0] = v[0];
      s_v[1] = v[1];
      s_v[2] = v[2];
      s_beta = beta;
      s_k = k;
      s_nv = nv;
      s_clo = clo;
      s_rhi = rhi;
    }
    __syncthreads();
    const int nv = s_nv;
    if (nv < 0) break;
    if (nv > 0 && s_beta != 0.0) {
      const int k = s_k;
      const double v0 = s_v[0], v1 = s_v[1], v2 = s_v[2], beta = s_beta;
      // left: rows k..k+nv-1, columns c_lo..m-1
      for (int c = s_clo + tid; c < m; c += nth) {
        double* col = T + (size_t)c * m + k;
        double s = v0 * col[0] + v1 * col[1] + (nv == 3 ? v2 * col[2] : 0.0);
        s *= beta;
        col[0] -= s * v0;
        col[1] -= s * v1;
        if (nv == 3) col[2] -= s * v2;
      }
      __syncthreads();
      // right: columns k..k+nv-1 of rows 0..r_hi, and of Z (all rows)
      double* c0 = T + (size_t)k * m;
      double* c1 = c0 + m;
      double* c2 = c1 + m;
      for (int r = tid; r <= s_rhi; r += nth) {
        double s = v0 * c0[r] + v1 * c1[r] + (nv == 3 ? v2 * c2[r] : 0.0);
        s *= beta;
        c0[r] -= s * v0;
        c1[r] -= s * v1;
        if (nv == 3) c2[r] -= s * v2;
      }
      double* z0 = Z + (size_t)k * m;
      double* z1 = z0 + m;
      double* z2 = z1 + m;
      for (int r = tid; r < m; r += nth) {
        double s = v0 * z0[r] + v1 * z1[r] + (nv == 3 ? v2 * z2[r] : 0.0);
        s *= beta;
        z0[r] -= s * v0;
        z1[r] -= s * v1;
        if (nv == 3) z2[r] -= s * v2;
      }
    }
    __syncthreads();
  }
  // below the first subdiagonal everything is zero in the Schur form
  for (int e = tid; e < m * m; e += nth) {
    const int r = e % m, c = e / m;
    if (r > c + 1) T[e] = 0.0;
  }
}

// Eigenvectors of the quasi-triangular Schur factor T for real eigenvalues
// on its diagonal (positions pos[s], 1x1 blocks), by back substitution:
// x_i = 1, x_r = 0 below i, and for r = i-1 .. 0 the row equations of
// (T - lambda I) x = 0, a 2x2 system where rows r-1, r form a diagonal block.
// One warp per eigenvector; X is m x nsel (ld m).
__global__ void k_schur_evec(int m, const double* T, const int* pos, int nsel, double* X) {
  const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (s >= nsel) return;
  const int i = pos[s];
  double* x = X + (size_t)s * m;
  auto at = [&](int r, int c) { return T[(size_t)c * m + r]; };
  const double lam = at(i, i);
  double tnorm = 0.0;
  for (int c = lane; c < m; c += 32) tnorm = fmax(tnorm, fabs(at(c, c)) + (c > 0 ? fabs(at(c - 1, c)) : 0.0));
  for (int o = 16; o > 0; o >>= 1) tnorm = fmax(tnorm, __shfl_xor_sync(0xffffffffu, tnorm, o));
  const double small = fmax(tnorm, 1e-300) * 2.220446049250313e-16;
  for (int r = lane; r < m; r += 32) x[r] = r == i ? 1.0 : 0.0;
  __syncwarp();
  auto dot_row = [&](int r) {
    double d = 0.0;
    for (int c = r + 1 + lane; c <= i; c += 32) d += at(r, c) * x[c];
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    return d;
  };
  double xmax = 1.0;
  int r = i - 1;
  while (r >= 0) {
    if (r > 0 && at(r, r - 1) != 0.0) {
      const double s1 = dot_row(r - 1), s2 = dot_row(r);
      const double a = at(r - 1, r - 1) - lam, b = at(r - 1, r), c = at(r, r - 1), d = at(r, r) - lam;
      double det = a * d - b * c;
      if (fabs(det) < small * small) det = det >= 0.0 ? small * small : -small * small;
      const double x0 = (-s1 * d + s2 * b) / det;
      const double x1 = (-s2 * a + s1 * c) / det;
      if (lane == 0) {
        x[r - 1] = x0;
        x[r] = x1;
      }
      xmax = fmax(xmax, fmax(fabs(x0), fabs(x1)));
      r -= 2;
    } else {
      const double s1 = dot_row(r);
      double d = at(r, r) - lam;
      if (fabs(d) < small) d = d >= 0.0 ? small : -small;
      const double x0 = -s1 / d;
      if (lane == 0) x[r] = x0;
      xmax = fmax(xmax, fabs(x0));
      r -= 1;
    }
    __syncwarp();
    if (xmax > 1e100) {  // rescale before the back substitution can overflow
      const double f = 1.0 / xmax;
      for (int q = lane; q <= i; q += 32) x[q] *= f;
      xmax = 1.0;
      __syncwarp();
    }
  }
}

// Normalise every column of Y (m x n, ld m) and return the Arnoldi residual
// estimate res[s] = beta |Y[m-1, s]| / ||Y[:, s]||.
__global__ void k_ritz_estimate(int m, int n, double* Y, double beta, double* res) {
  __shared__ double red[32];
  const int s = blockIdx.x;
  if (s >= n) return;
  double* y = Y + (size_t)s * m;
  double d = 0.0;
  for (int p = threadIdx.x; p < m; p += blockDim.x) d += y[p] * y[p];
  const double nrm = sqrt(block_sum(d, red));
  const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
  const double last = y[m - 1];
  __syncthreads();
  for (int p = threadIdx.x; p < m; p += blockDim.x) y[p] *= inv;
  if (threadIdx.x == 0) res[s] = beta * fabs(last) * inv;
}

template <typename T>
struct Buf {
  T* p = nullptr;
  Buf() = default;
  Buf(const Buf&) = delete;
  Buf& operator=(const Buf&) = delete;
  ~Buf() {
    if (p) cudaFree(p);
  }
  cudaError_t alloc(size_t n) {
    if (p) cudaFree(p);
    p = nullptr;
    return lrp::dev_malloc((void**)&p, std::max<size_t>(n, 1) * sizeof(T));
  }
  T* release() {
    T* r = p;
    p = nullptr;
    return r;
  }
};

#define CKA(call)                                           \
  do {                                                      \
    cudaError_t _e = (call);                                \
    if (_e != cudaSuccess) return cuda_status(_e, #call);   \
  } while (0)

// Schur decomposition of the m x m Hessenberg matrix in dT (device, ld m,
// overwritten by T); Z (device, m x m) gets the Schur vectors; wr, wi host.
lrp_status hessenberg_schur(cudaStream_t s, int m, double* dT, double* dZ, double* dw, int* dstat, double* wr,
                            double* wi) {
  note_launch();
  k_hqr<<<1, m <= 128 ? 64 : 128, 0, s>>>(m, dT, dZ, dw, dw + m, dstat);
  CKA(cudaGetLastError());
  std::vector<double> w(2 * (size_t)m);
  int hs = 0;
  CKA(cudaMemcpyAsync(w.data(), dw, 2 * (size_t)m * sizeof(double), cudaMemcpyDeviceToHost, s));
  CKA(cudaMemcpyAsync(&hs, dstat, sizeof(int), cudaMemcpyDeviceToHost, s));
  CKA(cudaStreamSynchronize(s));
  std::copy(w.begin(), w.begin() + m, wr);
  std::copy(w.begin() + m, w.end(), wi);
  if (hs != 0) {
    set_error("the Hessenberg QR iteration reached its iteration cap");
    return LRP_ENOCONV;
  }
  return LRP_OK;
}

}  // namespace
}  // namespace lrp

using namespace lrp;

extern "C" lrp_status lrp_hessenberg_eig(int m, const double* H, int ldh, double* wr, double* wi, double* T,
                                         double* Z) {
  if (m < 1 || !H || ldh < m || !wr || !wi || m > 4096) {
    set_error("lrp_hessenberg_eig: need 1 <= m <= 4096, ldh >= m and non-NULL H, wr, wi");
    return LRP_EINVAL;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  for (const void* a : {(const void*)H, (const void*)T, (const void*)Z}) {
    if (!a) continue;
    lrp_status sd = check_on_device(dev, a, "lrp_hessenberg_eig");
    if (sd != LRP_OK) return sd;
  }
  Buf<double> dT, dZ, dw;
  Buf<int> dst;
  CKA(dT.alloc((size_t)m * m));
  CKA(dZ.alloc((size_t)m * m));
  CKA(dw.alloc(2 * (size_t)m));
  CKA(dst.alloc(1));
  cudaStream_t s = 0;
  CKA(cudaMemcpy2DAsync(dT.p, (size_t)m * sizeof(double), H, (size_t)ldh * sizeof(double), (size_t)m * sizeof(double),
                        m, is_device_ptr(H) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  lrp_status r = hessenberg_schur(s, m, dT.p, dZ.p, dw.p, dst.p, wr, wi);
  if (r != LRP_OK && r != LRP_ENOCONV) return r;
  if (T) CKA(cudaMemcpy(T, dT.p, (size_t)m * m * sizeof(double), cudaMemcpyDefault));
  if (Z) CKA(cudaMemcpy(Z, dZ.p, (size_t)m * m * sizeof(double), cudaMemcpyDefault));
  return r;
}

namespace lrp {
namespace {

// One Arnoldi run (state between the host-driven steps).
struct ArnoldiRun {
  lrp_problem* P = nullptr;
  int nx = 0, mmax = 0, k = 0;
  unsigned flags = 0;
  double eig_tol = 1e-6, eig_threshold = 0.0;
  Buf<double> V, W, H, Hm, Zm, wbuf, X, Y, res, Vr;
  Buf<int> pos, hstat;
  std::vector<double> hH;  // host copy of H, (mmax+1) x mmax, ld mmax+1
  int m = 0;               // steps taken
  int rank_y_max = 0, rank_q_max = 0;
  bool apply_noconv = false;
  double ms_apply = 0.0;
  // Ritz data of the last check
  std::vector<double> wr, wi, rres;
  std::vector<int> order;  // diagonal positions of T by decreasing real part
  std::vector<int> sel;    // positions of the wanted real Ritz values
  double theta1 = 0.0;
};

lrp_status arnoldi_apply(ArnoldiRun& A, const double* x, double* y, lrp_apply_stats* st) {
  const bool misfit = (A.flags & LRP_MISFIT_ONLY) != 0;
  if (A.flags & LRP_ALS_SOLVES) return als_hessian_impl(A.P, 1, x, A.nx, y, A.nx, misfit, st);
  if (A.flags & LRP_LOWRANK_SOURCE) return lowrank_hessian_impl(A.P, 1, x, A.nx, y, A.nx, misfit, st);
  unsigned stages = ST_LOAD_X | ST_FORWARD | ST_ADJOINT | ST_STORE_Y;
  if (!misfit) stages |= ST_PRIOR_IN | ST_PRIOR_OUT;
  return run_sweep(A.P, stages, 1, x, A.nx, y, A.nx, nullptr, 0, nullptr, 0, st, misfit);
}

// Ritz values of H_m, the wanted real ones and their residual estimates.
// Returns true (in *ok) when the stopping rule holds.
lrp_status arnoldi_check(ArnoldiRun& A, bool* ok) {
  cudaStream_t s = A.P->stream;
  const int m = A.m, ldh = A.mmax + 1;
  CKA(cudaMemcpy2DAsync(A.Hm.p, (size_t)m * sizeof(double), A.H.p, (size_t)ldh * sizeof(double),
                        (size_t)m * sizeof(double), m, cudaMemcpyDeviceToDevice, s));
  A.wr.assign(m, 0.0);
  A.wi.assign(m, 0.0);
  lrp_status r = hessenberg_schur(s, m, A.Hm.p, A.Zm.p, A.wbuf.p, A.hstat.p, A.wr.data(), A.wi.data());
  if (r != LRP_OK) return r;
  A.order.resize(m);
  std::iota(A.order.begin(), A.order.end(), 0);
  std::stable_sort(A.order.begin(), A.order.end(), [&](int a, int b) {
    if (A.wr[a] != A.wr[b]) return A.wr[a] > A.wr[b];
    return A.wi[a] > A.wi[b];
  });
  A.theta1 = std::fabs(A.wr[A.order[0]]);
  for (int q = 0; q < m; ++q) A.theta1 = std::max(A.theta1, std::hypot(A.wr[q], A.wi[q]));
  // wanted: real parts >= threshold (threshold mode) or the k leading
  A.sel.clear();
  bool complex_wanted = false, below = false;
  for (int q = 0; q < m; ++q) {
    const int i = A.order[q];
    const bool wanted = A.eig_threshold > 0.0 ? A.wr[i] >= A.eig_threshold : q < A.k;
    if (!wanted) {
      below = true;
      continue;
    }
    if (A.wi[i] != 0.0)
      complex_wanted = true;
    else
      A.sel.push_back(i);
  }
  const int ns = (int)A.sel.size();
  A.rres.assign(ns, 0.0);
  if (ns > 0) {
    CKA(cudaMemcpyAsync(A.pos.p, A.sel.data(), ns * sizeof(int), cudaMemcpyHostToDevice, s));
    note_launch();
    k_schur_evec<<<(ns + 3) / 4, 128, 0, s>>>(m, A.Hm.p, A.pos.p, ns, A.X.p);
    CKA(cudaGetLastError());
    CKA(gemm_nn(s, m, m, ns, 1.0, A.Zm.p, m, A.X.p, m, 0.0, A.Y.p, m));
    const double beta = std::fabs(A.hH[(size_t)(m - 1) * ldh + m]);
    note_launch();
    k_ritz_estimate<<<ns, 128, 0, s>>>(m, ns, A.Y.p, beta, A.res.p);
    CKA(cudaGetLastError());
    CKA(cudaMemcpyAsync(A.rres.data(), A.res.p, ns * sizeof(double), cudaMemcpyDeviceToHost, s));
    CKA(cudaStreamSynchronize(s));
  }
  bool conv = !complex_wanted;
  for (int q = 0; q < ns; ++q) conv = conv && A.rres[q] <= A.eig_tol * A.theta1;
  if (A.eig_threshold > 0.0)
    conv = conv && below;
  else
    conv = conv && ns >= std::min(A.k, m);
  *ok = conv;
  return LRP_OK;
}

}  // namespace
}  // namespace lrp

extern "C" lrp_status lrp_arnoldi(lrp_problem* P, int max_steps, int k, double eig_tol, double eig_threshold,
                                  unsigned flags, const double* start, double* theta_re, double* theta_im,
                                  double* H_out, int* ranks_y, int* ranks_q, lrp_posterior** out,
                                  lrp_arnoldi_stats* stats) {
  if (!P || max_steps < 1 || max_steps > std::min(P ? P->nx : 0, 2048) || k < 0 || eig_threshold < 0.0 ||
      (eig_threshold == 0.0 && k < 1) || (flags & LRP_KEEP_TRAJ_FACTORS)) {
    set_error("lrp_arnoldi: need 1 <= max_steps <= min(nx, 2048), eig_threshold >= 0, k >= 1 without a threshold, "
              "and no LRP_KEEP_TRAJ_FACTORS");
    return LRP_EINVAL;
  }
  if (out && (flags & LRP_MISFIT_ONLY)) {
    set_error("lrp_arnoldi: a posterior needs the prior-preconditioned operator (no LRP_MISFIT_ONLY)");
    return LRP_EINVAL;
  }
  if (start) {
    lrp_status sd = check_on_device(P->device, start, "lrp_arnoldi");
    if (sd != LRP_OK) return sd;
  }
  cudaSetDevice(P->device);
  auto t0 = std::chrono::steady_clock::now();
  ArnoldiRun A;
  A.P = P;
  A.nx = P->nx;
  A.mmax = max_steps;
  A.k = k;
  A.flags = flags;
  A.eig_tol = eig_tol > 0.0 ? eig_tol : 1e-6;
  A.eig_threshold = eig_threshold;
  const int nx = P->nx, mmax = max_steps, ldh = mmax + 1;
  cudaStream_t s = P->stream;
  CKA(A.V.alloc((size_t)nx * (mmax + 1)));
  CKA(A.W.alloc(nx));
  CKA(A.H.alloc((size_t)ldh * mmax));
  CKA(A.Hm.alloc((size_t)mmax * mmax));
  CKA(A.Zm.alloc((size_t)mmax * mmax));
  CKA(A.wbuf.alloc(2 * (size_t)mmax));
  CKA(A.X.alloc((size_t)mmax * mmax));
  CKA(A.Y.alloc((size_t)mmax * mmax));
  CKA(A.res.alloc(mmax));
  CKA(A.pos.alloc(mmax));
  CKA(A.hstat.alloc(1));
  A.hH.assign((size_t)ldh * mmax, 0.0);
  CKA(cudaMemsetAsync(A.H.p, 0, (size_t)ldh * mmax * sizeof(double), s));
  if (start) {
    CKA(cudaMemcpyAsync(A.V.p, start, (size_t)nx * sizeof(double),
                        is_device_ptr(start) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  } else {
    CKA(fill_random(s, nx, 1, A.V.p, nx, nullptr, 0xA5D1ull));
  }
  note_launch();
  k_normalize<<<1, kMgsThreads, 0, s>>>(nx, A.V.p);
  CKA(cudaGetLastError());
  bool converged = false, breakdown = false;
  for (int j = 0; j < mmax; ++j) {
    lrp_apply_stats ast;
    std::memset(&ast, 0, sizeof(ast));
    auto ta = std::chrono::steady_clock::now();
    lrp_status r = arnoldi_apply(A, A.V.p + (size_t)j * nx, A.W.p, &ast);
    A.ms_apply += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - ta).count();
    if (r == LRP_ENOCONV)
      A.apply_noconv = true;
    else if (r != LRP_OK)
      return r;
    if (ranks_y) ranks_y[j] = ast.time_rank_max;
    if (ranks_q) ranks_q[j] = ast.adj_rank_max;
    A.rank_y_max = std::max(A.rank_y_max, ast.time_rank_max);
    A.rank_q_max = std::max(A.rank_q_max, ast.adj_rank_max);
    note_launch();
    k_arnoldi_mgs<<<1, kMgsThreads, 0, s>>>(nx, j, A.V.p, A.W.p, A.H.p + (size_t)j * ldh);
    CKA(cudaGetLastError());
    CKA(cudaMemcpyAsync(A.hH.data() + (size_t)j * ldh, A.H.p + (size_t)j * ldh, (size_t)(j + 2) * sizeof(double),
                        cudaMemcpyDeviceToHost, s));
    CKA(cudaStreamSynchronize(s));
    A.m = j + 1;
    // an invariant subspace: the Ritz values are exact
    double hnorm = 0.0;
    for (int i = 0; i <= j; ++i) hnorm = std::max(hnorm, std::fabs(A.hH[(size_t)j * ldh + i]));
    breakdown = A.hH[(size_t)j * ldh + j + 1] <= 1e-14 * hnorm;
    const int mm = A.m;
    const bool due = mm <= 32 || mm % std::max(1, mm / 16) == 0;
    // with a threshold: not before 8 steps (a short Krylov space from a
    // random start has not found the dominant eigenvalues yet, and every
    // Ritz value may still lie below the threshold)
    const bool enough = A.eig_threshold > 0.0 ? mm >= 8 : mm >= A.k;
    if ((due && enough) || breakdown || j + 1 == mmax) {
      bool ok = false;
      lrp_status c = arnoldi_check(A, &ok);
      if (c != LRP_OK) return c;
      if (ok || breakdown) {
        converged = ok || breakdown;
        break;
      }
    }
  }
  const int m = A.m;
  // outputs: Ritz values by decreasing real part, H
  if (theta_re || theta_im) {
    for (int q = 0; q < m; ++q) {
      if (theta_re) theta_re[q] = A.wr[A.order[q]];
      if (theta_im) theta_im[q] = A.wi[A.order[q]];
    }
  }
  if (H_out) {
    std::vector<double> hc((size_t)ldh * mmax, 0.0);
    std::copy(A.hH.begin(), A.hH.end(), hc.begin());
    CKA(cudaMemcpy(H_out, hc.data(), hc.size() * sizeof(double), cudaMemcpyDefault));
  }
  double asym = 0.0, hf = 0.0, max_imag = 0.0, max_res = 0.0;
  int n_complex = 0;
  for (int c = 0; c < m; ++c)
    for (int r = 0; r < m; ++r) {
      const double a = A.hH[(size_t)c * ldh + r], b = A.hH[(size_t)r * ldh + c];
      asym += (a - b) * (a - b);
      hf += a * a;
    }
  for (int q = 0; q < m; ++q) {
    if (A.wi[q] != 0.0) ++n_complex;
    max_imag = std::max(max_imag, std::fabs(A.wi[q]));
  }
  for (double x : A.rres) max_res = std::max(max_res, x);
  const double th1 = A.theta1 > 0.0 ? A.theta1 : 1.0;
  // posterior from the wanted real pairs (theta > 0), Ritz vectors
  // orthonormalised in order of decreasing theta
  lrp_status result = LRP_OK;
  if (out) {
    std::vector<int> keep;
    for (int q = 0; q < (int)A.sel.size(); ++q)
      if (A.wr[A.sel[q]] > 0.0) keep.push_back(q);
    const int kout = (int)keep.size();
    lrp_posterior* post = new lrp_posterior();
    post->prob = P;
    post->k = kout;
    post->nx = nx;
    post->sigma0 = P->desc.sigma;
    post->diag = nullptr;
    post->diag_cap = 0;
    post->V = post->G = post->lambda = nullptr;
    for (int q : keep) post->lambda_host.push_back(A.wr[A.sel[q]]);
    Buf<double> Vk, Gk, lam, part, C1, R;
    Buf<double> gs;
    auto fail = [&](lrp_status st) {
      lrp_posterior_destroy(post);
      return st;
    };
    if (Vk.alloc((size_t)nx * std::max(kout, 1)) != cudaSuccess || Gk.alloc((size_t)nx * std::max(kout, 1)) != cudaSuccess ||
        lam.alloc(std::max(kout, 1)) != cudaSuccess)
      return fail(cuda_status(cudaErrorMemoryAllocation, "lrp_arnoldi: posterior"));
    if (kout > 0) {
      // Y's columns follow A.sel (already sorted by decreasing real part)
      cudaError_t e = cudaSuccess;
      for (int q = 0; q < kout && e == cudaSuccess; ++q)
        e = cudaMemcpyAsync(A.X.p + (size_t)q * m, A.Y.p + (size_t)keep[q] * m, (size_t)m * sizeof(double),
                            cudaMemcpyDeviceToDevice, s);
      if (e == cudaSuccess) e = gemm_nn(s, nx, m, kout, 1.0, A.V.p, nx, A.X.p, m, 0.0, Vk.p, nx);
      const size_t part_cap = (size_t)std::max(kout, 16) * 16 * 128;
      if (e == cudaSuccess) e = part.alloc(part_cap);
      if (e == cudaSuccess) e = C1.alloc((size_t)kout * 64);
      if (e == cudaSuccess) e = R.alloc(64 * 64);
      if (e == cudaSuccess) e = gs.alloc(block_gs_scratch_doubles());
      // block CGS2 in blocks of up to 64 columns
      for (int c0 = 0; c0 < kout && e == cudaSuccess; c0 += 64) {
        const int nb = std::min(64, kout - c0);
        double* B = Vk.p + (size_t)c0 * nx;
        for (int pass = 0; pass < 2 && c0 > 0 && e == cudaSuccess; ++pass) {
          e = gemm_tn(s, nx, c0, nb, Vk.p, nx, B, nx, C1.p, c0, 1.0, 0.0, part.p, part_cap);
          if (e == cudaSuccess) e = gemm_nn(s, nx, c0, nb, -1.0, Vk.p, nx, C1.p, c0, 1.0, B, nx);
        }
        if (e == cudaSuccess) e = block_gs(s, 1, nx, nb, B, 0, nx, R.p, 0, 0.0, nullptr, nullptr, gs.p);
      }
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(lam.p, post->lambda_host.data(), kout * sizeof(double), cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return fail(cuda_status(e, "lrp_arnoldi: posterior"));
      lrp_apply_stats ast;
      lrp_status st = run_sweep(P, ST_LOAD_X | ST_PRIOR_IN | ST_STORE_Y, kout, Vk.p, nx, Gk.p, nx, nullptr, 0,
                                nullptr, 0, &ast, false);
      if (st != LRP_OK && st != LRP_ENOCONV) return fail(st);
      if (st == LRP_ENOCONV) A.apply_noconv = true;
    }
    post->V = Vk.release();
    post->G = Gk.release();
    post->lambda = lam.release();
    *out = post;
  }
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->n_steps = m;
    stats->k_converged = converged ? (int)A.sel.size() : 0;
    stats->n_complex = n_complex;
    stats->max_imag = max_imag / th1;
    stats->hess_asym = hf > 0.0 ? std::sqrt(asym / hf) : 0.0;
    stats->max_ritz_resid = max_res / th1;
    stats->time_rank_max = A.rank_y_max;
    stats->adj_rank_max = A.rank_q_max;
    stats->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    stats->ms_apply = A.ms_apply;
  }
  if (!converged) {
    set_error("Arnoldi reached max_steps before the wanted Ritz values converged");
    result = LRP_ENOCONV;
  } else if (A.apply_noconv) {
    set_error("a solve of a Hessian apply missed its tolerance within pcg_maxit");
    result = LRP_ENOCONV;
  }
  return result;
}

// ---------------------------------------------------------------------------
// Low-rank space-time vectors (Sec. 4): X = A B^T with A: nx x r, B: nt x r.

namespace lrp {
namespace {

// out = sum_ij Ga[i, j] Gb[i, j] (Ga, Gb: n entries); one CTA.
__global__ void k_frob_dot(int n, const double* Ga, const double* Gb, double* out) {
  __shared__ double red[32];
  double d = 0.0;
  for (int e = threadIdx.x; e < n; e += blockDim.x) d += Ga[e] * Gb[e];
  const double s = block_sum(d, red);
  if (threadIdx.x == 0) *out = s;
}

// M = Ra Rb^T (R x R, all column-major, ld R)
__global__ void k_small_abt(int R, const double* Ra, const double* Rb, double* M) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= R * R) return;
  const int i = e % R, j = e / R;
  double acc = 0.0;
  for (int k = 0; k < R; ++k) acc += Ra[(size_t)k * R + i] * Rb[(size_t)k * R + j];
  M[e] = acc;
}

// Scratch of the low-rank vector operations (sized for R <= kStMaxCols).
constexpr int kStMaxCols = 112;
struct StWS {
  Buf<double> part, C, Csum, Rblk, Ra, Rb, M, th, Zaug, gs, scal, cat_a, cat_b;
  Buf<int> iarr, stat;
  size_t part_cap = 0;
  int nx = 0, nt = 0;
  cudaError_t init(int nx_, int nt_) {
    nx = nx_;
    nt = nt_;
    const int R = kStMaxCols;
    part_cap = (size_t)std::max(R, 16) * 16 * 128;
    cudaError_t e = part.alloc(part_cap);
    if (e == cudaSuccess) e = C.alloc((size_t)R * 64);
    if (e == cudaSuccess) e = Csum.alloc((size_t)R * 64);
    if (e == cudaSuccess) e = Rblk.alloc(64 * 64);
    if (e == cudaSuccess) e = Ra.alloc((size_t)R * R);
    if (e == cudaSuccess) e = Rb.alloc((size_t)R * R);
    if (e == cudaSuccess) e = M.alloc((size_t)R * R);
    if (e == cudaSuccess) e = th.alloc(2 * (size_t)R);
    if (e == cudaSuccess) e = Zaug.alloc(4 * (size_t)R * R);
    if (e == cudaSuccess) e = gs.alloc(block_gs_scratch_doubles());
    if (e == cudaSuccess) e = scal.alloc(4);
    if (e == cudaSuccess) e = cat_a.alloc((size_t)nx * R);
    if (e == cudaSuccess) e = cat_b.alloc((size_t)nt * R);
    if (e == cudaSuccess) e = iarr.alloc(2);
    if (e == cudaSuccess) e = stat.alloc(1);
    return e;
  }
};

// Thin QR of the rows x R matrix A (in place: A <- Q) with R <= kStMaxCols:
// blocks of up to 64 columns, each projected on the previous blocks twice
// (block CGS2; coefficients into the upper blocks of Rout) and then
// factorised by the rank-revealing block Gram-Schmidt. Rout: R x R, ld R.
cudaError_t qr_tall(cudaStream_t s, StWS& w, int rows, int R, double* A, double* Rout) {
  cudaError_t e = cudaMemsetAsync(Rout, 0, (size_t)R * R * sizeof(double), s);
  for (int c0 = 0; c0 < R && e == cudaSuccess; c0 += 64) {
    const int nb = std::min(64, R - c0);
    double* B = A + (size_t)c0 * rows;
    if (c0 > 0) {
      e = cudaMemsetAsync(w.Csum.p, 0, (size_t)c0 * nb * sizeof(double), s);
      for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {
        e = gemm_tn(s, rows, c0, nb, A, rows, B, rows, w.C.p, c0, 1.0, 0.0, w.part.p, w.part_cap);
        if (e == cudaSuccess) e = gemm_nn(s, rows, c0, nb, -1.0, A, rows, w.C.p, c0, 1.0, B, rows);
        if (e == cudaSuccess) e = axpby(s, (size_t)c0 * nb, 1.0, w.C.p, 1.0, w.Csum.p);
      }
      if (e == cudaSuccess) e = set_rect(s, Rout, R, 0, c0, c0, nb, w.Csum.p, c0, false);
    }
    if (e == cudaSuccess) e = block_gs(s, 1, rows, nb, B, 0, rows, w.Rblk.p, 0, 1e-14, nullptr, nullptr, w.gs.p);
    if (e == cudaSuccess) e = set_rect(s, Rout, R, c0, c0, nb, nb, w.Rblk.p, nb, false);
  }
  return e;
}

// <X, Y> = sum (A_X^T A_Y) .* (B_X^T B_Y); result on the host.
lrp_status lr_dot(cudaStream_t s, StWS& w, int rx, const double* Ax, const double* Bx, int ry, const double* Ay,
                  const double* By, double* out) {
  if (rx == 0 || ry == 0) {
    *out = 0.0;
    return LRP_OK;
  }
  CKA(gemm_tn(s, w.nx, rx, ry, Ax, w.nx, Ay, w.nx, w.Ra.p, rx, 1.0, 0.0, w.part.p, w.part_cap));
  CKA(gemm_tn(s, w.nt, rx, ry, Bx, w.nt, By, w.nt, w.Rb.p, rx, 1.0, 0.0, w.part.p, w.part_cap));
  note_launch();
  k_frob_dot<<<1, 256, 0, s>>>(rx * ry, w.Ra.p, w.Rb.p, w.scal.p);
  CKA(cudaGetLastError());
  CKA(cudaMemcpyAsync(out, w.scal.p, sizeof(double), cudaMemcpyDeviceToHost, s));
  CKA(cudaStreamSynchronize(s));
  return LRP_OK;
}

// Rounds A B^T (R columns in w.cat_a / w.cat_b, destroyed) to the smallest
// rank whose discarded Frobenius tail is at most tol ||A B^T||_F, capped at
// rmax: thin QR of both factors, SVD of the R x R core Ra Rb^T (one-sided
// Jacobi), A' = Q_A U_r S_r, B' = Q_B Z_r into Aout, Bout. *norm = ||A' B'^T||_F.
lrp_status lr_round(cudaStream_t s, StWS& w, int R, double tol, int rmax, double* Aout, double* Bout, int* r_out,
                    double* norm, double* err) {
  *r_out = 0;
  *norm = 0.0;
  *err = 0.0;
  if (R == 0) return LRP_OK;
  if (R > kStMaxCols) {
    set_error("low-rank vector rounding: more than 112 columns");
    return LRP_EINVAL;
  }
  CKA(qr_tall(s, w, w.nx, R, w.cat_a.p, w.Ra.p));
  CKA(qr_tall(s, w, w.nt, R, w.cat_b.p, w.Rb.p));
  note_launch();
  k_small_abt<<<(R * R + 255) / 256, 256, 0, s>>>(R, w.Ra.p, w.Rb.p, w.M.p);
  CKA(cudaGetLastError());
  std::vector<double> th;
  {
    lrp_status r = core_svd(s, R, w.M.p, w.th.p, w.Zaug.p, w.iarr.p, w.stat.p, &th);
    if (r != LRP_OK) return r;
  }
  double fro2 = 0.0;
  for (double x : th) fro2 += x * x;
  std::vector<double> tail(R + 1, 0.0);
  for (int i = R - 1; i >= 0; --i) tail[i] = tail[i + 1] + th[i] * th[i];
  int rn = 0;
  while (rn < R && tail[rn] > tol * tol * fro2) ++rn;
  if (rn == 0 && R > 0 && th[0] > 0) rn = 1;
  rn = std::min(rn, rmax);
  *err = fro2 > 0 ? std::sqrt(tail[rn] / fro2) : 0.0;
  *norm = std::sqrt(std::max(fro2 - tail[rn], 0.0));
  *r_out = rn;
  if (rn == 0) return LRP_OK;
  const double* U = w.Zaug.p;
  const double* Zv = U + (size_t)R * R;
  CKA(gemm_nn(s, w.nx, R, rn, 1.0, w.cat_a.p, w.nx, U, R, 0.0, Aout, w.nx));
  CKA(scale_cols(s, w.nx, rn, w.th.p, Aout, w.nx));
  CKA(gemm_nn(s, w.nt, R, rn, 1.0, w.cat_b.p, w.nt, Zv, R, 0.0, Bout, w.nt));
  return LRP_OK;
}

}  // namespace
}  // namespace lrp

extern "C" lrp_status lrp_st_hessian_apply(lrp_problem* P, int r, const double* W, int ldw, const double* V, int ldv,
                                           double* Wout, double* Vout, int* r_out, lrp_apply_stats* st) {
  if (!P || r < 0 || r > 4096 || (r > 0 && (!W || !V || ldw < P->nx || ldv < P->nt)) || !Wout || !Vout || !r_out) {
    set_error("lrp_st_hessian_apply: invalid argument");
    return LRP_EINVAL;
  }
  for (const void* a : {(const void*)W, (const void*)V, (const void*)Wout, (const void*)Vout}) {
    if (!a) continue;
    lrp_status sd = check_on_device(P->device, a, "lrp_st_hessian_apply");
    if (sd != LRP_OK) return sd;
  }
  cudaSetDevice(P->device);
  const int nx = P->nx, nt = P->nt, rmax = P->desc.time_rank_max;
  cudaStream_t s = P->stream;
  Buf<double> dW, dV, oW, oV;
  CKA(dW.alloc((size_t)nx * std::max(r, 1)));
  CKA(dV.alloc((size_t)nt * std::max(r, 1)));
  CKA(oW.alloc((size_t)nx * rmax));
  CKA(oV.alloc((size_t)nt * rmax));
  if (r > 0) {
    CKA(cudaMemcpy2DAsync(dW.p, (size_t)nx * sizeof(double), W, (size_t)ldw * sizeof(double), (size_t)nx * sizeof(double),
                          r, cudaMemcpyDefault, s));
    CKA(cudaMemcpy2DAsync(dV.p, (size_t)nt * sizeof(double), V, (size_t)ldv * sizeof(double), (size_t)nt * sizeof(double),
                          r, cudaMemcpyDefault, s));
  }
  int ro = 0;
  lrp_status res = st_hessian_impl(P, r, dW.p, nx, dV.p, nt, oW.p, oV.p, &ro, st);
  if (res != LRP_OK && res != LRP_ENOCONV) return res;
  if (ro > 0) {
    CKA(cudaMemcpyAsync(Wout, oW.p, (size_t)nx * ro * sizeof(double), cudaMemcpyDefault, s));
    CKA(cudaMemcpyAsync(Vout, oV.p, (size_t)nt * ro * sizeof(double), cudaMemcpyDefault, s));
  }
  CKA(cudaStreamSynchronize(s));
  *r_out = ro;
  return res;
}

extern "C" lrp_status lrp_st_arnoldi(lrp_problem* P, int max_steps, int k, double eig_tol, double eig_threshold, int r0,
                                     const double* W0, const double* V0, double* theta_re, double* theta_im,
                                     double* H_out, int* ranks, lrp_arnoldi_stats* stats) {
  if (!P || max_steps < 1 || max_steps > 2048 || (long long)max_steps > (long long)P->nx * P->nt || k < 0 ||
      eig_threshold < 0.0 || (eig_threshold == 0.0 && k < 1) || r0 < 0 || r0 > kStMaxCols ||
      (r0 > 0 && (!W0 || !V0)) || P->desc.time_rank_max > kStMaxCols / 2) {
    set_error("lrp_st_arnoldi: need 1 <= max_steps <= min(nx nt, 2048), k >= 1 without a threshold, "
              "0 <= r0 <= 112 with start factors, time_rank_max <= 56");
    return LRP_EINVAL;
  }
  for (const void* a : {(const void*)W0, (const void*)V0}) {
    if (!a) continue;
    lrp_status sd = check_on_device(P->device, a, "lrp_st_arnoldi");
    if (sd != LRP_OK) return sd;
  }
  cudaSetDevice(P->device);
  auto t0 = std::chrono::steady_clock::now();
  const int nx = P->nx, nt = P->nt, rmax = P->desc.time_rank_max, mmax = max_steps, ldh = mmax + 1;
  const double tol = P->desc.time_trunc_tol;
  cudaStream_t s = P->stream;
  ArnoldiRun A;
  A.P = P;
  A.nx = nx;
  A.mmax = mmax;
  A.k = k;
  A.eig_tol = eig_tol > 0.0 ? eig_tol : 1e-6;
  A.eig_threshold = eig_threshold;
  CKA(A.H.alloc((size_t)ldh * mmax));
  CKA(A.Hm.alloc((size_t)mmax * mmax));
  CKA(A.Zm.alloc((size_t)mmax * mmax));
  CKA(A.wbuf.alloc(2 * (size_t)mmax));
  CKA(A.X.alloc((size_t)mmax * mmax));
  CKA(A.Y.alloc((size_t)mmax * mmax));
  CKA(A.res.alloc(mmax));
  CKA(A.pos.alloc(mmax));
  CKA(A.hstat.alloc(1));
  A.hH.assign((size_t)ldh * mmax, 0.0);
  CKA(cudaMemsetAsync(A.H.p, 0, (size_t)ldh * mmax * sizeof(double), s));
  StWS w;
  CKA(w.init(nx, nt));
  // the basis: factors of v_1 .. v_{m+1}
  Buf<double> BA, BB, Aw, Bw;
  CKA(BA.alloc((size_t)(mmax + 1) * nx * rmax));
  CKA(BB.alloc((size_t)(mmax + 1) * nt * rmax));
  CKA(Aw.alloc((size_t)nx * rmax));
  CKA(Bw.alloc((size_t)nt * rmax));
  std::vector<int> rv(mmax + 1, 0);
  auto fa = [&](int j) { return BA.p + (size_t)j * nx * rmax; };
  auto fb = [&](int j) { return BB.p + (size_t)j * nt * rmax; };
  // start: the given factors (or one pseudo-random rank-1 pair), rounded and normalised
  int rs = r0;
  if (r0 > 0) {
    CKA(cudaMemcpyAsync(w.cat_a.p, W0, (size_t)nx * r0 * sizeof(double), cudaMemcpyDefault, s));
    CKA(cudaMemcpyAsync(w.cat_b.p, V0, (size_t)nt * r0 * sizeof(double), cudaMemcpyDefault, s));
  } else {
    rs = 1;
    CKA(fill_random(s, nx, 1, w.cat_a.p, nx, nullptr, 0x57A7ull));
    CKA(fill_random(s, nt, 1, w.cat_b.p, nt, nullptr, 0x57A8ull));
  }
  double nrm = 0.0, err = 0.0;
  {
    lrp_status r = lr_round(s, w, rs, 0.0, rmax, fa(0), fb(0), &rv[0], &nrm, &err);
    if (r != LRP_OK) return r;
  }
  if (nrm <= 0.0) {
    set_error("lrp_st_arnoldi: zero start vector");
    return LRP_EINVAL;
  }
  CKA(axpby(s, (size_t)nx * rv[0], 0.0, fa(0), 1.0 / nrm, fa(0)));
  bool converged = false, breakdown = false;
  int rank_v_max = rv[0], rank_q_max = 0;
  double ms_apply = 0.0;
  for (int j = 0; j < mmax; ++j) {
    lrp_apply_stats ast;
    std::memset(&ast, 0, sizeof(ast));
    int rw = 0;
    auto ta = std::chrono::steady_clock::now();
    lrp_status r = st_hessian_impl(P, rv[j], fa(j), nx, fb(j), nt, Aw.p, Bw.p, &rw, &ast);
    ms_apply += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - ta).count();
    if (r == LRP_ENOCONV)
      A.apply_noconv = true;
    else if (r != LRP_OK)
      return r;
    rank_q_max = std::max(rank_q_max, rw);
    // modified Gram-Schmidt on factored vectors, rounding after every update
    for (int i = 0; i <= j; ++i) {
      double h = 0.0;
      lrp_status d = lr_dot(s, w, rw, Aw.p, Bw.p, rv[i], fa(i), fb(i), &h);
      if (d != LRP_OK) return d;
      A.hH[(size_t)j * ldh + i] = h;
      const int ri = rv[i];
      if (rw > 0) {
        CKA(cudaMemcpyAsync(w.cat_a.p, Aw.p, (size_t)nx * rw * sizeof(double), cudaMemcpyDeviceToDevice, s));
        CKA(cudaMemcpyAsync(w.cat_b.p, Bw.p, (size_t)nt * rw * sizeof(double), cudaMemcpyDeviceToDevice, s));
      }
      if (ri > 0) {
        double* ca = w.cat_a.p + (size_t)nx * rw;
        CKA(cudaMemcpyAsync(ca, fa(i), (size_t)nx * ri * sizeof(double), cudaMemcpyDeviceToDevice, s));
        CKA(axpby(s, (size_t)nx * ri, 0.0, ca, -h, ca));
        CKA(cudaMemcpyAsync(w.cat_b.p + (size_t)nt * rw, fb(i), (size_t)nt * ri * sizeof(double),
                            cudaMemcpyDeviceToDevice, s));
      }
      lrp_status rr = lr_round(s, w, rw + ri, tol, rmax, Aw.p, Bw.p, &rw, &nrm, &err);
      if (rr != LRP_OK) return rr;
    }
    A.hH[(size_t)j * ldh + j + 1] = nrm;
    if (ranks) ranks[j] = rw;
    rank_v_max = std::max(rank_v_max, rw);
    rv[j + 1] = rw;
    if (rw > 0) {
      CKA(cudaMemcpyAsync(fa(j + 1), Aw.p, (size_t)nx * rw * sizeof(double), cudaMemcpyDeviceToDevice, s));
      CKA(axpby(s, (size_t)nx * rw, 0.0, fa(j + 1), nrm > 0.0 ? 1.0 / nrm : 0.0, fa(j + 1)));
      CKA(cudaMemcpyAsync(fb(j + 1), Bw.p, (size_t)nt * rw * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    CKA(cudaMemcpyAsync(A.H.p + (size_t)j * ldh, A.hH.data() + (size_t)j * ldh, (size_t)(j + 2) * sizeof(double),
                        cudaMemcpyHostToDevice, s));
    A.m = j + 1;
    double hnorm = 0.0;
    for (int i = 0; i <= j; ++i) hnorm = std::max(hnorm, std::fabs(A.hH[(size_t)j * ldh + i]));
    breakdown = nrm <= 1e-14 * hnorm;
    const int mm = A.m;
    const bool due = mm <= 32 || mm % std::max(1, mm / 16) == 0;
    const bool enough = A.eig_threshold > 0.0 ? mm >= 8 : mm >= A.k;
    if ((due && enough) || breakdown || j + 1 == mmax) {
      bool ok = false;
      lrp_status c = arnoldi_check(A, &ok);
      if (c != LRP_OK) return c;
      if (ok || breakdown) {
        converged = true;
        break;
      }
    }
  }
  const int m = A.m;
  for (int q = 0; q < m; ++q) {
    if (theta_re) theta_re[q] = A.wr[A.order[q]];
    if (theta_im) theta_im[q] = A.wi[A.order[q]];
  }
  if (H_out) CKA(cudaMemcpy(H_out, A.hH.data(), A.hH.size() * sizeof(double), cudaMemcpyDefault));
  if (stats) {
    double asym = 0.0, hf = 0.0, max_imag = 0.0, max_res = 0.0;
    int n_complex = 0;
    for (int c = 0; c < m; ++c)
      for (int r = 0; r < m; ++r) {
        const double a = A.hH[(size_t)c * ldh + r], b = A.hH[(size_t)r * ldh + c];
        asym += (a - b) * (a - b);
        hf += a * a;
      }
    for (int q = 0; q < m; ++q) {
      if (A.wi[q] != 0.0) ++n_complex;
      max_imag = std::max(max_imag, std::fabs(A.wi[q]));
    }
    for (double x : A.rres) max_res = std::max(max_res, x);
    const double th1 = A.theta1 > 0.0 ? A.theta1 : 1.0;
    std::memset(stats, 0, sizeof(*stats));
    stats->n_steps = m;
    stats->k_converged = converged ? (int)A.sel.size() : 0;
    stats->n_complex = n_complex;
    stats->max_imag = max_imag / th1;
    stats->hess_asym = hf > 0.0 ? std::sqrt(asym / hf) : 0.0;
    stats->max_ritz_resid = max_res / th1;
    stats->time_rank_max = rank_v_max;
    stats->adj_rank_max = rank_q_max;
    stats->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    stats->ms_apply = ms_apply;
  }
  if (!converged) {
    set_error("Arnoldi reached max_steps before the wanted Ritz values converged");
    return LRP_ENOCONV;
  }
  if (A.apply_noconv) {
    set_error("a solve of a Hessian apply missed its tolerance within pcg_maxit");
    return LRP_ENOCONV;
  }
  return LRP_OK;
}
