// Alternating low-rank solver of the space-time system (Sec. 6.1,
// Eq. (st_pde), (amen_1), (amen_2), (pre_1)) and the Hessian product whose
// forward and adjoint solves use it.
//
// The implicit-Euler sweep y_n = A^{-1}(y_{n-1} + f_n), n = 1..nt, y_0 = 0,
// A = I + tau L, is the space-time system A Y - Y S^T = F with
// Y = [y_1 .. y_nt], F = [f_1 .. f_nt] and (Y S^T)[:, n] = y_{n-1}
// (Eq. (st_pde) with M = I). With Y ~ W V^T (W: nx x r, V: nt x r, V
// orthonormal) one sweep takes
//  * the space step (Eq. (amen_1)): the Galerkin projection onto span(V) in
//    time, A W - W T = F V, T = V^T S^T V (an nx r system), solved by
//    right-preconditioned flexible GMRES with the block-diagonal
//    preconditioner of Eq. (pre_1): blocks A - T_jj I, each applied by one
//    multigrid-preconditioned solve of the sweep kernel (stage ST_SHIFTED,
//    one column per team, all r columns in one launch);
//  * the time step (Eq. (amen_2)): W orthonormalised to Q (Cholesky QR),
//    the Galerkin projection onto span(Q) in space,
//    Ahat z_n - z_{n-1} = Q^T f_n with Ahat = Q^T A Q (r x r), solved
//    directly (one CTA: Gauss-Jordan inverse, then the nt-step recurrence),
//    Y = Q Z^T, V = orth(Z), W = Q R_Z^T.
// Several independent solves (the columns of a Hessian product) run as one
// batch: their GMRES iterations are shared (one preconditioner launch for
// all their columns), each with its own Hessenberg matrix.
// The adjoint system A^T q_n = q_{n+1} + f_n (n = nt..1) is the same system
// with A^T in reversed time.
//
// AMEn (the paper's solver) also enriches the basis with residual
// directions; this is the fixed-rank alternating scheme (ALS) it builds on.
// Host code drives the iteration; every arithmetic step runs in kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "lrp_dense.h"
#include "lrp_internal.h"
#include "lrp_sweep_kernel.cuh"

namespace lrp {
namespace {

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
};

#define CKL(call)                                         \
  do {                                                    \
    cudaError_t _e = (call);                              \
    if (_e != cudaSuccess) return cuda_status(_e, #call); \
  } while (0)
#define CKS(call)                 \
  do {                            \
    lrp_status _s = (call);       \
    if (_s != LRP_OK) return _s;  \
  } while (0)

constexpr int kMaxRank = 64;     // rank limit: the Cholesky QR's and the GMRES update's small tiles
constexpr int kGmresMax = 40;    // Krylov vectors per GMRES cycle
constexpr int kGmresCycles = 6;  // restarts per space step
constexpr double kPrecondRtol = 1e-8;  // stop of a preconditioner solve before its iteration cap
constexpr int kPrecondIts = 2;         // default CG iterations per preconditioner solve

// ---------------------------------------------------------------------------
// kernels

// Y[:, j] = (A x_j) - sum_i x_i Tm[i, j] for the columns of X (nx x ncol,
// ld nx; ncol = nb r: nb solves of r columns each, solve c with its own
// r x r matrix Tm + c r r): the operator of the space step (Tm = T) or plain
// A X (Tm NULL). A = I + tau L of the problem on its finest level
// (transpose: A^T).
template <int DIM, bool KAPPA, bool CONV>
__global__ void k_kron_apply(const OpLevel l0, int r, int ncol, const double* X, const double* Tm, int transpose,
                             double* Y) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (p >= l0.N || y >= ncol) return;
  const size_t nx = (size_t)l0.N;
  int i0, i1, i2;
  decomp<DIM>(l0, p, i0, i1, i2);
  Ld<double> ld{X + (size_t)y * nx, 0, 0};
  double d;
  double v;
  if (CONV)
    v = op_conv_at<DIM>(l0, ld, p, i0, i1, i2, transpose != 0, d);
  else
    v = op_at<double, DIM, KAPPA>(l0, ld, p, i0, i1, i2, d);
  if (Tm) {
    const int c = y / r, j = y - c * r;
    const double* Xc = X + (size_t)c * r * nx;
    const double* Tc = Tm + (size_t)c * r * r;
    for (int i = 0; i < r; ++i) v -= Xc[(size_t)i * nx + p] * Tc[(size_t)j * r + i];
  }
  Y[(size_t)y * nx + p] = v;
}

// Per-node inverse diagonal of I + (c / s) L from that of I + c L:
// 1 / (1 + (1/dinv - 1) / s).
__global__ void k_shift_dinv(int N, const double* dinv, double inv_s, double* outd, float* outf) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  const double v = 1.0 / (1.0 + (1.0 / dinv[p] - 1.0) * inv_s);
  outd[p] = v;
  outf[p] = (float)v;
}

// GMRES: applies the j earlier Givens rotations to column j of the
// Hessenberg matrix H (ld ldh), forms rotation j that zeroes H[j+1, j],
// updates the rotated right-hand side g; res = |g[j+1]| (the residual norm).
// (one thread per solve c = blockIdx.x; its H, cs, sn, g at strides hs, kmax,
// kmax + 1; res[c])
__global__ void k_givens(int j, double* H, int ldh, size_t hs, double* cs, double* sn, double* g, int kmax,
                         double* res) {
  if (threadIdx.x != 0) return;
  const int col = blockIdx.x;
  H += (size_t)col * hs;
  cs += (size_t)col * kmax;
  sn += (size_t)col * kmax;
  g += (size_t)col * (kmax + 1);
  res += col;
  double* h = H + (size_t)j * ldh;
  for (int i = 0; i < j; ++i) {
    const double a = h[i], b = h[i + 1];
    h[i] = cs[i] * a + sn[i] * b;
    h[i + 1] = -sn[i] * a + cs[i] * b;
  }
  const double a = h[j], b = h[j + 1];
  const double rr = hypot(a, b);
  const double c = rr > 0.0 ? a / rr : 1.0;
  const double s = rr > 0.0 ? b / rr : 0.0;
  cs[j] = c;
  sn[j] = s;
  h[j] = rr;
  h[j + 1] = 0.0;
  g[j + 1] = -s * g[j];
  g[j] = c * g[j];
  *res = fabs(g[j + 1]);
}

// y = R^{-1} g with R the leading m x m upper triangle of H (ld ldh); a zero
// pivot (a vanished direction) leaves its component at zero.
// (one thread per solve c = blockIdx.x, strides as k_givens)
__global__ void k_backsolve(int m, const double* H, int ldh, size_t hs, const double* g, double* y, int kmax) {
  if (threadIdx.x != 0) return;
  const int c = blockIdx.x;
  H += (size_t)c * hs;
  g += (size_t)c * (kmax + 1);
  y += (size_t)c * kmax;
  for (int i = m - 1; i >= 0; --i) {
    double acc = g[i];
    for (int k = i + 1; k < m; ++k) acc -= H[(size_t)k * ldh + i] * y[k];
    const double d = H[(size_t)i * ldh + i];
    y[i] = d != 0.0 ? acc / d : 0.0;
  }
}

// H[j+1, j] = sqrt(*nrm2) and g[0] = that norm for j < 0 (the start of a
// cycle); inv = 1 / the norm (0 for a vanished vector).
// (solve c = blockIdx.x: nrm2[c], dst + c dst_stride, inv[c])
__global__ void k_norm_entry(const double* nrm2, double* dst, size_t dst_stride, double* inv) {
  if (threadIdx.x != 0) return;
  const int c = blockIdx.x;
  const double v = sqrt(fmax(nrm2[c], 0.0));
  dst[(size_t)c * dst_stride] = v;
  inv[c] = v > 0.0 ? 1.0 / v : 0.0;
}

// y_c = scale[c] x_c for the solves c = blockIdx.y (n entries each, offset c n)
__global__ void k_scale_by(size_t n, const double* scale, const double* x, double* y) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t c = blockIdx.y;
  if (i < n) y[c * n + i] = scale[c] * x[c * n + i];
}

// H_c[0:m, j] += hv_c[0:m] for the solves c = blockIdx.x
__global__ void k_hadd(int m, const double* hv, size_t hvs, double* H, size_t hs) {
  const int c = blockIdx.x;
  for (int i = threadIdx.x; i < m; i += blockDim.x) H[(size_t)c * hs + i] += hv[(size_t)c * hvs + i];
}

// out[i] = v[i] * s[i / nx] (column scaling by a device vector), in place allowed
__global__ void k_col_scale(size_t nx, int r, const double* s, double* v) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nx * (size_t)r) v[i] *= s[i / nx];
}

// T = V[0:nt-1]^T V[1:nt] (r x r): T[i, j] = sum_{n >= 1} V[n-1, i] V[n, j];
// also the diagonal shifts inv_s[j] = 1 / (1 - T[j, j]) and status bit 1 if
// some 1 - T[j, j] <= 0 (cannot happen for orthonormal columns: |T_jj| < 1).
__global__ void k_shift_gram(int nt, int r, const double* V, double* T, double* inv_s, int* status) {
  __shared__ double red[32];
  const int e = blockIdx.x;
  {
    const size_t c = blockIdx.y;  // solve c: its V, T and shifts
    V += c * nt * r;
    T += c * r * r;
    inv_s += c * r;
  }
  const int i = e % r, j = e / r;
  double acc = 0.0;
  for (int n = 1 + threadIdx.x; n < nt; n += blockDim.x) acc += V[(size_t)i * nt + n - 1] * V[(size_t)j * nt + n];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    T[(size_t)j * r + i] = s;
    if (i == j) {
      const double sh = 1.0 - s;
      inv_s[j] = sh > 0.0 ? 1.0 / sh : 0.0;
      if (!(sh > 0.0)) atomicOr(status, 1);
    }
  }
}

// The time step: Z (nt x r, ld nt) with Ahat z_n - z_{n-1} = Gt[n, :]^T
// (Gt: nt x r, ld nt), z_{-1} = 0. One CTA: the inverse of Ahat (r x r) by
// Gauss-Jordan elimination with partial pivoting in shared memory (a column
// without a nonzero pivot candidate belongs to a vanished basis vector: its
// row becomes the identity row, so that component stays zero), then the
// recurrence z_n = Ahat^{-1} (z_{n-1} + g_n), one warp per row and step.
// (solve c = blockIdx.x: its Ahat, Gt, Z at strides r r, nt r, nt r)
__global__ void __launch_bounds__(1024) k_als_time(int r, int nt, const double* Ahat, const double* Gt, double* Z) {
  extern __shared__ double sm[];
  Ahat += (size_t)blockIdx.x * r * r;
  Gt += (size_t)blockIdx.x * nt * r;
  Z += (size_t)blockIdx.x * nt * r;
  double* M = sm;                       // r x 2r, row-major: [Ahat | I] -> [I | Ahat^{-1}]
  double* u = M + (size_t)r * 2 * r;    // r: z_{n-1} + g_n
  __shared__ int s_piv;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int w2 = 2 * r;
  for (int e = tid; e < r * w2; e += nthr) {
    const int i = e / w2, c = e % w2;
    M[e] = c < r ? Ahat[(size_t)c * r + i] : (c - r == i ? 1.0 : 0.0);
  }
  __syncthreads();
  for (int k = 0; k < r; ++k) {
    if (tid < 32) {
      // pivot: largest |M[i, k]|, i >= k (ties -> smallest i)
      double best = -1.0;
      int bi = k;
      for (int i = k + tid; i < r; i += 32) {
        const double a = fabs(M[(size_t)i * w2 + k]);
        if (a > best) {
          best = a;
          bi = i;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (tid == 0) s_piv = best > 0.0 ? bi : -1;
    }
    __syncthreads();
    const int piv = s_piv;
    if (piv < 0) {
      // vanished direction: identity row and column
      for (int c = tid; c < w2; c += nthr) M[(size_t)k * w2 + c] = (c == k || c == r + k) ? 1.0 : 0.0;
      __syncthreads();
      continue;
    }
    if (piv != k) {
      for (int c = tid; c < w2; c += nthr) {
        const double a = M[(size_t)k * w2 + c];
        M[(size_t)k * w2 + c] = M[(size_t)piv * w2 + c];
        M[(size_t)piv * w2 + c] = a;
      }
    }
    __syncthreads();
    const double inv = 1.0 / M[(size_t)k * w2 + k];
    __syncthreads();
    for (int c = tid; c < w2; c += nthr) M[(size_t)k * w2 + c] *= inv;
    __syncthreads();
    for (int e = tid; e < r * w2; e += nthr) {
      const int i = e / w2, c = e % w2;
      if (i == k) continue;
      const double f = M[(size_t)i * w2 + k];
      if (c != k) M[e] -= f * M[(size_t)k * w2 + c];
    }
    __syncthreads();
    for (int i = tid; i < r; i += nthr)
      if (i != k) M[(size_t)i * w2 + k] = 0.0;
    __syncthreads();
  }
  // recurrence
  const int lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
  for (int i = tid; i < r; i += nthr) u[i] = 0.0;
  __syncthreads();
  double* zrow = u + r;  // r: z_n
  for (int n = 0; n < nt; ++n) {
    for (int i = tid; i < r; i += nthr) u[i] += Gt[(size_t)i * nt + n];
    __syncthreads();
    for (int i = warp; i < r; i += nwarps) {
      double acc = 0.0;
      for (int k = lane; k < r; k += 32) acc += M[(size_t)i * w2 + r + k] * u[k];
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) zrow[i] = acc;
    }
    __syncthreads();
    for (int i = tid; i < r; i += nthr) {
      Z[(size_t)i * nt + n] = zrow[i];
      u[i] = zrow[i];
    }
    __syncthreads();
  }
}

// out (nt x c, ld nt) = rows of V (nt x c, ld ldv) in reversed order
// (row m <- row nt-1-m), optionally keeping only the rows of observed steps:
// with mask_every > 0 the source row n-1 (step n) is kept iff n is a
// multiple of mask_every and n / mask_every <= mask_steps.
__global__ void k_rows_reverse(int nt, int c, const double* V, int ldv, double* out, int mask_every, int mask_steps) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (m >= nt || j >= c) return;
  const int src = nt - 1 - m;
  double v = V[(size_t)j * ldv + src];
  if (mask_every > 0) {
    const int n = src + 1;
    if ((n % mask_every) != 0 || n / mask_every > mask_steps) v = 0.0;
  }
  out[(size_t)j * nt + m] = v;
}

// D (n_obs x r, ld n_obs) = B W (W: nx x r, ld nx): the sensors' interpolants
__global__ void k_observe_cols(int n_obs, int r, const int* obs_node, const double* obs_w, const double* W, int nx,
                               double* D) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (s >= n_obs || j >= r) return;
  double y = 0.0;
  for (int c = 0; c < 8; ++c) {
    const int node = obs_node[s * 8 + c];
    if (node >= 0) y += obs_w[s * 8 + c] * W[(size_t)j * nx + node];
  }
  D[(size_t)j * n_obs + s] = y;
}

// out (nx x r) = scale B^T D (D: n_obs x r), through the CSR transpose of B
__global__ void k_bt_cols(int nx, int r, const int* bt_ptr, const int* bt_idx, const double* bt_w, const double* D,
                          int n_obs, double scale, double* out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (p >= nx || j >= r) return;
  double acc = 0.0;
  for (int e = bt_ptr[p]; e < bt_ptr[p + 1]; ++e) acc += bt_w[e] * D[(size_t)j * n_obs + bt_idx[e]];
  out[(size_t)j * nx + p] = scale * acc;
}

// out[p] = sum_k W[p, k] V[row, k]  (one time column of the factored W V^T)
__global__ void k_factor_row(int nx, int r, const double* W, const double* V, int ldv, int row, double* out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nx) return;
  double acc = 0.0;
  for (int k = 0; k < r; ++k) acc += W[(size_t)k * nx + p] * V[(size_t)k * ldv + row];
  out[p] = acc;
}

// Partial inner products of the m vectors V[:, k] (n entries each, ld n)
// with w over this CTA's contiguous range of rows: part[blk * m + k]. Many
// CTAs over long vectors (n = nx r), eight vectors per pass over the range.
constexpr int kDotRows = 2048;
// (solve c = blockIdx.y: vectors V + k ldv + c n, w + c n; partials at
// part + c gridDim.x m)
__global__ void __launch_bounds__(256) k_mdot(size_t n, int m, const double* V, size_t ldv, const double* w,
                                              size_t rows, double* part) {
  __shared__ double red[8][8];
  {
    const size_t c = blockIdx.y;
    V += c * n;
    w += c * n;
    part += c * gridDim.x * (size_t)m;
  }
  const size_t i0 = (size_t)blockIdx.x * rows;
  const size_t i1 = min(n, i0 + rows);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k0 = 0; k0 < m; k0 += 8) {
    const int kn = min(8, m - k0);
    double acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.0;
    for (size_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
      const double wi = w[i];
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (q < kn) acc[q] += V[(size_t)(k0 + q) * ldv + i] * wi;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      double v = acc[q];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[q][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < kn) {
      double t = 0.0;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[threadIdx.x][q];
      part[(size_t)blockIdx.x * m + k0 + threadIdx.x] = t;
    }
    __syncthreads();
  }
}

// w[i] += alpha sum_k h[k] V[k n + i], i < n (m <= kGmresMax + 1 vectors of
// n entries, coefficients on the device): the Gram-Schmidt update of GMRES
// and its final combination, streaming the basis once with many loads in
// flight per thread.
// (solve c = blockIdx.y: V + k ldv + c n, h + c hs, w + c n)
__global__ void __launch_bounds__(256) k_mupdate(size_t n, int m, const double* V, size_t ldv, const double* h,
                                                 size_t hs, double alpha, double* w) {
  __shared__ double sh[64];
  const size_t c = blockIdx.y;
  if (threadIdx.x < m && threadIdx.x < 64) sh[threadIdx.x] = h[c * hs + threadIdx.x];
  __syncthreads();
  V += c * n;
  w += c * n;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
#pragma unroll 8
    for (int k = 0; k < m; ++k) acc += sh[k] * V[(size_t)k * ldv + i];
    w[i] += alpha * acc;
  }
}

// out_c[k] = beta out_c[k] + sum_b part_c[b * m + k] (fixed order); one warp
// per k; solve c = blockIdx.y (partials at c nblk m, output at out + c os)
__global__ void k_mdot_sum(int nblk, int m, const double* part, double* out, size_t os, double beta) {
  const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (k >= m) return;
  const size_t c = blockIdx.y;
  part += c * nblk * (size_t)m;
  out += c * os;
  double t = 0.0;
  for (int b = lane; b < nblk; b += 32) t += part[(size_t)b * m + k];
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (lane == 0) out[k] = (beta == 0.0 ? 0.0 : beta * out[k]) + t;
}

// Partial products A^T B (A: nx x m, B: nx x nb, m nb <= kTnMaxEntries) over
// this CTA's contiguous range of rows, staged through shared memory
// kTnRows rows at a time: part[blk * m nb + e], e = k + m j. Many CTAs over
// the rows (the library's FP64 product splits rows into chunks of at least
// 4096, one CTA each, which leaves a 127^2 grid with 4 CTAs).
constexpr int kTnRows = 16;
constexpr int kTnMaxEntries = 4096;
__global__ void __launch_bounds__(256) k_tn_small(int nx, int m, int nb, const double* A, int lda, const double* B,
                                                  int ldb, int rows, double* part) {
  extern __shared__ double sh[];  // [kTnRows][m + nb]
  const int wd = m + nb;
  const int r0 = blockIdx.x * rows, r1 = min(nx, r0 + rows);
  const int ne = m * nb;
  double acc[kTnMaxEntries / 256];
#pragma unroll
  for (int q = 0; q < kTnMaxEntries / 256; ++q) acc[q] = 0.0;
  for (int base = r0; base < r1; base += kTnRows) {
    const int nr = min(kTnRows, r1 - base);
    __syncthreads();
    for (int e = threadIdx.x; e < nr * wd; e += blockDim.x) {
      const int c = e / nr, i = e - c * nr;
      sh[i * wd + c] = c < m ? A[(size_t)c * lda + base + i] : B[(size_t)(c - m) * ldb + base + i];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kTnMaxEntries / 256; ++q) {
      const int e = threadIdx.x + q * 256;
      if (e < ne) {
        const int j = e / m, k = e - j * m;
        double a = acc[q];
        for (int i = 0; i < nr; ++i) a += sh[i * wd + k] * sh[i * wd + m + j];
        acc[q] = a;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < kTnMaxEntries / 256; ++q) {
    const int e = threadIdx.x + q * 256;
    if (e < ne) part[(size_t)blockIdx.x * ne + e] = acc[q];
  }
}

// C[k, j] = alpha sum_b part[b, e] + beta C[k, j] (fixed order), e = k + m j
__global__ void k_tn_small_sum(int nblk, int m, int nb, const double* part, double* C, int ldc, double alpha,
                               double beta) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int ne = m * nb;
  if (e >= ne) return;
  double t = 0.0;
  for (int b = 0; b < nblk; ++b) t += part[(size_t)b * ne + e];
  const int j = e / m, k = e - j * m;
  double* c = C + (size_t)j * ldc + k;
  *c = alpha * t + (beta == 0.0 ? 0.0 : beta * *c);
}

// Cholesky factor and its inverse for Cholesky QR (one CTA, r <= 64): with
// M = G + shift_rel trace(G) I, M = R^T R (R upper triangular, column
// oriented right-looking elimination), then Rinv = R^{-1} by backward
// elimination on [R | I]. A pivot d <= floor_rel trace(G) (a column of the factored
// matrix that is zero, or dependent to rounding) marks a vanished direction:
// its row of R and column of Rinv are zero, so A Rinv has a zero column there.
// Rinv: r x r column-major.
__global__ void __launch_bounds__(256) k_chol_inv_rel(int r, const double* G, double shift_rel, double floor_rel,
                                                      double* Rinv) {
  extern __shared__ double sh_chol[];
  double* M = sh_chol;          // M[i + r j]: R (upper triangle)
  double* X = sh_chol + r * r;  // the right half of [R | I]: Rinv
  __shared__ double s_tr;
  __shared__ int s_dead;
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int e = tid; e < r * r; e += nthr) {
    const int i = e % r, j = e / r;
    M[i + r * j] = G[e];
    X[i + r * j] = i == j ? 1.0 : 0.0;
  }
  __syncthreads();
  if (tid == 0) {
    double tr = 0.0;
    for (int i = 0; i < r; ++i) tr += M[i + r * i];
    s_tr = tr;
  }
  __syncthreads();
  const double floor_abs = floor_rel * s_tr;
  for (int i = tid; i < r; i += nthr) M[i + r * i] += shift_rel * s_tr;
  __syncthreads();
  for (int k = 0; k < r; ++k) {
    if (tid == 0) {
      const double d = M[k + r * k];
      const bool dead = !(d > floor_abs);
      s_dead = dead;
      M[k + r * k] = dead ? 0.0 : sqrt(d);
    }
    __syncthreads();
    const double rkk = M[k + r * k];
    const bool dead = s_dead != 0;
    for (int j = k + 1 + tid; j < r; j += nthr) M[k + r * j] = dead ? 0.0 : M[k + r * j] / rkk;
    __syncthreads();
    // trailing update of the upper triangle: M[i][j] -= R[k][i] R[k][j], k < i <= j
    const int m = r - k - 1;
    for (int e = tid; e < m * m; e += nthr) {
      const int i = k + 1 + e % m, j = k + 1 + e / m;
      if (i <= j) M[i + r * j] -= M[k + r * i] * M[k + r * j];
    }
    __syncthreads();
  }
  // R^{-1}: rows k = r-1 .. 0 of [R | I]: scale row k by 1 / R_kk, then
  // eliminate column k from the rows above (their right halves)
  for (int k = r - 1; k >= 0; --k) {
    const double rkk = M[k + r * k];
    const double inv = rkk > 0.0 ? 1.0 / rkk : 0.0;
    for (int j = tid; j < r; j += nthr) X[k + r * j] *= inv;
    __syncthreads();
    for (int e = tid; e < k * r; e += nthr) {
      const int i = e % k, j = e / k;
      X[i + r * j] -= M[i + r * k] * X[k + r * j];
    }
    __syncthreads();
  }
  for (int e = tid; e < r * r; e += nthr) {
    const int i = e % r, j = e / r;
    Rinv[e] = j >= i ? X[i + r * j] : 0.0;
  }
}

// out = trace(G) of an r x r matrix (column-major); one thread
__global__ void k_trace(int r, const double* G, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double t = 0.0;
  for (int i = 0; i < r; ++i) t += G[(size_t)i * r + i];
  *out = t;
}

// out = sum_ij Ga[i, j] Gb[i, j]; one CTA.
__global__ void k_frob(int n, const double* Ga, const double* Gb, double* out) {
  __shared__ double red[32];
  double d = 0.0;
  for (int e = threadIdx.x; e < n; e += blockDim.x) d += Ga[e] * Gb[e];
  for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    *out = s;
  }
}

// ---------------------------------------------------------------------------
// host side
//
// A call solves nb independent systems (same operator, own sources and
// starts) at once: every per-solve array holds nb copies at a fixed stride,
// the GMRES of the space steps runs with a Hessenberg matrix per solve, and
// one preconditioner launch serves the r blocks of every solve.

unsigned grid1(size_t n) { return (unsigned)((n + 255) / 256); }

// Y = A X - X T for the ncol = nb r columns of X (solve c with its own
// r x r matrix Tm + c r r), or Y = A X (Tm NULL); A^T if transpose.
lrp_status kron_apply(lrp_problem* P, int r, int ncol, const double* X, const double* Tm, int transpose, double* Y) {
  const OpLevel& l0 = P->step.lv[0];
  dim3 g(grid1(P->nx), ncol);
  cudaStream_t s = P->stream;
  note_launch();
  if (P->step.conv) {
    if (P->dim == 2)
      k_kron_apply<2, false, true><<<g, 256, 0, s>>>(l0, r, ncol, X, Tm, transpose, Y);
    else
      k_kron_apply<3, false, true><<<g, 256, 0, s>>>(l0, r, ncol, X, Tm, transpose, Y);
  } else if (P->step.has_kappa) {
    if (P->dim == 2)
      k_kron_apply<2, true, false><<<g, 256, 0, s>>>(l0, r, ncol, X, Tm, transpose, Y);
    else
      k_kron_apply<3, true, false><<<g, 256, 0, s>>>(l0, r, ncol, X, Tm, transpose, Y);
  } else {
    if (P->dim == 2)
      k_kron_apply<2, false, false><<<g, 256, 0, s>>>(l0, r, ncol, X, Tm, transpose, Y);
    else
      k_kron_apply<3, false, false><<<g, 256, 0, s>>>(l0, r, ncol, X, Tm, transpose, Y);
  }
  CKL(cudaGetLastError());
  return LRP_OK;
}

// slots of AlsWS::scal, nb entries each
enum { S_G = 0, S_R0, S_INV0, S_W, S_INV, S_RES, S_F, S_RA, S_RB, S_NSLOT };

// Work arrays of nb alternating solves (r columns, source rank rf).
struct AlsWS {
  int nx = 0, nt = 0, r = 0, rf = 0, nb = 0, nb_cap = 0;
  size_t n1 = 0;  // nx r: one solve's space factor
  Buf<double> V, W, Q, G, Tm, inv_s, Ahat, Gt, Z, M1, AQ, part, scal;
  Buf<double> Vb, Zb, H, cs, sn, g, y, hv;  // GMRES
  Buf<double> Xc, Yc, Gx, Gy;                 // residual
  Buf<double> Gq, Rq;                         // Cholesky QR: Gram matrix and inverse factor
  Buf<double> tn;                             // partials of the thin products
  size_t tn_cap = 0;
  Buf<double> dinv;                           // per-column shifted inverse diagonals (kappa), FP64 then FP32
  Buf<Op> ops;                                // device copy of the per-column operators
  Buf<int> stat;
  size_t part_cap = 0;
  size_t lev_nodes = 0;  // sum of the level sizes
  std::vector<double> inv_s_host;
  int rc() const { return r + std::max(rf, 1); }
  size_t hs() const { return (size_t)(kGmresMax + 1) * kGmresMax; }
  cudaError_t init(lrp_problem* P, int r_, int rf_, int nb_) {
    nx = P->nx;
    nt = P->nt;
    r = r_;
    rf = rf_;
    nb = nb_cap = nb_;
    n1 = (size_t)nx * r;
    const size_t B = (size_t)nb_cap;
    const int c2 = rc();
    part_cap = B * 1024 * (kGmresMax + 1);
    cudaError_t e = V.alloc(B * nt * r);
    if (e == cudaSuccess) e = W.alloc(B * n1);
    if (e == cudaSuccess) e = Q.alloc(B * n1);
    if (e == cudaSuccess) e = G.alloc(B * n1);
    if (e == cudaSuccess) e = Tm.alloc(B * r * r);
    if (e == cudaSuccess) e = inv_s.alloc(B * r);
    if (e == cudaSuccess) e = Ahat.alloc(B * r * r);
    if (e == cudaSuccess) e = Gt.alloc(B * nt * r);
    if (e == cudaSuccess) e = Z.alloc(B * nt * r);
    if (e == cudaSuccess) e = M1.alloc(B * c2 * c2);
    if (e == cudaSuccess) e = AQ.alloc(B * n1);
    if (e == cudaSuccess) e = part.alloc(part_cap);
    if (e == cudaSuccess) e = scal.alloc(B * S_NSLOT);
    if (e == cudaSuccess) e = Vb.alloc(B * n1 * (kGmresMax + 1));
    if (e == cudaSuccess) e = Zb.alloc(B * n1 * kGmresMax);
    if (e == cudaSuccess) e = H.alloc(B * hs());
    if (e == cudaSuccess) e = cs.alloc(B * kGmresMax);
    if (e == cudaSuccess) e = sn.alloc(B * kGmresMax);
    if (e == cudaSuccess) e = g.alloc(B * (kGmresMax + 1));
    if (e == cudaSuccess) e = y.alloc(B * kGmresMax);
    if (e == cudaSuccess) e = hv.alloc(B * (kGmresMax + 1));
    if (e == cudaSuccess) e = Xc.alloc(B * nx * c2);
    if (e == cudaSuccess) e = Yc.alloc(B * nt * c2);
    if (e == cudaSuccess) e = Gx.alloc((size_t)c2 * c2);
    if (e == cudaSuccess) e = Gy.alloc((size_t)c2 * c2);
    if (e == cudaSuccess) e = stat.alloc(1);
    if (e == cudaSuccess) e = ops.alloc(B * r);
    if (e == cudaSuccess) e = Gq.alloc((size_t)r * r);
    if (e == cudaSuccess) e = Rq.alloc((size_t)r * r);
    tn_cap = (size_t)512 * kTnMaxEntries;
    if (e == cudaSuccess) e = tn.alloc(tn_cap);
    lev_nodes = 0;
    for (int l = 0; l < P->L; ++l) lev_nodes += (size_t)P->step.lv[l].N;
    if (e == cudaSuccess && P->step.has_kappa) e = dinv.alloc(lev_nodes * B * r * 3 / 2 + B * r * 2 * P->L);
    inv_s_host.assign(B * r, 1.0);
    return e;
  }
  // per-solve views
  double* Vc(int c) const { return V.p + (size_t)c * nt * r; }
  double* Wc(int c) const { return W.p + (size_t)c * n1; }
  double* Qc(int c) const { return Q.p + (size_t)c * n1; }
  double* Gc(int c) const { return G.p + (size_t)c * n1; }
  double* AQc(int c) const { return AQ.p + (size_t)c * n1; }
  double* Ahatc(int c) const { return Ahat.p + (size_t)c * r * r; }
  double* Gtc(int c) const { return Gt.p + (size_t)c * nt * r; }
  double* Zc(int c) const { return Z.p + (size_t)c * nt * r; }
  double* M1c(int c) const { return M1.p + (size_t)c * rc() * rc(); }
  double* Xcc(int c) const { return Xc.p + (size_t)c * nx * rc(); }
  double* Ycc(int c) const { return Yc.p + (size_t)c * nt * rc(); }
  double* slot(int k) const { return scal.p + (size_t)k * nb_cap; }
};

// Solves per call of the product: as many as fit a budget of ~6 GB for the
// Krylov bases of one AlsWS, at most 32.
int als_batch_cap(const lrp_problem* P, int r) {
  const double per = 8.0 * (2 * kGmresMax + 1) * (double)P->nx * r;
  return (int)std::max(1.0, std::min(32.0, std::floor(6e9 / per)));
}

// Drops the per-column operators from the problem handle when a solve ends
// (their device copy belongs to the solve's work arrays).
struct ShiftOpsGuard {
  lrp_problem* P;
  ~ShiftOpsGuard() {
    P->shift_ops.clear();
    P->shift_ops_dev = nullptr;
    P->shift_transpose = 0;
  }
};

struct AlsCounters {
  int gmres_iters = 0, gmres_iters_max = 0, precond_solves = 0;
  bool noconv = false;        // some GMRES space step missed its tolerance
  bool pcg_capped = false;    // some preconditioner solve stopped at its iteration cap (not an error)
  double gmres_worst = 0.0;   // largest final relative residual of a GMRES space step that missed
  double ms_space = 0.0, ms_time = 0.0;
};

std::string noconv_message(bool pcg, double gmres_worst) {
  std::string m;
  if (pcg) m = "a spatial solve missed its tolerance within pcg_maxit";
  if (gmres_worst > 0.0) {
    if (!m.empty()) m += "; ";
    char buf[160];
    std::snprintf(buf, sizeof(buf), "a GMRES space step stopped at relative residual %.3e after %d cycles",
                  gmres_worst, kGmresCycles);
    m += buf;
  }
  return m;
}

// The per-column operators A - T_jj I = (1 - T_jj)(I + (tau / (1 - T_jj)) L)
// of the preconditioner, as scaled copies of the time-step operator (nb r
// of them: column j of solve c at c r + j).
lrp_status build_shift_ops(lrp_problem* P, AlsWS& w) {
  cudaStream_t s = P->stream;
  const int ncol = w.nb * w.r;
  CKL(cudaMemcpyAsync(w.inv_s_host.data(), w.inv_s.p, sizeof(double) * ncol, cudaMemcpyDeviceToHost, s));
  CKL(cudaStreamSynchronize(s));
  P->shift_ops.assign(ncol, P->step);
  P->shift_ops_dev = w.ops.p;
  size_t off = 0;
  double* dd = w.dinv.p;
  float* df = w.dinv.p ? (float*)(w.dinv.p + w.lev_nodes * (size_t)w.nb_cap * w.r) : nullptr;
  for (int j = 0; j < ncol; ++j) {
    const double is = w.inv_s_host[j];  // 1 / (1 - T_jj)
    Op& op = P->shift_ops[j];
    for (int l = 0; l < P->L; ++l) {
      OpLevel& lv = op.lv[l];
      lv.ch2 *= is;
      double cs = 0.0;
      for (int a = 0; a < 3; ++a) {
        lv.cw[a] *= is;
        if (a < P->dim) cs += std::fabs(lv.cw[a]);
      }
      lv.dinv = 1.0 / (1.0 + lv.ch2 * 2 * P->dim + cs);
      if (P->step.has_kappa) {
        const int N = lv.N;
        note_launch();
        k_shift_dinv<<<grid1(N), 256, 0, s>>>(N, P->step.lv[l].dinvd, is, dd + off, df + off);
        CKL(cudaGetLastError());
        lv.dinvd = dd + off;
        lv.dinvf = df + off;
        off += (size_t)N;
      }
    }
  }
  return LRP_OK;
}

// z = blockdiag(A - T_jj I)^{-1} v for the nb r columns: one sweep launch,
// one solve per column with its own operator, then the 1/(1 - T_jj) scaling.
// Each solve is als_prec_its (0 -> kPrecondIts) CG iterations from zero, or,
// with als_prec_rtol > 0, a solve to that relative residual (at least the
// problem's own). Flexible GMRES accepts an inexact, even iteration-dependent
// preconditioner; measured on the 127^2 workload (rank 16, 3 sweeps), two
// iterations per application took the GMRES from 37 to 40 iterations and the
// solve from 123 ms to 41 ms against solves to 1e-4. (A full solve to the
// problem's 1e-13 is not even attainable when 1 - T_jj is near zero: the
// block is then ill-conditioned.) A solve that stops at its iteration cap is
// not an error here: the GMRES residual decides.
lrp_status precond(lrp_problem* P, AlsWS& w, const double* v, double* z, AlsCounters& c) {
  lrp_apply_stats st;
  std::memset(&st, 0, sizeof(st));
  const int ncol = w.nb * w.r;
  const SolveCfg saved = P->cfg;
  if (P->desc.als_prec_rtol > 0.0) {
    P->cfg.rtol = std::max(saved.rtol, P->desc.als_prec_rtol);
  } else {
    // a fixed number of PCG iterations (one FP32 inner solve on the mixed path)
    P->cfg.rtol = std::max(saved.rtol, kPrecondRtol);
    P->cfg.maxit = P->desc.als_prec_its > 0 ? P->desc.als_prec_its : kPrecondIts;
    P->cfg.maxref = 1;
  }
  lrp_status res = run_sweep_ex(P, ST_LOAD_X | ST_SHIFTED | ST_STORE_Y, ncol, v, w.nx, z, w.nx, nullptr, 0, nullptr,
                                0, &st, 0, 0, nullptr, 0);
  P->cfg = saved;
  if (res == LRP_ENOCONV)
    c.pcg_capped = true;
  else if (res != LRP_OK)
    return res;
  c.precond_solves += st.n_solves;
  note_launch();
  k_col_scale<<<grid1((size_t)w.nx * ncol), 256, 0, P->stream>>>((size_t)w.nx, ncol, w.inv_s.p, z);
  CKL(cudaGetLastError());
  return LRP_OK;
}

// For every solve c < w.nb: out[c os + k] = beta out + <V_k, x> over n
// entries, V_k = V + k ldv + c n, x = X + c n; many CTAs per solve
// (k_mdot) and a fixed-order sum of their partials.
cudaError_t mdot(cudaStream_t s, AlsWS& w, size_t n, int m, const double* V, size_t ldv, const double* X,
                 double* out, size_t os, double beta) {
  size_t rows = kDotRows;
  size_t nblk = (n + rows - 1) / rows;
  const size_t cap = std::min<size_t>(1024, w.part_cap / ((size_t)std::max(m, 1) * w.nb));
  if (nblk > cap) {
    rows = (n + cap - 1) / cap;
    nblk = (n + rows - 1) / rows;
  }
  note_launch();
  k_mdot<<<dim3((unsigned)nblk, w.nb), 256, 0, s>>>(n, m, V, ldv, X, rows, w.part.p);
  note_launch();
  k_mdot_sum<<<dim3((m + 7) / 8, w.nb), 256, 0, s>>>((int)nblk, m, w.part.p, out, os, beta);
  return cudaGetLastError();
}

// For every solve c < w.nb: x_c += alpha sum_k h[c hs + k] V_k (V_k = V + k
// ldv + c n; x_c = X + c n)
cudaError_t mupdate(cudaStream_t s, AlsWS& w, size_t n, int m, const double* V, size_t ldv, const double* h,
                    size_t hs, double alpha, double* X) {
  if (m <= 0) return cudaSuccess;
  const size_t per = std::max<size_t>(1, (1216 + w.nb - 1) / w.nb);
  const unsigned grid = (unsigned)std::min<size_t>((n + 255) / 256, per);
  note_launch();
  k_mupdate<<<dim3(grid, w.nb), 256, 0, s>>>(n, m, V, ldv, h, hs, alpha, X);
  return cudaGetLastError();
}

// C (m x nb, ld ldc) = alpha A^T B + beta C for thin products (A: nx x m,
// B: nx x nb): k_tn_small over many CTAs when m nb <= kTnMaxEntries and
// m + nb <= 256 (its shared-memory tile), else the library's FP64 product.
cudaError_t small_tn(cudaStream_t s, AlsWS& w, int nx, int m, int nb, const double* A, int lda, const double* B,
                     int ldb, double* C, int ldc, double alpha, double beta) {
  const int ne = m * nb;
  if (ne <= 0) return cudaSuccess;
  if (ne > kTnMaxEntries || m + nb > 256) return gemm_tn(s, nx, m, nb, A, lda, B, ldb, C, ldc, alpha, beta, w.part.p, w.part_cap);
  int nblk = std::min<int>((nx + 127) / 128, (int)std::min<size_t>(512, w.tn_cap / (size_t)ne));
  nblk = std::max(nblk, 1);
  const int rows = (nx + nblk - 1) / nblk;
  nblk = (nx + rows - 1) / rows;
  const size_t smem = (size_t)kTnRows * (m + nb) * sizeof(double);
  note_launch();
  k_tn_small<<<nblk, 256, smem, s>>>(nx, m, nb, A, lda, B, ldb, rows, w.tn.p);
  note_launch();
  k_tn_small_sum<<<(ne + 255) / 256, 256, 0, s>>>(nblk, m, nb, w.tn.p, C, ldc, alpha, beta);
  return cudaGetLastError();
}

// A (rows x r, ld rows; r <= 64) <- an orthonormal basis of its columns by
// shifted Cholesky QR followed by two Cholesky QR passes (Fukaya, Kannan,
// Nakatsukasa, Yamamoto, Yanagisawa, "Shifted Cholesky QR for computing the
// QR factorization of ill-conditioned matrices", SIAM J. Sci. Comput. 2020):
// the shift 11 (rows r + r (r + 1)) u ||A||_F^2 makes the first factorisation
// succeed for condition numbers up to about 1/u, after which the basis is
// well conditioned and CholeskyQR2 restores orthogonality to rounding. Each
// pass is a thin Gram product, one small CTA and one tall product (no
// cooperative launch). tmp: rows x r scratch. Columns that vanish (zero,
// or dependent to rounding) come out as zero columns.
cudaError_t orth_cholqr(cudaStream_t s, AlsWS& w, int rows, int r, double* A, double* tmp) {
  const double u = 1.1102230246251565e-16;  // unit roundoff 2^-53
  double* src = A;
  double* dst = tmp;
  for (int pass = 0; pass < 3; ++pass) {
    cudaError_t e = small_tn(s, w, rows, r, r, src, rows, src, rows, w.Gq.p, r, 1.0, 0.0);
    if (e != cudaSuccess) return e;
    // shift relative to ||A||_F^2 = trace(G): applied inside k_chol_inv
    const double shift_rel = pass == 0 ? 11.0 * ((double)rows * r + (double)r * (r + 1)) * u : 0.0;
    const size_t smem = 2 * (size_t)r * r * sizeof(double);
    if (smem > 48 * 1024) {
      e = cudaFuncSetAttribute(k_chol_inv_rel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    note_launch();
    k_chol_inv_rel<<<1, 256, smem, s>>>(r, w.Gq.p, shift_rel, 64.0 * u, w.Rq.p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = gemm_nn(s, rows, r, r, 1.0, src, rows, w.Rq.p, r, 0.0, dst, rows);
    if (e != cudaSuccess) return e;
    std::swap(src, dst);
  }
  // three passes: the result is in tmp
  return cudaMemcpyAsync(A, src, (size_t)rows * r * sizeof(double), cudaMemcpyDeviceToDevice, s);
}

// Space step of every solve: A W_c - W_c T_c = G_c by flexible GMRES,
// right-preconditioned with blockdiag(A - T_jj I), from the start in W (zero
// if !warm), each to a relative residual gtol ||G_c||. The solves share the
// iterations (one preconditioner launch and one kernel per step for all of
// them) and have their own Hessenberg matrices, rotations and residuals; the
// iteration ends when every solve has reached its tolerance.
lrp_status space_step(lrp_problem* P, AlsWS& w, int transpose, bool warm, double gtol, AlsCounters& c) {
  cudaStream_t s = P->stream;
  const int nb = w.nb, r = w.r, kmax = kGmresMax;
  const size_t n1 = w.n1, N = (size_t)nb * n1;
  const int ldh = kmax + 1;
  const size_t hs = w.hs();
  CKS(build_shift_ops(P, w));
  P->shift_transpose = transpose;
  std::vector<double> h(2 * (size_t)nb), rres(nb), target(nb), gnorm(nb);
  // ||G_c||^2
  CKL(mdot(s, w, n1, 1, w.G.p, n1, w.G.p, w.slot(S_G), 1, 0.0));
  if (!warm) CKL(cudaMemsetAsync(w.W.p, 0, N * sizeof(double), s));
  int iters = 0;
  for (int cyc = 0; cyc < kGmresCycles; ++cyc) {
    // r0 = G - K(W) into Vb[0]
    double* v0 = w.Vb.p;
    if (warm || cyc > 0) {
      CKS(kron_apply(P, r, nb * r, w.W.p, w.Tm.p, transpose, v0));
      CKL(axpby(s, N, 1.0, w.G.p, -1.0, v0));
    } else {
      CKL(cudaMemcpyAsync(v0, w.G.p, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    CKL(cudaMemsetAsync(w.H.p, 0, (size_t)nb * hs * sizeof(double), s));
    CKL(cudaMemsetAsync(w.g.p, 0, (size_t)nb * (kmax + 1) * sizeof(double), s));
    CKL(mdot(s, w, n1, 1, v0, n1, v0, w.slot(S_R0), 1, 0.0));
    note_launch();
    k_norm_entry<<<nb, 1, 0, s>>>(w.slot(S_R0), w.g.p, (size_t)(kmax + 1), w.slot(S_INV0));
    CKL(cudaGetLastError());
    note_launch();
    k_scale_by<<<dim3(grid1(n1), nb), 256, 0, s>>>(n1, w.slot(S_INV0), v0, v0);
    CKL(cudaGetLastError());
    CKL(cudaMemcpyAsync(h.data(), w.slot(S_G), nb * sizeof(double), cudaMemcpyDeviceToHost, s));
    CKL(cudaMemcpyAsync(h.data() + nb, w.slot(S_R0), nb * sizeof(double), cudaMemcpyDeviceToHost, s));
    CKL(cudaStreamSynchronize(s));
    bool all_done = true;
    for (int i = 0; i < nb; ++i) {
      gnorm[i] = std::sqrt(std::max(h[i], 0.0));
      target[i] = gtol * gnorm[i];
      rres[i] = std::sqrt(std::max(h[nb + i], 0.0));
      if (!std::isfinite(rres[i])) {
        set_error("alternating solve: non-finite residual in the space step");
        return LRP_ENONFINITE;
      }
      if (!(gnorm[i] > 0.0)) {
        // a zero right-hand side: the solution is zero, and the solve's
        // Krylov start and rotated right-hand side are zeroed so that the
        // shared iterations leave it at zero
        CKL(cudaMemsetAsync(w.Wc(i), 0, n1 * sizeof(double), s));
        CKL(cudaMemsetAsync(v0 + (size_t)i * n1, 0, n1 * sizeof(double), s));
        CKL(cudaMemsetAsync(w.g.p + (size_t)i * (kmax + 1), 0, (kmax + 1) * sizeof(double), s));
        rres[i] = 0.0;
      }
      if (rres[i] > target[i]) all_done = false;
    }
    if (all_done) break;
    int m = 0;
    for (int j = 0; j < kmax; ++j) {
      double* vj = w.Vb.p + (size_t)j * N;
      double* zj = w.Zb.p + (size_t)j * N;
      double* wv = w.Vb.p + (size_t)(j + 1) * N;
      CKS(precond(P, w, vj, zj, c));
      CKS(kron_apply(P, r, nb * r, zj, w.Tm.p, transpose, wv));
      // classical Gram-Schmidt twice against v_0..v_j of each solve
      for (int pass = 0; pass < 2; ++pass) {
        CKL(mdot(s, w, n1, j + 1, w.Vb.p, N, wv, w.hv.p, (size_t)(kmax + 1), 0.0));
        CKL(mupdate(s, w, n1, j + 1, w.Vb.p, N, w.hv.p, (size_t)(kmax + 1), -1.0, wv));
        note_launch();
        k_hadd<<<nb, 64, 0, s>>>(j + 1, w.hv.p, (size_t)(kmax + 1), w.H.p + (size_t)j * ldh, hs);
        CKL(cudaGetLastError());
      }
      CKL(mdot(s, w, n1, 1, wv, n1, wv, w.slot(S_W), 1, 0.0));
      note_launch();
      k_norm_entry<<<nb, 1, 0, s>>>(w.slot(S_W), w.H.p + (size_t)j * ldh + j + 1, hs, w.slot(S_INV));
      CKL(cudaGetLastError());
      note_launch();
      k_scale_by<<<dim3(grid1(n1), nb), 256, 0, s>>>(n1, w.slot(S_INV), wv, wv);
      CKL(cudaGetLastError());
      note_launch();
      k_givens<<<nb, 1, 0, s>>>(j, w.H.p, ldh, hs, w.cs.p, w.sn.p, w.g.p, kmax, w.slot(S_RES));
      CKL(cudaGetLastError());
      CKL(cudaMemcpyAsync(rres.data(), w.slot(S_RES), nb * sizeof(double), cudaMemcpyDeviceToHost, s));
      CKL(cudaStreamSynchronize(s));
      m = j + 1;
      ++iters;
      all_done = true;
      for (int i = 0; i < nb; ++i) {
        if (!std::isfinite(rres[i])) {
          set_error("alternating solve: non-finite residual in the space step");
          return LRP_ENONFINITE;
        }
        if (gnorm[i] > 0.0 && rres[i] > target[i]) all_done = false;
      }
      if (all_done) break;
    }
    // W_c += Z_c y_c
    note_launch();
    k_backsolve<<<nb, 1, 0, s>>>(m, w.H.p, ldh, hs, w.g.p, w.y.p, kmax);
    CKL(cudaGetLastError());
    CKL(mupdate(s, w, n1, m, w.Zb.p, N, w.y.p, (size_t)kmax, 1.0, w.W.p));
    warm = true;
    if (all_done) break;
    if (cyc == kGmresCycles - 1) {
      c.noconv = true;
      for (int i = 0; i < nb; ++i)
        if (gnorm[i] > 0.0) c.gmres_worst = std::max(c.gmres_worst, rres[i] / gnorm[i]);
    }
  }
  c.gmres_iters += iters;
  c.gmres_iters_max = std::max(c.gmres_iters_max, iters);
  return LRP_OK;
}

// nb alternating solves of A Y_c - Y_c S^T = Wf_c Vf_c^T (A^T with transpose)
// with the factors Wf_c (nx x rf, at Wf + c nx rf), Vf_c (nt x rf, at Vf + c
// nt rf) and the starts in w.V (nt x r each). Runs `sweeps` sweeps (or until
// every residual is <= tol); Y_c ~ W_c V_c^T on return, res[c sweeps + s] the
// relative residual of solve c after sweep s. *done_sweeps: sweeps taken.
lrp_status als_run(lrp_problem* P, AlsWS& w, int transpose, const double* Wf, const double* Vf, int sweeps,
                   double tol, double* res, int* done_sweeps, AlsCounters& c) {
  cudaStream_t s = P->stream;
  const int nx = w.nx, nt = w.nt, r = w.r, rf = w.rf, nb = w.nb;
  const double gtol = std::max(10.0 * P->cfg.rtol, 1e-12);
  const int rc = r + rf;
  auto Wfc = [&](int i) { return Wf + (size_t)i * nx * rf; };
  auto Vfc = [&](int i) { return Vf + (size_t)i * nt * rf; };
  // ||F_c||_F^2 = sum (Wf^T Wf) .* (Vf^T Vf)
  std::vector<double> f2(nb, 0.0);
  if (rf > 0) {
    for (int i = 0; i < nb; ++i) {
      CKL(small_tn(s, w, nx, rf, rf, Wfc(i), nx, Wfc(i), nx, w.Gx.p, rf, 1.0, 0.0));
      CKL(small_tn(s, w, nt, rf, rf, Vfc(i), nt, Vfc(i), nt, w.Gy.p, rf, 1.0, 0.0));
      note_launch();
      k_frob<<<1, 256, 0, s>>>(rf * rf, w.Gx.p, w.Gy.p, w.slot(S_F) + i);
      CKL(cudaGetLastError());
    }
    CKL(cudaMemcpyAsync(f2.data(), w.slot(S_F), nb * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  // orthonormal starts
  for (int i = 0; i < nb; ++i) CKL(orth_cholqr(s, w, nt, r, w.Vc(i), w.Gtc(i)));
  CKL(cudaStreamSynchronize(s));
  *done_sweeps = 0;
  bool any = false;
  for (int i = 0; i < nb; ++i) any = any || f2[i] > 0.0;
  if (!any) {
    CKL(cudaMemsetAsync(w.W.p, 0, (size_t)nb * w.n1 * sizeof(double), s));
    if (res)
      for (size_t k = 0; k < (size_t)nb * sweeps; ++k) res[k] = 0.0;
    CKL(cudaStreamSynchronize(s));
    return LRP_OK;
  }
  const size_t smem_t = ((size_t)r * 2 * r + 2 * r) * sizeof(double);
  CKL(cudaFuncSetAttribute(k_als_time, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_t));
  std::vector<double> rr(2 * (size_t)nb);
  for (int sw = 0; sw < sweeps; ++sw) {
    auto t0 = std::chrono::steady_clock::now();
    // ---- space step
    CKL(cudaMemsetAsync(w.stat.p, 0, sizeof(int), s));
    note_launch();
    k_shift_gram<<<dim3(r * r, nb), 256, 0, s>>>(nt, r, w.V.p, w.Tm.p, w.inv_s.p, w.stat.p);
    CKL(cudaGetLastError());
    for (int i = 0; i < nb; ++i) {
      CKL(small_tn(s, w, nt, rf, r, Vfc(i), nt, w.Vc(i), nt, w.M1c(i), rf, 1.0, 0.0));
      CKL(gemm_nn(s, nx, rf, r, 1.0, Wfc(i), nx, w.M1c(i), rf, 0.0, w.Gc(i), nx));
    }
    int hstat = 0;
    CKL(cudaMemcpyAsync(&hstat, w.stat.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    CKL(cudaStreamSynchronize(s));
    if (hstat) {
      set_error("alternating solve: a time basis vector with 1 - T_jj <= 0 (basis not orthonormal)");
      return LRP_ENONFINITE;
    }
    CKS(space_step(P, w, transpose, sw > 0, gtol, c));
    auto t1 = std::chrono::steady_clock::now();
    c.ms_space += std::chrono::duration<double, std::milli>(t1 - t0).count();
    // ---- time step
    CKL(cudaMemcpyAsync(w.Q.p, w.W.p, (size_t)nb * w.n1 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    for (int i = 0; i < nb; ++i) CKL(orth_cholqr(s, w, nx, r, w.Qc(i), w.AQc(i)));
    CKS(kron_apply(P, r, nb * r, w.Q.p, nullptr, transpose, w.AQ.p));
    for (int i = 0; i < nb; ++i) {
      CKL(small_tn(s, w, nx, r, r, w.Qc(i), nx, w.AQc(i), nx, w.Ahatc(i), r, 1.0, 0.0));
      // Gt (nt x r) = Vf (Wf^T Q)
      CKL(small_tn(s, w, nx, rf, r, Wfc(i), nx, w.Qc(i), nx, w.M1c(i), rf, 1.0, 0.0));
      CKL(gemm_nn(s, nt, rf, r, 1.0, Vfc(i), nt, w.M1c(i), rf, 0.0, w.Gtc(i), nt));
    }
    note_launch();
    k_als_time<<<nb, 1024, smem_t, s>>>(r, nt, w.Ahat.p, w.Gt.p, w.Z.p);
    CKL(cudaGetLastError());
    // V, R_Z = qr(Z); W = Q R_Z^T = Q (Z^T V)
    CKL(cudaMemcpyAsync(w.V.p, w.Z.p, (size_t)nb * nt * r * sizeof(double), cudaMemcpyDeviceToDevice, s));
    for (int i = 0; i < nb; ++i) {
      CKL(orth_cholqr(s, w, nt, r, w.Vc(i), w.Gtc(i)));
      CKL(small_tn(s, w, nt, r, r, w.Zc(i), nt, w.Vc(i), nt, w.M1c(i), r, 1.0, 0.0));
      CKL(gemm_nn(s, nx, r, r, 1.0, w.Qc(i), nx, w.M1c(i), r, 0.0, w.Wc(i), nx));
    }
    // ---- residual. After the time step Q^T R = 0, so with X1 = (I - Q Q^T) A W,
    // X2 = (I - Q Q^T) Wf and the source's time factor split along V,
    // Vf = V C + Pv (C = V^T Vf, V^T Pv = 0):
    //   R = X1 V^T - X2 Vf^T = (X1 - X2 C^T) V^T - X2 Pv^T,
    // two mutually orthogonal terms, and ||(X1 - X2 C^T) V^T|| = ||X1 - X2 C^T||
    // (V orthonormal). The state and the source cancel in the vector
    // X1 - X2 C^T (rounding relative to the residual itself), not in a sum
    // of squares (which would floor the relative residual near 1e-8).
    for (int i = 0; i < nb; ++i) {
      double* X1 = w.Xcc(i);
      double* X2 = X1 + (size_t)nx * r;
      double* Pv = w.Ycc(i);
      double* M1 = w.M1c(i);
      CKS(kron_apply(P, r, r, w.Wc(i), nullptr, transpose, X1));
      CKL(cudaMemcpyAsync(X2, Wfc(i), (size_t)nx * rf * sizeof(double), cudaMemcpyDeviceToDevice, s));
      for (int pass = 0; pass < 2; ++pass) {
        CKL(small_tn(s, w, nx, r, rc, w.Qc(i), nx, X1, nx, w.Gx.p, r, 1.0, 0.0));
        CKL(gemm_nn(s, nx, r, rc, -1.0, w.Qc(i), nx, w.Gx.p, r, 1.0, X1, nx));
      }
      CKL(small_tn(s, w, nt, rf, r, Vfc(i), nt, w.Vc(i), nt, M1, rf, 1.0, 0.0));
      CKL(gemm_nn(s, nx, rf, r, -1.0, X2, nx, M1, rf, 1.0, X1, nx));
      CKL(cudaMemcpyAsync(Pv, Vfc(i), (size_t)nt * rf * sizeof(double), cudaMemcpyDeviceToDevice, s));
      for (int pass = 0; pass < 2; ++pass) {
        CKL(small_tn(s, w, nt, r, rf, w.Vc(i), nt, Pv, nt, w.Gx.p, r, 1.0, 0.0));
        CKL(gemm_nn(s, nt, r, rf, -1.0, w.Vc(i), nt, w.Gx.p, r, 1.0, Pv, nt));
      }
      CKL(small_tn(s, w, nx, r, r, X1, nx, X1, nx, w.Gy.p, r, 1.0, 0.0));
      note_launch();
      k_trace<<<1, 64, 0, s>>>(r, w.Gy.p, w.slot(S_RA) + i);
      CKL(cudaGetLastError());
      CKL(small_tn(s, w, nx, rf, rf, X2, nx, X2, nx, w.Gx.p, rf, 1.0, 0.0));
      CKL(small_tn(s, w, nt, rf, rf, Pv, nt, Pv, nt, w.Gy.p, rf, 1.0, 0.0));
      note_launch();
      k_frob<<<1, 256, 0, s>>>(rf * rf, w.Gx.p, w.Gy.p, w.slot(S_RB) + i);
      CKL(cudaGetLastError());
    }
    CKL(cudaMemcpyAsync(rr.data(), w.slot(S_RA), nb * sizeof(double), cudaMemcpyDeviceToHost, s));
    CKL(cudaMemcpyAsync(rr.data() + nb, w.slot(S_RB), nb * sizeof(double), cudaMemcpyDeviceToHost, s));
    CKL(cudaStreamSynchronize(s));
    c.ms_time += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t1).count();
    bool all_tol = tol > 0.0;
    for (int i = 0; i < nb; ++i) {
      const double rel = f2[i] > 0.0 ? std::sqrt(std::max(rr[i] + rr[nb + i], 0.0) / f2[i]) : 0.0;
      if (!std::isfinite(rel)) {
        set_error("alternating solve: non-finite residual");
        return LRP_ENONFINITE;
      }
      if (res) res[(size_t)i * sweeps + sw] = rel;
      all_tol = all_tol && rel <= tol;
    }
    *done_sweeps = sw + 1;
    if (all_tol) break;
  }
  return LRP_OK;
}

}  // namespace

namespace {

constexpr unsigned kPriorStages = ST_LOAD_X | ST_PRIOR_IN | ST_STORE_Y;

}  // namespace

// The Hessian product with both space-time solves by the alternating solver
// (flag LRP_ALS_SOLVES of lrp_hessian_apply; X, Y device arrays). The
// columns go in batches (als_batch_cap): one prior solve launch for the
// batch, the forward solves of the batch as one batched alternating solve
// (source z_c e_1^T), the adjoint sources B^T B W_Y / sigma^2 with the
// unobserved steps' rows of V_Y zeroed, the adjoint solves as one batched
// alternating solve in reversed time, q_1 of each, one prior solve launch.
lrp_status als_hessian_impl(lrp_problem* P, int nvec, const double* X, int ldx, double* Y, int ldy, bool misfit,
                            lrp_apply_stats* stats) {
  auto t0 = std::chrono::steady_clock::now();
  const int nx = P->nx, nt = P->nt;
  const int r = std::min({P->desc.als_rank > 0 ? P->desc.als_rank : 16, nt, nx, kMaxRank});
  const int sweeps = P->desc.als_sweeps > 0 ? P->desc.als_sweeps : 3;
  const double tol = P->desc.als_tol;
  cudaStream_t s = P->stream;
  const int nbc = std::max(1, std::min(nvec, als_batch_cap(P, r)));
  AlsWS fw, aw;
  CKL(fw.init(P, r, 1, nbc));
  CKL(aw.init(P, r, r, nbc));
  Buf<double> z, e1, Wa, Va, D, q1;
  CKL(z.alloc((size_t)nx * nbc));
  CKL(e1.alloc((size_t)nt * nbc));
  CKL(Wa.alloc((size_t)nx * r * nbc));
  CKL(Va.alloc((size_t)nt * r * nbc));
  CKL(D.alloc((size_t)P->n_obs * r * nbc));
  CKL(q1.alloc((size_t)nx * nbc));
  {
    std::vector<double> unit((size_t)nt * nbc, 0.0);
    for (int i = 0; i < nbc; ++i) unit[(size_t)i * nt] = 1.0;
    CKL(cudaMemcpyAsync(e1.p, unit.data(), unit.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  }
  // starts: the first r time steps (unit vectors), for every solve
  std::vector<double> start((size_t)nt * r * nbc, 0.0);
  for (int i = 0; i < nbc; ++i)
    for (int j = 0; j < r; ++j) start[(size_t)i * nt * r + (size_t)j * nt + j] = 1.0;
  std::vector<double> hist((size_t)nbc * sweeps);
  AlsCounters c;
  ShiftOpsGuard guard{P};
  double res_f = 0.0, res_a = 0.0;
  bool noconv = false;
  lrp_apply_stats pst;
  for (int col0 = 0; col0 < nvec; col0 += nbc) {
    const int nb = std::min(nbc, nvec - col0);
    fw.nb = aw.nb = nb;
    const double* x = X + (size_t)col0 * ldx;
    if (misfit) {
      CKL(cudaMemcpy2DAsync(z.p, (size_t)nx * sizeof(double), x, (size_t)ldx * sizeof(double),
                            (size_t)nx * sizeof(double), nb, cudaMemcpyDeviceToDevice, s));
    } else {
      lrp_status pr = run_sweep_ex(P, kPriorStages, nb, x, ldx, z.p, nx, nullptr, 0, nullptr, 0, &pst, 0, 0,
                                   nullptr, 0);
      if (pr == LRP_ENOCONV)
        noconv = true;
      else if (pr != LRP_OK)
        return pr;
    }
    // forward: A Y_c - Y_c S^T = z_c e_1^T
    CKL(cudaMemcpyAsync(fw.V.p, start.data(), (size_t)nb * nt * r * sizeof(double), cudaMemcpyHostToDevice, s));
    int done = 0;
    CKS(als_run(P, fw, 0, z.p, e1.p, sweeps, tol, hist.data(), &done, c));
    for (int i = 0; i < nb && done > 0; ++i) res_f = std::max(res_f, hist[(size_t)i * sweeps + done - 1]);
    // adjoint sources: f_n = B^T B y_n / sigma^2 at the observed steps, as
    // factors (B^T B W / sigma^2) (mask V)^T, in reversed time (all nb r
    // columns of the batch at once: the factors are stored solve by solve)
    {
      const int ncol = nb * r;
      dim3 go((P->n_obs + 255) / 256, ncol);
      note_launch();
      k_observe_cols<<<go, 256, 0, s>>>(P->n_obs, ncol, P->obs_node, P->obs_w, fw.W.p, nx, D.p);
      CKL(cudaGetLastError());
      dim3 gb(grid1(nx), ncol);
      const double is2 = 1.0 / (P->desc.sigma * P->desc.sigma);
      note_launch();
      k_bt_cols<<<gb, 256, 0, s>>>(nx, ncol, P->bt_ptr, P->bt_idx, P->bt_w, D.p, P->n_obs, is2, Wa.p);
      CKL(cudaGetLastError());
      dim3 gr(grid1(nt), ncol);
      note_launch();
      k_rows_reverse<<<gr, 256, 0, s>>>(nt, ncol, fw.V.p, nt, Va.p, P->desc.obs_every, P->n_steps);
      CKL(cudaGetLastError());
    }
    CKL(cudaMemcpyAsync(aw.V.p, start.data(), (size_t)nb * nt * r * sizeof(double), cudaMemcpyHostToDevice, s));
    CKS(als_run(P, aw, 1, Wa.p, Va.p, sweeps, tol, hist.data(), &done, c));
    for (int i = 0; i < nb && done > 0; ++i) res_a = std::max(res_a, hist[(size_t)i * sweeps + done - 1]);
    // q_1 = the last column of each reversed solution
    for (int i = 0; i < nb; ++i) {
      note_launch();
      k_factor_row<<<grid1(nx), 256, 0, s>>>(nx, r, aw.Wc(i), aw.Vc(i), nt, nt - 1, q1.p + (size_t)i * nx);
      CKL(cudaGetLastError());
    }
    double* y = Y + (size_t)col0 * ldy;
    if (misfit) {
      CKL(cudaMemcpy2DAsync(y, (size_t)ldy * sizeof(double), q1.p, (size_t)nx * sizeof(double),
                            (size_t)nx * sizeof(double), nb, cudaMemcpyDeviceToDevice, s));
    } else {
      lrp_status pr = run_sweep_ex(P, kPriorStages, nb, q1.p, nx, y, ldy, nullptr, 0, nullptr, 0, &pst, 0, 0,
                                   nullptr, 0);
      if (pr == LRP_ENOCONV)
        noconv = true;
      else if (pr != LRP_OK)
        return pr;
    }
  }
  CKL(cudaStreamSynchronize(s));
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->n_solves = nvec > 0 ? c.precond_solves / nvec : 0;
    stats->time_rank_max = r;
    stats->time_trunc_err = res_f;
    stats->adj_rank_max = r;
    stats->adj_trunc_err = res_a;
    stats->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  if (noconv || c.noconv) {
    set_error(noconv_message(noconv, c.gmres_worst));
    return LRP_ENOCONV;
  }
  return LRP_OK;
}

}  // namespace lrp

using namespace lrp;

extern "C" lrp_status lrp_als_solve(lrp_problem* P, int transpose, int rf, const double* Wf, int ldwf,
                                    const double* Vf, int ldvf, int r, const double* V0, int ldv0, int sweeps,
                                    double tol, double* W, int ldw, double* V, int ldv, double* res,
                                    lrp_als_stats* st) {
  if (!P || rf < 0 || rf > kMaxRank || r < 1 || r > kMaxRank || r > P->nt || r > P->nx || sweeps < 1 ||
      (rf > 0 && (!Wf || !Vf || ldwf < P->nx || ldvf < P->nt)) || !V0 || ldv0 < P->nt || !W || ldw < P->nx || !V ||
      ldv < P->nt) {
    set_error("lrp_als_solve: need 1 <= r <= min(64, nt, nx), 0 <= rf <= 64, sweeps >= 1, non-NULL factors with "
              "leading dimensions >= nx (space) and nt (time)");
    return LRP_EINVAL;
  }
  for (const void* a : {(const void*)Wf, (const void*)Vf, (const void*)V0, (const void*)W, (const void*)V}) {
    if (!a) continue;
    lrp_status sd = check_on_device(P->device, a, "lrp_als_solve");
    if (sd != LRP_OK) return sd;
  }
  cudaSetDevice(P->device);
  auto t0 = std::chrono::steady_clock::now();
  const int nx = P->nx, nt = P->nt;
  cudaStream_t s = P->stream;
  AlsWS w;
  CKL(w.init(P, r, rf, 1));
  Buf<double> dWf, dVf, tmp;
  CKL(dWf.alloc((size_t)nx * std::max(rf, 1)));
  CKL(dVf.alloc((size_t)nt * std::max(rf, 1)));
  CKL(tmp.alloc((size_t)nt * std::max(r, rf)));
  if (rf > 0) {
    CKL(cudaMemcpy2DAsync(dWf.p, (size_t)nx * sizeof(double), Wf, (size_t)ldwf * sizeof(double),
                          (size_t)nx * sizeof(double), rf, cudaMemcpyDefault, s));
    CKL(cudaMemcpy2DAsync(transpose ? tmp.p : dVf.p, (size_t)nt * sizeof(double), Vf, (size_t)ldvf * sizeof(double),
                          (size_t)nt * sizeof(double), rf, cudaMemcpyDefault, s));
    if (transpose) {
      dim3 g(grid1(nt), rf);
      note_launch();
      k_rows_reverse<<<g, 256, 0, s>>>(nt, rf, tmp.p, nt, dVf.p, 0, 0);
      CKL(cudaGetLastError());
    }
  }
  CKL(cudaMemcpy2DAsync(transpose ? tmp.p : w.V.p, (size_t)nt * sizeof(double), V0, (size_t)ldv0 * sizeof(double),
                        (size_t)nt * sizeof(double), r, cudaMemcpyDefault, s));
  if (transpose) {
    dim3 g(grid1(nt), r);
    note_launch();
    k_rows_reverse<<<g, 256, 0, s>>>(nt, r, tmp.p, nt, w.V.p, 0, 0);
    CKL(cudaGetLastError());
  }
  AlsCounters c;
  int done = 0;
  std::vector<double> hist(sweeps, 0.0);
  lrp_status rs;
  {
    ShiftOpsGuard guard{P};
    rs = als_run(P, w, transpose, dWf.p, dVf.p, sweeps, tol, hist.data(), &done, c);
  }
  if (rs != LRP_OK) return rs;
  CKL(cudaMemcpy2DAsync(W, (size_t)ldw * sizeof(double), w.W.p, (size_t)nx * sizeof(double),
                        (size_t)nx * sizeof(double), r, cudaMemcpyDefault, s));
  if (transpose) {
    dim3 g(grid1(nt), r);
    note_launch();
    k_rows_reverse<<<g, 256, 0, s>>>(nt, r, w.V.p, nt, tmp.p, 0, 0);
    CKL(cudaGetLastError());
  }
  CKL(cudaMemcpy2DAsync(V, (size_t)ldv * sizeof(double), transpose ? tmp.p : w.V.p, (size_t)nt * sizeof(double),
                        (size_t)nt * sizeof(double), r, cudaMemcpyDefault, s));
  CKL(cudaStreamSynchronize(s));
  if (res)
    for (int k = 0; k < sweeps; ++k) res[k] = k < done ? hist[k] : 0.0;
  if (st) {
    std::memset(st, 0, sizeof(*st));
    st->sweeps = done;
    st->gmres_iters = c.gmres_iters;
    st->gmres_iters_max = c.gmres_iters_max;
    st->precond_solves = c.precond_solves;
    st->residual = done > 0 ? hist[done - 1] : 0.0;
    st->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    st->ms_space = c.ms_space;
    st->ms_time = c.ms_time;
  }
  if (c.noconv) {
    set_error(noconv_message(false, c.gmres_worst));
    return LRP_ENOCONV;
  }
  return LRP_OK;
}
