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
//  * the time step (Eq. (amen_2)): W orthonormalised to Q, the Galerkin
//    projection onto span(Q) in space, Ahat z_n - z_{n-1} = Q^T f_n with
//    Ahat = Q^T A Q (r x r), solved directly (one CTA: Gauss-Jordan inverse,
//    then the nt-step recurrence), Y = Q Z^T, V = orth(Z), W = Q R_Z^T.
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
#include <memory>
#include <string>
#include <thread>
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

constexpr int kMaxRank = 64;     // block Gram-Schmidt limit (columns of W and of Z)
constexpr int kGmresMax = 40;    // Krylov vectors per GMRES cycle
constexpr int kGmresCycles = 6;  // restarts per space step
constexpr double kPrecondRtol = 1e-8;  // stop of a preconditioner solve before its iteration cap
constexpr int kPrecondIts = 2;         // default CG iterations per preconditioner solve

// ---------------------------------------------------------------------------
// kernels

// Y[:, j] = (A x_j) - sum_i x_i Tm[i, j] for the r columns of X (nx x r,
// ld nx): the operator of the space step (Tm = T) or plain A X (Tm NULL).
// A = I + tau L of the problem on its finest level (transpose: A^T).
template <int DIM, bool KAPPA, bool CONV>
__global__ void k_kron_apply(const OpLevel l0, int r, const double* X, const double* Tm, int transpose, double* Y) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (p >= l0.N || j >= r) return;
  const size_t nx = (size_t)l0.N;
  int i0, i1, i2;
  decomp<DIM>(l0, p, i0, i1, i2);
  Ld<double> ld{X + (size_t)j * nx, 0, 0};
  double d;
  double v;
  if (CONV)
    v = op_conv_at<DIM>(l0, ld, p, i0, i1, i2, transpose != 0, d);
  else
    v = op_at<double, DIM, KAPPA>(l0, ld, p, i0, i1, i2, d);
  if (Tm) {
    for (int i = 0; i < r; ++i) v -= X[(size_t)i * nx + p] * Tm[(size_t)j * r + i];
  }
  Y[(size_t)j * nx + p] = v;
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
__global__ void k_givens(int j, double* H, int ldh, double* cs, double* sn, double* g, double* res) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
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
__global__ void k_backsolve(int m, const double* H, int ldh, const double* g, double* y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = m - 1; i >= 0; --i) {
    double acc = g[i];
    for (int k = i + 1; k < m; ++k) acc -= H[(size_t)k * ldh + i] * y[k];
    const double d = H[(size_t)i * ldh + i];
    y[i] = d != 0.0 ? acc / d : 0.0;
  }
}

// H[j+1, j] = sqrt(*nrm2) and g[0] = that norm for j < 0 (the start of a
// cycle); inv = 1 / the norm (0 for a vanished vector).
__global__ void k_norm_entry(const double* nrm2, double* dst, double* inv) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double v = sqrt(fmax(*nrm2, 0.0));
  *dst = v;
  *inv = v > 0.0 ? 1.0 / v : 0.0;
}

// y = (*scale) x (n entries)
__global__ void k_scale_by(size_t n, const double* scale, const double* x, double* y) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = (*scale) * x[i];
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
__global__ void __launch_bounds__(1024) k_als_time(int r, int nt, const double* Ahat, const double* Gt, double* Z) {
  extern __shared__ double sm[];
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
__global__ void __launch_bounds__(256) k_mdot(size_t n, int m, const double* V, const double* w, size_t rows,
                                              double* part) {
  __shared__ double red[8][8];
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
        if (q < kn) acc[q] += V[(size_t)(k0 + q) * n + i] * wi;
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
__global__ void __launch_bounds__(256) k_mupdate(size_t n, int m, const double* V, const double* h, double alpha,
                                                 double* w) {
  __shared__ double sh[64];
  if (threadIdx.x < m && threadIdx.x < 64) sh[threadIdx.x] = h[threadIdx.x];
  __syncthreads();
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
#pragma unroll 8
    for (int k = 0; k < m; ++k) acc += sh[k] * V[(size_t)k * n + i];
    w[i] += alpha * acc;
  }
}

// out[k] = beta out[k] + sum_b part[b * m + k] (fixed order); one warp per k.
__global__ void k_mdot_sum(int nb, int m, const double* part, double* out, double beta) {
  const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (k >= m) return;
  double t = 0.0;
  for (int b = lane; b < nb; b += 32) t += part[(size_t)b * m + k];
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

unsigned grid1(size_t n) { return (unsigned)((n + 255) / 256); }

// Y = A X - X Tm for the r columns of X (Tm NULL: Y = A X); A^T if transpose.
lrp_status kron_apply(lrp_problem* P, int r, const double* X, const double* Tm, int transpose, double* Y) {
  const OpLevel& l0 = P->step.lv[0];
  dim3 g(grid1(P->nx), r);
  cudaStream_t s = P->stream;
  note_launch();
  if (P->step.conv) {
    if (P->dim == 2)
      k_kron_apply<2, false, true><<<g, 256, 0, s>>>(l0, r, X, Tm, transpose, Y);
    else
      k_kron_apply<3, false, true><<<g, 256, 0, s>>>(l0, r, X, Tm, transpose, Y);
  } else if (P->step.has_kappa) {
    if (P->dim == 2)
      k_kron_apply<2, true, false><<<g, 256, 0, s>>>(l0, r, X, Tm, transpose, Y);
    else
      k_kron_apply<3, true, false><<<g, 256, 0, s>>>(l0, r, X, Tm, transpose, Y);
  } else {
    if (P->dim == 2)
      k_kron_apply<2, false, false><<<g, 256, 0, s>>>(l0, r, X, Tm, transpose, Y);
    else
      k_kron_apply<3, false, false><<<g, 256, 0, s>>>(l0, r, X, Tm, transpose, Y);
  }
  CKL(cudaGetLastError());
  return LRP_OK;
}

// Work arrays of one alternating solve (r columns, source rank rf).
struct AlsWS {
  int nx = 0, nt = 0, r = 0, rf = 0;
  Buf<double> V, W, Q, G, Tm, inv_s, Ahat, Gt, Z, Rz, M1, AQ, part, gs, scal;
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
  cudaError_t init(lrp_problem* P, int r_, int rf_) {
    nx = P->nx;
    nt = P->nt;
    r = r_;
    rf = rf_;
    const size_t blk = (size_t)nx * r;
    const int rc = r + std::max(rf, 1);
    part_cap = (size_t)128 * std::max(rc, kGmresMax + 1) * 16;  // >= 1024 (kGmresMax + 1) for mdot
    cudaError_t e = V.alloc((size_t)nt * r);
    if (e == cudaSuccess) e = W.alloc(blk);
    if (e == cudaSuccess) e = Q.alloc(blk);
    if (e == cudaSuccess) e = G.alloc(blk);
    if (e == cudaSuccess) e = Tm.alloc((size_t)r * r);
    if (e == cudaSuccess) e = inv_s.alloc(r);
    if (e == cudaSuccess) e = Ahat.alloc((size_t)r * r);
    if (e == cudaSuccess) e = Gt.alloc((size_t)nt * r);
    if (e == cudaSuccess) e = Z.alloc((size_t)nt * r);
    if (e == cudaSuccess) e = Rz.alloc((size_t)r * r);
    if (e == cudaSuccess) e = M1.alloc((size_t)rc * rc);
    if (e == cudaSuccess) e = AQ.alloc(blk);
    if (e == cudaSuccess) e = part.alloc(part_cap);
    if (e == cudaSuccess) e = gs.alloc(block_gs_scratch_doubles());
    if (e == cudaSuccess) e = scal.alloc(8);
    if (e == cudaSuccess) e = Vb.alloc(blk * (kGmresMax + 1));
    if (e == cudaSuccess) e = Zb.alloc(blk * kGmresMax);
    if (e == cudaSuccess) e = H.alloc((size_t)(kGmresMax + 1) * kGmresMax);
    if (e == cudaSuccess) e = cs.alloc(kGmresMax);
    if (e == cudaSuccess) e = sn.alloc(kGmresMax);
    if (e == cudaSuccess) e = g.alloc(kGmresMax + 1);
    if (e == cudaSuccess) e = y.alloc(kGmresMax);
    if (e == cudaSuccess) e = hv.alloc(kGmresMax + 1);
    if (e == cudaSuccess) e = Xc.alloc((size_t)nx * rc);
    if (e == cudaSuccess) e = Yc.alloc((size_t)nt * rc);
    if (e == cudaSuccess) e = Gx.alloc((size_t)rc * rc);
    if (e == cudaSuccess) e = Gy.alloc((size_t)rc * rc);
    if (e == cudaSuccess) e = stat.alloc(1);
    if (e == cudaSuccess) e = ops.alloc(r);
    if (e == cudaSuccess) e = Gq.alloc((size_t)r * r);
    if (e == cudaSuccess) e = Rq.alloc((size_t)r * r);
    tn_cap = (size_t)512 * kTnMaxEntries;
    if (e == cudaSuccess) e = tn.alloc(tn_cap);
    lev_nodes = 0;
    for (int l = 0; l < P->L; ++l) lev_nodes += (size_t)P->step.lv[l].N;
    if (e == cudaSuccess && P->step.has_kappa) e = dinv.alloc(lev_nodes * r * 3 / 2 + r * 2 * P->L);
    inv_s_host.assign(r, 1.0);
    return e;
  }
};

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
// of the preconditioner, as scaled copies of the time-step operator.
lrp_status build_shift_ops(lrp_problem* P, AlsWS& w) {
  cudaStream_t s = P->stream;
  CKL(cudaMemcpyAsync(w.inv_s_host.data(), w.inv_s.p, sizeof(double) * w.r, cudaMemcpyDeviceToHost, s));
  CKL(cudaStreamSynchronize(s));
  P->shift_ops.assign(w.r, P->step);
  P->shift_ops_dev = w.ops.p;
  size_t off = 0;
  double* dd = w.dinv.p;
  float* df = w.dinv.p ? (float*)(w.dinv.p + w.lev_nodes * w.r) : nullptr;
  for (int j = 0; j < w.r; ++j) {
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

// z (nx x r) = blockdiag(A - T_jj I)^{-1} v: one sweep launch, one solve per
// column with its own operator, then the 1/(1 - T_jj) scaling.
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
  const SolveCfg saved = P->cfg;
  if (P->desc.als_prec_rtol > 0.0) {
    P->cfg.rtol = std::max(saved.rtol, P->desc.als_prec_rtol);
  } else {
    // a fixed number of PCG iterations (one FP32 inner solve on the mixed path)
    P->cfg.rtol = std::max(saved.rtol, kPrecondRtol);
    P->cfg.maxit = P->desc.als_prec_its > 0 ? P->desc.als_prec_its : kPrecondIts;
    P->cfg.maxref = 1;
  }
  lrp_status res = run_sweep_ex(P, ST_LOAD_X | ST_SHIFTED | ST_STORE_Y, w.r, v, w.nx, z, w.nx, nullptr, 0, nullptr,
                                0, &st, 0, 0, nullptr, 0);
  P->cfg = saved;
  if (res == LRP_ENOCONV)
    c.pcg_capped = true;
  else if (res != LRP_OK)
    return res;
  c.precond_solves += st.n_solves;
  note_launch();
  k_col_scale<<<grid1((size_t)w.nx * w.r), 256, 0, P->stream>>>((size_t)w.nx, w.r, w.inv_s.p, z);
  CKL(cudaGetLastError());
  return LRP_OK;
}

// out[0:m] = beta out + V^T x for m vectors of n entries (V: ld n), over
// many CTAs (k_mdot) and a fixed-order sum of their partials.
cudaError_t mdot(cudaStream_t s, AlsWS& w, size_t n, int m, const double* V, const double* x, double* out,
                 double beta) {
  size_t rows = kDotRows;
  size_t nb = (n + rows - 1) / rows;
  const size_t cap = std::min<size_t>(1024, w.part_cap / (size_t)std::max(m, 1));
  if (nb > cap) {
    rows = (n + cap - 1) / cap;
    nb = (n + rows - 1) / rows;
  }
  note_launch();
  k_mdot<<<(unsigned)nb, 256, 0, s>>>(n, m, V, x, rows, w.part.p);
  note_launch();
  k_mdot_sum<<<(m + 7) / 8, 256, 0, s>>>((int)nb, m, w.part.p, out, beta);
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

// w += alpha V h (V: m vectors of n entries, ld n; h: m device coefficients)
cudaError_t mupdate(cudaStream_t s, size_t n, int m, const double* V, const double* h, double alpha, double* w) {
  if (m <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)std::min<size_t>((n + 255) / 256, 152 * 8);
  note_launch();
  k_mupdate<<<grid, 256, 0, s>>>(n, m, V, h, alpha, w);
  return cudaGetLastError();
}

// <a, b> over n entries into dst (device)
cudaError_t dot_into(cudaStream_t s, AlsWS& w, size_t n, const double* a, const double* b, double* dst, double beta) {
  return mdot(s, w, n, 1, a, b, dst, beta);
}

// Space step: A W - W T = G by flexible GMRES, right-preconditioned with
// blockdiag(A - T_jj I), from the start in w.W (zero if !warm), to a
// relative residual gtol ||G||.
lrp_status space_step(lrp_problem* P, AlsWS& w, int transpose, bool warm, double gtol, AlsCounters& c) {
  cudaStream_t s = P->stream;
  const size_t n = (size_t)w.nx * w.r;
  const int ldh = kGmresMax + 1;
  CKS(build_shift_ops(P, w));
  P->shift_transpose = transpose;
  double hres[2];
  // ||G||
  CKL(dot_into(s, w, n, w.G.p, w.G.p, w.scal.p + 1, 0.0));
  if (!warm) CKL(cudaMemsetAsync(w.W.p, 0, n * sizeof(double), s));
  int iters = 0;
  for (int cyc = 0; cyc < kGmresCycles; ++cyc) {
    // r0 = G - K(W) into Vb[0]
    double* v0 = w.Vb.p;
    if (warm || cyc > 0) {
      CKS(kron_apply(P, w.r, w.W.p, w.Tm.p, transpose, v0));
      CKL(axpby(s, n, 1.0, w.G.p, -1.0, v0));
    } else {
      CKL(cudaMemcpyAsync(v0, w.G.p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    CKL(cudaMemsetAsync(w.H.p, 0, (size_t)ldh * kGmresMax * sizeof(double), s));
    CKL(cudaMemsetAsync(w.g.p, 0, (kGmresMax + 1) * sizeof(double), s));
    CKL(dot_into(s, w, n, v0, v0, w.scal.p + 2, 0.0));
    note_launch();
    k_norm_entry<<<1, 1, 0, s>>>(w.scal.p + 2, w.g.p, w.scal.p + 3);
    CKL(cudaGetLastError());
    note_launch();
    k_scale_by<<<grid1(n), 256, 0, s>>>(n, w.scal.p + 3, v0, v0);
    CKL(cudaGetLastError());
    CKL(cudaMemcpyAsync(hres, w.scal.p + 1, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CKL(cudaStreamSynchronize(s));
    const double gnorm = std::sqrt(std::max(hres[0], 0.0));
    const double target = gtol * gnorm;
    double rnorm = std::sqrt(std::max(hres[1], 0.0));
    if (!(gnorm > 0.0)) {
      CKL(cudaMemsetAsync(w.W.p, 0, n * sizeof(double), s));
      break;
    }
    if (!std::isfinite(rnorm)) {
      set_error("alternating solve: non-finite residual in the space step");
      return LRP_ENONFINITE;
    }
    if (rnorm <= target) break;
    int m = 0;
    for (int j = 0; j < kGmresMax; ++j) {
      double* vj = w.Vb.p + (size_t)j * n;
      double* zj = w.Zb.p + (size_t)j * n;
      double* wv = w.Vb.p + (size_t)(j + 1) * n;
      CKS(precond(P, w, vj, zj, c));
      CKS(kron_apply(P, w.r, zj, w.Tm.p, transpose, wv));
      // classical Gram-Schmidt twice against v_0..v_j (vectors of n entries)
      double* hcol = w.H.p + (size_t)j * ldh;
      for (int pass = 0; pass < 2; ++pass) {
        CKL(mdot(s, w, n, j + 1, w.Vb.p, wv, w.hv.p, 0.0));
        CKL(mupdate(s, n, j + 1, w.Vb.p, w.hv.p, -1.0, wv));
        CKL(axpby(s, (size_t)(j + 1), 1.0, w.hv.p, 1.0, hcol));
      }
      CKL(dot_into(s, w, n, wv, wv, w.scal.p + 4, 0.0));
      note_launch();
      k_norm_entry<<<1, 1, 0, s>>>(w.scal.p + 4, hcol + j + 1, w.scal.p + 5);
      CKL(cudaGetLastError());
      note_launch();
      k_scale_by<<<grid1(n), 256, 0, s>>>(n, w.scal.p + 5, wv, wv);
      CKL(cudaGetLastError());
      note_launch();
      k_givens<<<1, 1, 0, s>>>(j, w.H.p, ldh, w.cs.p, w.sn.p, w.g.p, w.scal.p + 6);
      CKL(cudaGetLastError());
      CKL(cudaMemcpyAsync(&rnorm, w.scal.p + 6, sizeof(double), cudaMemcpyDeviceToHost, s));
      CKL(cudaStreamSynchronize(s));
      m = j + 1;
      ++iters;
      if (!std::isfinite(rnorm)) {
        set_error("alternating solve: non-finite residual in the space step");
        return LRP_ENONFINITE;
      }
      if (rnorm <= target) break;
    }
    // W += Z y
    note_launch();
    k_backsolve<<<1, 1, 0, s>>>(m, w.H.p, ldh, w.g.p, w.y.p);
    CKL(cudaGetLastError());
    CKL(mupdate(s, n, m, w.Zb.p, w.y.p, 1.0, w.W.p));
    warm = true;
    if (rnorm <= target) break;
    if (cyc == kGmresCycles - 1) {
      c.noconv = true;
      c.gmres_worst = std::max(c.gmres_worst, rnorm / gnorm);
    }
  }
  c.gmres_iters += iters;
  c.gmres_iters_max = std::max(c.gmres_iters_max, iters);
  return LRP_OK;
}

// One alternating solve of A Y - Y S^T = Wf Vf^T (A^T with transpose) with
// the factors Wf (nx x rf), Vf (nt x rf) and the start w.V (nt x r), all
// device arrays with leading dimensions nx / nt. Runs `sweeps` sweeps (or
// until the residual is <= tol); Y ~ w.W w.V^T on return, res[s] the
// relative residual after sweep s. *done_sweeps: sweeps taken.
lrp_status als_run(lrp_problem* P, AlsWS& w, int transpose, const double* Wf, const double* Vf, int sweeps,
                   double tol, double* res, int* done_sweeps, AlsCounters& c) {
  cudaStream_t s = P->stream;
  const int nx = w.nx, nt = w.nt, r = w.r, rf = w.rf;
  const double gtol = std::max(10.0 * P->cfg.rtol, 1e-12);
  const int rc = r + rf;
  // ||F||_F^2 = sum (Wf^T Wf) .* (Vf^T Vf)
  double f2 = 0.0;
  if (rf > 0) {
    CKL(small_tn(s, w, nx, rf, rf, Wf, nx, Wf, nx, w.Gx.p, rf, 1.0, 0.0));
    CKL(small_tn(s, w, nt, rf, rf, Vf, nt, Vf, nt, w.Gy.p, rf, 1.0, 0.0));
    note_launch();
    k_frob<<<1, 256, 0, s>>>(rf * rf, w.Gx.p, w.Gy.p, w.scal.p);
    CKL(cudaGetLastError());
    CKL(cudaMemcpyAsync(&f2, w.scal.p, sizeof(double), cudaMemcpyDeviceToHost, s));
    CKL(cudaStreamSynchronize(s));
  }
  // orthonormal start
  CKL(orth_cholqr(s, w, nt, r, w.V.p, w.Gt.p));
  *done_sweeps = 0;
  if (!(f2 > 0.0)) {
    CKL(cudaMemsetAsync(w.W.p, 0, (size_t)nx * r * sizeof(double), s));
    if (res)
      for (int k = 0; k < sweeps; ++k) res[k] = 0.0;
    CKL(cudaStreamSynchronize(s));
    return LRP_OK;
  }
  for (int sw = 0; sw < sweeps; ++sw) {
    auto t0 = std::chrono::steady_clock::now();
    // ---- space step
    CKL(cudaMemsetAsync(w.stat.p, 0, sizeof(int), s));
    note_launch();
    k_shift_gram<<<r * r, 256, 0, s>>>(nt, r, w.V.p, w.Tm.p, w.inv_s.p, w.stat.p);
    CKL(cudaGetLastError());
    CKL(small_tn(s, w, nt, rf, r, Vf, nt, w.V.p, nt, w.M1.p, rf, 1.0, 0.0));
    CKL(gemm_nn(s, nx, rf, r, 1.0, Wf, nx, w.M1.p, rf, 0.0, w.G.p, nx));
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
    CKL(cudaMemcpyAsync(w.Q.p, w.W.p, (size_t)nx * r * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CKL(orth_cholqr(s, w, nx, r, w.Q.p, w.AQ.p));
    CKS(kron_apply(P, r, w.Q.p, nullptr, transpose, w.AQ.p));
    CKL(small_tn(s, w, nx, r, r, w.Q.p, nx, w.AQ.p, nx, w.Ahat.p, r, 1.0, 0.0));
    // Gt (nt x r) = Vf (Wf^T Q)
    CKL(small_tn(s, w, nx, rf, r, Wf, nx, w.Q.p, nx, w.M1.p, rf, 1.0, 0.0));
    CKL(gemm_nn(s, nt, rf, r, 1.0, Vf, nt, w.M1.p, rf, 0.0, w.Gt.p, nt));
    const size_t smem = ((size_t)r * 2 * r + 2 * r) * sizeof(double);
    CKL(cudaFuncSetAttribute(k_als_time, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    note_launch();
    k_als_time<<<1, 1024, smem, s>>>(r, nt, w.Ahat.p, w.Gt.p, w.Z.p);
    CKL(cudaGetLastError());
    // V, R_Z = qr(Z); W = Q R_Z^T = Q (Z^T V)
    CKL(cudaMemcpyAsync(w.V.p, w.Z.p, (size_t)nt * r * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CKL(orth_cholqr(s, w, nt, r, w.V.p, w.Gt.p));
    CKL(small_tn(s, w, nt, r, r, w.Z.p, nt, w.V.p, nt, w.M1.p, r, 1.0, 0.0));
    CKL(gemm_nn(s, nx, r, r, 1.0, w.Q.p, nx, w.M1.p, r, 0.0, w.W.p, nx));
    // ---- residual. After the time step Q^T R = 0, so with X1 = (I - Q Q^T) A W,
    // X2 = (I - Q Q^T) Wf and the source's time factor split along V,
    // Vf = V C + Pv (C = V^T Vf, V^T Pv = 0):
    //   R = X1 V^T - X2 Vf^T = (X1 - X2 C^T) V^T - X2 Pv^T,
    // two mutually orthogonal terms, and ||(X1 - X2 C^T) V^T|| = ||X1 - X2 C^T||
    // (V orthonormal). The state and the source cancel in the vector
    // X1 - X2 C^T (rounding relative to the residual itself), not in a sum
    // of squares (which would floor the relative residual near 1e-8).
    double* X1 = w.Xc.p;
    double* X2 = w.Xc.p + (size_t)nx * r;
    double* Pv = w.Yc.p;
    CKS(kron_apply(P, r, w.W.p, nullptr, transpose, X1));
    CKL(cudaMemcpyAsync(X2, Wf, (size_t)nx * rf * sizeof(double), cudaMemcpyDeviceToDevice, s));
    for (int pass = 0; pass < 2; ++pass) {
      CKL(small_tn(s, w, nx, r, rc, w.Q.p, nx, w.Xc.p, nx, w.Gx.p, r, 1.0, 0.0));
      CKL(gemm_nn(s, nx, r, rc, -1.0, w.Q.p, nx, w.Gx.p, r, 1.0, w.Xc.p, nx));
    }
    CKL(small_tn(s, w, nt, rf, r, Vf, nt, w.V.p, nt, w.M1.p, rf, 1.0, 0.0));
    CKL(gemm_nn(s, nx, rf, r, -1.0, X2, nx, w.M1.p, rf, 1.0, X1, nx));
    CKL(cudaMemcpyAsync(Pv, Vf, (size_t)nt * rf * sizeof(double), cudaMemcpyDeviceToDevice, s));
    for (int pass = 0; pass < 2; ++pass) {
      CKL(small_tn(s, w, nt, r, rf, w.V.p, nt, Pv, nt, w.Gx.p, r, 1.0, 0.0));
      CKL(gemm_nn(s, nt, r, rf, -1.0, w.V.p, nt, w.Gx.p, r, 1.0, Pv, nt));
    }
    CKL(dot_into(s, w, (size_t)nx * r, X1, X1, w.scal.p + 1, 0.0));
    CKL(small_tn(s, w, nx, rf, rf, X2, nx, X2, nx, w.Gx.p, rf, 1.0, 0.0));
    CKL(small_tn(s, w, nt, rf, rf, Pv, nt, Pv, nt, w.Gy.p, rf, 1.0, 0.0));
    note_launch();
    k_frob<<<1, 256, 0, s>>>(rf * rf, w.Gx.p, w.Gy.p, w.scal.p);
    CKL(cudaGetLastError());
    double rr[2] = {0.0, 0.0};
    CKL(cudaMemcpyAsync(rr, w.scal.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CKL(cudaStreamSynchronize(s));
    const double r2 = rr[0] + rr[1];
    c.ms_time += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t1).count();
    const double rel = std::sqrt(std::max(r2, 0.0) / f2);
    if (!std::isfinite(rel)) {
      set_error("alternating solve: non-finite residual");
      return LRP_ENONFINITE;
    }
    if (res) res[sw] = rel;
    *done_sweeps = sw + 1;
    if (tol > 0.0 && rel <= tol) break;
  }
  return LRP_OK;
}

}  // namespace

namespace {

// Work arrays of the product for one column at a time.
struct ColWS {
  AlsWS fw, aw;
  Buf<double> z, e1, Wa, Va, D, q1;
  std::vector<double> start, hist;
  cudaError_t init(lrp_problem* P, int r, int sweeps) {
    const int nx = P->nx, nt = P->nt;
    cudaError_t e = fw.init(P, r, 1);
    if (e == cudaSuccess) e = aw.init(P, r, r);
    if (e == cudaSuccess) e = z.alloc(nx);
    if (e == cudaSuccess) e = e1.alloc(nt);
    if (e == cudaSuccess) e = Wa.alloc((size_t)nx * r);
    if (e == cudaSuccess) e = Va.alloc((size_t)nt * r);
    if (e == cudaSuccess) e = D.alloc((size_t)P->n_obs * r);
    if (e == cudaSuccess) e = q1.alloc(nx);
    std::vector<double> unit(nt, 0.0);
    unit[0] = 1.0;
    if (e == cudaSuccess) e = cudaMemcpy(e1.p, unit.data(), nt * sizeof(double), cudaMemcpyHostToDevice);
    // start: the first r time steps (unit vectors), for both solves
    start.assign((size_t)nt * r, 0.0);
    for (int j = 0; j < r; ++j) start[(size_t)j * nt + j] = 1.0;
    hist.assign(sweeps, 0.0);
    return e;
  }
};

struct ColResult {
  double res_f = 0.0, res_a = 0.0;
  bool noconv = false;
  AlsCounters c;
};

// y = Htilde x (H_mis x) for one column with both space-time systems solved
// by the alternating solver; x, y device vectors.
lrp_status als_column(lrp_problem* P, ColWS& w, int r, int sweeps, double tol, bool misfit, const double* x,
                      double* y, ColResult& cr) {
  const int nx = P->nx, nt = P->nt;
  cudaStream_t s = P->stream;
  const unsigned prior_st = ST_LOAD_X | ST_PRIOR_IN | ST_STORE_Y;
  lrp_apply_stats pst;
  if (misfit) {
    CKL(cudaMemcpyAsync(w.z.p, x, nx * sizeof(double), cudaMemcpyDeviceToDevice, s));
  } else {
    lrp_status pr = run_sweep_ex(P, prior_st, 1, x, nx, w.z.p, nx, nullptr, 0, nullptr, 0, &pst, 0, 0, nullptr, 0);
    if (pr == LRP_ENOCONV)
      cr.noconv = true;
    else if (pr != LRP_OK)
      return pr;
  }
  // forward: A Y - Y S^T = z e_1^T
  CKL(cudaMemcpyAsync(w.fw.V.p, w.start.data(), w.start.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  int done = 0;
  CKS(als_run(P, w.fw, 0, w.z.p, w.e1.p, sweeps, tol, w.hist.data(), &done, cr.c));
  cr.res_f = std::max(cr.res_f, done > 0 ? w.hist[done - 1] : 0.0);
  // adjoint source: f_n = B^T B y_n / sigma^2 at the observed steps, as
  // factors (B^T B W / sigma^2) (mask V)^T, in reversed time
  {
    dim3 go((P->n_obs + 255) / 256, r);
    note_launch();
    k_observe_cols<<<go, 256, 0, s>>>(P->n_obs, r, P->obs_node, P->obs_w, w.fw.W.p, nx, w.D.p);
    CKL(cudaGetLastError());
    dim3 gb(grid1(nx), r);
    const double is2 = 1.0 / (P->desc.sigma * P->desc.sigma);
    note_launch();
    k_bt_cols<<<gb, 256, 0, s>>>(nx, r, P->bt_ptr, P->bt_idx, P->bt_w, w.D.p, P->n_obs, is2, w.Wa.p);
    CKL(cudaGetLastError());
    dim3 gr(grid1(nt), r);
    note_launch();
    k_rows_reverse<<<gr, 256, 0, s>>>(nt, r, w.fw.V.p, nt, w.Va.p, P->desc.obs_every, P->n_steps);
    CKL(cudaGetLastError());
  }
  CKL(cudaMemcpyAsync(w.aw.V.p, w.start.data(), w.start.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  CKS(als_run(P, w.aw, 1, w.Wa.p, w.Va.p, sweeps, tol, w.hist.data(), &done, cr.c));
  cr.res_a = std::max(cr.res_a, done > 0 ? w.hist[done - 1] : 0.0);
  // q_1 = the last column of the reversed solution
  note_launch();
  k_factor_row<<<grid1(nx), 256, 0, s>>>(nx, r, w.aw.W.p, w.aw.V.p, nt, nt - 1, w.q1.p);
  CKL(cudaGetLastError());
  if (misfit) {
    CKL(cudaMemcpyAsync(y, w.q1.p, nx * sizeof(double), cudaMemcpyDeviceToDevice, s));
  } else {
    lrp_status pr = run_sweep_ex(P, prior_st, 1, w.q1.p, nx, y, nx, nullptr, 0, nullptr, 0, &pst, 0, 0, nullptr, 0);
    if (pr == LRP_ENOCONV)
      cr.noconv = true;
    else if (pr != LRP_OK)
      return pr;
  }
  CKL(cudaStreamSynchronize(s));
  return LRP_OK;
}

// A handle that shares the problem's operators, sensors and settings (all
// read-only in a solve) but has its own stream, sweep workspace, statistics
// and per-column operators, so that independent columns can run from
// separate host threads at the same time.
struct SideHandle {
  lrp_problem* h = nullptr;
  lrp_status make(const lrp_problem* P) {
    h = new lrp_problem(*P);
    h->allocs.clear();  // owns none of the problem's arrays
    h->stream = nullptr;
    h->ws = nullptr;
    h->ws_bytes = 0;
    h->ws_fixed = nullptr;
    h->ws_fixed_bytes = 0;
    h->stats = nullptr;
    h->end_buf = nullptr;
    h->prof_on = 0;
    h->prof_ev[0] = h->prof_ev[1] = nullptr;
    h->shift_ops.clear();
    h->shift_ops_dev = nullptr;
    h->src_W = h->src_V = nullptr;
    CKL(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    CKL(dev_malloc(&h->stats, sizeof(Stats)));
    CKL(dev_malloc(&h->end_buf, 65536 * sizeof(int)));
    CKL(cudaMemset(h->end_buf, 0, 65536 * sizeof(int)));
    return LRP_OK;
  }
  ~SideHandle() {
    if (!h) return;
    if (h->stream) {
      cudaStreamSynchronize(h->stream);
      cudaStreamDestroy(h->stream);
    }
    if (h->ws) cudaFree(h->ws);
    if (h->stats) cudaFree(h->stats);
    if (h->end_buf) cudaFree(h->end_buf);
    delete h;
  }
};

constexpr int kAlsStreams = 8;  // columns of a product solved at the same time

}  // namespace

// The Hessian product with both space-time solves by the alternating solver
// (flag LRP_ALS_SOLVES of lrp_hessian_apply; X, Y device arrays). One
// column is one chain of small, synchronising steps (GMRES iterations), so
// up to kAlsStreams columns run at once, each from its own host thread on a
// side handle with its own stream; the results do not depend on this.
lrp_status als_hessian_impl(lrp_problem* P, int nvec, const double* X, int ldx, double* Y, int ldy, bool misfit,
                            lrp_apply_stats* stats) {
  auto t0 = std::chrono::steady_clock::now();
  const int nx = P->nx, nt = P->nt;
  const int r = std::min({P->desc.als_rank > 0 ? P->desc.als_rank : 16, nt, nx, kMaxRank});
  const int sweeps = P->desc.als_sweeps > 0 ? P->desc.als_sweeps : 3;
  const double tol = P->desc.als_tol;
  const int nw = std::max(1, std::min(nvec, kAlsStreams));
  CKL(cudaStreamSynchronize(P->stream));  // X is ready
  std::vector<std::unique_ptr<SideHandle>> side(nw);
  std::vector<ColResult> res(nw);
  std::vector<lrp_status> st(nw, LRP_OK);
  std::vector<std::string> msg(nw);
  // the side handles are copies of P made before any worker runs (the
  // workers change P's per-call state: its settings during a preconditioner
  // solve and its per-column operators)
  for (int wi = 1; wi < nw; ++wi) {
    side[wi].reset(new SideHandle());
    lrp_status sm = side[wi]->make(P);
    if (sm != LRP_OK) return sm;
  }
  auto worker = [&](int wi) {
    cudaSetDevice(P->device);
    lrp_problem* H = wi > 0 ? side[wi]->h : P;
    ColWS w;
    cudaError_t e = w.init(H, r, sweeps);
    if (e != cudaSuccess) {
      st[wi] = cuda_status(e, "alternating solve work arrays");
      msg[wi] = lrp_last_error();
      return;
    }
    ShiftOpsGuard guard{H};
    for (int col = wi; col < nvec; col += nw) {
      st[wi] = als_column(H, w, r, sweeps, tol, misfit, X + (size_t)col * ldx, Y + (size_t)col * ldy, res[wi]);
      if (st[wi] != LRP_OK) {
        msg[wi] = lrp_last_error();
        return;
      }
    }
  };
  {
    std::vector<std::thread> threads;
    for (int wi = 1; wi < nw; ++wi) threads.emplace_back(worker, wi);
    worker(0);
    for (auto& t : threads) t.join();
  }
  side.clear();
  for (int wi = 0; wi < nw; ++wi)
    if (st[wi] != LRP_OK) {
      set_error(msg[wi]);
      return st[wi];
    }
  AlsCounters c;
  double res_f = 0.0, res_a = 0.0;
  bool noconv = false;
  for (const ColResult& cr : res) {
    res_f = std::max(res_f, cr.res_f);
    res_a = std::max(res_a, cr.res_a);
    noconv = noconv || cr.noconv;
    c.noconv = c.noconv || cr.c.noconv;
    c.precond_solves += cr.c.precond_solves;
    c.gmres_worst = std::max(c.gmres_worst, cr.c.gmres_worst);
  }
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
  CKL(w.init(P, r, rf));
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
