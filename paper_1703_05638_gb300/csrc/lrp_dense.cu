// FP64 dense kernels of the Lanczos / posterior stage:
//  * gemm_tn: C = A^T B for tall-skinny A (nx x m) and B (nx x nb), split over
//    row chunks with a fixed-order second-stage reduction (deterministic);
//  * gemm_nn: Y = beta Y + alpha A M for A (nx x m) and a small M (m x nc);
//  * rank-revealing block Gram-Schmidt (CGS2) of up to 64 columns;
//  * symmetric eigensolver for the projected Lanczos matrix: Householder
//    reduction to tridiagonal form, implicit QL iterations with Wilkinson
//    shifts, back-transformation of the eigenvectors;
//  * small elementwise helpers (column norms, scaling, gathers, fills).
// FP64 throughout: the Lanczos eigensolve, re-orthogonalisation and the
// posterior factors stay in FP64.
#include <cuda_runtime.h>

#include <algorithm>

#include <cooperative_groups.h>

#include "lrp_dense.h"
#include "lrp_fp64.cuh"
#include "lrp_internal.h"

namespace lrp {

// ---------------------------------------------------------------- gemm_tn
#define TN_TI 16
#define TN_TR 64

__global__ void __launch_bounds__(256) k_gemm_tn(int nx, int m, int nb, const double* __restrict__ A,
                                                  int lda, const double* __restrict__ B, int ldb,
                                                  double* __restrict__ part, int rows_per_chunk) {
  __shared__ double As[TN_TI][TN_TR + 1];
  __shared__ double Bs[16][TN_TR + 1];
  const int i0 = blockIdx.x * TN_TI;
  const int chunk = blockIdx.y;
  const int r0 = chunk * rows_per_chunk;
  const int r1 = min(nx, r0 + rows_per_chunk);
  const int ti = threadIdx.x >> 4, tj = threadIdx.x & 15;
  double acc = 0.0;
  for (int rb = r0; rb < r1; rb += TN_TR) {
    for (int e = threadIdx.x; e < TN_TI * TN_TR; e += 256) {
      const int ci = e / TN_TR, rr = e % TN_TR;
      const int i = i0 + ci, r = rb + rr;
      As[ci][rr] = (i < m && r < r1) ? A[(size_t)i * lda + r] : 0.0;
    }
    for (int e = threadIdx.x; e < 16 * TN_TR; e += 256) {
      const int cj = e / TN_TR, rr = e % TN_TR;
      const int r = rb + rr;
      Bs[cj][rr] = (cj < nb && r < r1) ? B[(size_t)cj * ldb + r] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < TN_TR; ++rr) acc += As[ti][rr] * Bs[tj][rr];
    __syncthreads();
  }
  const int i = i0 + ti;
  if (i < m && tj < nb) part[((size_t)chunk * m + i) * 16 + tj] = acc;
}

__global__ void k_reduce_parts(int m, int nb, int nchunk, const double* __restrict__ part,
                               double* __restrict__ C, int ldc, double alpha, double beta) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * nb) return;
  const int i = e / nb, j = e % nb;
  double s = 0.0;
  for (int c = 0; c < nchunk; ++c) s += part[((size_t)c * m + i) * 16 + j];
  double* out = C + (size_t)j * ldc + i;
  *out = (beta == 0.0 ? 0.0 : beta * *out) + alpha * s;
}

// ---------------------------------------------------------------- gemm_nn
#define NN_TI 128

__global__ void __launch_bounds__(256) k_gemm_nn(int nx, int m, int nc, double alpha,
                                                  const double* __restrict__ A, int lda,
                                                  const double* __restrict__ M, int ldm, double beta,
                                                  double* Y, int ldy) {
  __shared__ double Ms[NN_TI][16];
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int j0 = blockIdx.y * 16;
  const int ncl = min(16, nc - j0);
  double acc[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) acc[j] = 0.0;
  for (int ib = 0; ib < m; ib += NN_TI) {
    const int ni = min(NN_TI, m - ib);
    __syncthreads();
    for (int e = threadIdx.x; e < NN_TI * 16; e += blockDim.x) {
      const int ii = e >> 4, jj = e & 15;
      Ms[ii][jj] = (ii < ni && jj < ncl) ? M[(size_t)(j0 + jj) * ldm + ib + ii] : 0.0;
    }
    __syncthreads();
    if (p < nx) {
      for (int ii = 0; ii < ni; ++ii) {
        const double a = A[(size_t)(ib + ii) * lda + p];
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[j] += a * Ms[ii][j];
      }
    }
  }
  if (p < nx) {
    for (int j = 0; j < ncl; ++j) {
      double* y = Y + (size_t)(j0 + j) * ldy + p;
      *y = (beta == 0.0 ? 0.0 : beta * *y) + alpha * acc[j];
    }
  }
}


// ---------------------------------------------------------------- eigensolver
// Symmetric eigendecomposition of the n x n matrix A (column-major, ld lda,
// destroyed) into theta (decreasing) and Z (n x n, ld ldz), in three kernels:
// 1. k_tridiag (one CTA): Householder reflections H_k = I - 2 v_k v_k^T zero
//    column k below the subdiagonal, A <- H_k A H_k; the tridiagonal (d, e)
//    and the unit vectors v_k (stored in A below the diagonal) are kept.
// 2. k_tql (several CTAs, each owning a band of rows of Z): implicit QL on
//    (d, e) with Wilkinson shifts: repeatedly pick the unreduced block [l, m],
//    shift by the eigenvalue of the leading 2x2 closest to d_l and chase the
//    bulge with plane rotations from m-1 down to l. The rotation angles depend
//    only on (d, e): lane 0 of warp 0 computes the next chase (every CTA the
//    same, from the same data) while the other warps apply the previous one
//    to the CTA's rows of the tridiagonal problem's eigenvector matrix (rows
//    of the identity at the start). Eigenvalues are then ranked (decreasing)
//    and the rows written with their columns in that order.
// 3. k_eig_back (one warp per column): Z <- H_0 H_1 ... H_{n-3} Z, the
//    eigenvectors of A.
#define EIG_NT 512
#define TQL_NT 64      // warp 0 computes the chases, warp 1 applies them
#define TQL_ROWS 32    // rows of Z per CTA (one per thread of warp 1)
#define BACK_WARPS 8   // columns per CTA of the back-transformation

__device__ __forceinline__ double eig_block_sum(double x, double* s_red) {
  const int tid = threadIdx.x;
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  if ((tid & 31) == 0) s_red[tid >> 5] = x;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < EIG_NT / 32; ++w) s += s_red[w];
  __syncthreads();
  return s;
}

// work: d (n), e (n), tau (n; 2 for a stored reflection, 0 for none), then
// two n-vectors of scratch.
__global__ void __launch_bounds__(EIG_NT) k_tridiag(int n, double* A, int lda, double* work) {
  __shared__ double s_red[EIG_NT / 32];
  const int tid = threadIdx.x;
  double* d = work;
  double* e = work + n;
  double* tau = work + 2 * n;
  double* v = work + 3 * n;
  double* pvec = work + 4 * n;
  auto At = [&](int i, int j) -> double& { return A[(size_t)j * lda + i]; };
  for (int k = 0; k + 2 < n; ++k) {
    const int m0 = k + 1, len = n - m0;
    double part = 0.0;
    for (int i = tid; i < len; i += EIG_NT) {
      const double x = At(m0 + i, k);
      part += x * x;
    }
    const double xnorm2 = eig_block_sum(part, s_red);
    const double x0 = At(m0, k);
    const double tail2 = xnorm2 - x0 * x0;
    if (!(tail2 > 1e-300)) {  // column already reduced
      if (tid == 0) {
        e[k] = x0;
        tau[k] = 0.0;
      }
      continue;
    }
    const double xnorm = sqrt(xnorm2);
    const double alpha = x0 > 0 ? -xnorm : xnorm;
    // v = x - alpha e1, normalised, kept in column k below the diagonal
    const double v0 = x0 - alpha;
    const double vnorm = sqrt(tail2 + v0 * v0);
    for (int i = tid; i < len; i += EIG_NT) {
      const double vi = (i == 0 ? v0 : At(m0 + i, k)) / vnorm;
      v[i] = vi;
      At(m0 + i, k) = vi;
    }
    __syncthreads();
    // p = 2 B v on the trailing block B = A[m0:, m0:]
    for (int i = tid; i < len; i += EIG_NT) {
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
      int j = 0;
      for (; j + 3 < len; j += 4) {
        s0 = fma(At(m0 + i, m0 + j), v[j], s0);
        s1 = fma(At(m0 + i, m0 + j + 1), v[j + 1], s1);
        s2 = fma(At(m0 + i, m0 + j + 2), v[j + 2], s2);
        s3 = fma(At(m0 + i, m0 + j + 3), v[j + 3], s3);
      }
      for (; j < len; ++j) s0 = fma(At(m0 + i, m0 + j), v[j], s0);
      pvec[i] = 2.0 * ((s0 + s1) + (s2 + s3));
    }
    __syncthreads();
    double kp = 0.0;
    for (int i = tid; i < len; i += EIG_NT) kp += v[i] * pvec[i];
    const double K = eig_block_sum(kp, s_red);
    // q = p - K v; B <- B - v q^T - q v^T
    for (int i = tid; i < len; i += EIG_NT) pvec[i] -= K * v[i];
    __syncthreads();
    for (int idx = tid; idx < len * len; idx += EIG_NT) {
      const int i = idx % len, j = idx / len;
      At(m0 + i, m0 + j) -= v[i] * pvec[j] + pvec[i] * v[j];
    }
    if (tid == 0) {
      e[k] = alpha;
      tau[k] = 2.0;
    }
    __syncthreads();
  }
  for (int i = tid; i < n; i += EIG_NT) {
    d[i] = At(i, i);
    if (i + 2 >= n) e[i] = (i + 1 < n) ? At(i + 1, i) : 0.0;
    if (i + 2 >= n) tau[i] = 0.0;
  }
}

// Dynamic shared memory: d, e (n each), two chase buffers (c then s, n each),
// the CTA's rows of the eigenvector matrix (rows x (n+1)), the ranking (n ints).
__global__ void __launch_bounds__(TQL_NT) k_tql(int n, const double* work, double* Z, int ldz, double* theta,
                                                int* status, int rows) {
  extern __shared__ double sm_tql[];
  double* d = sm_tql;
  double* e = d + n;
  double* cs = e + n;  // buffer b: c at cs + 2 n b, s at cs + 2 n b + n
  double* Zs = cs + 4 * n;
  const int ldzs = n + 1;
  int* perm = (int*)(Zs + (size_t)rows * ldzs);
  __shared__ int s_cnt[2], s_m[2], s_fail;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int r0 = blockIdx.x * rows, nr = min(rows, n - r0);
  for (int i = tid; i < n; i += TQL_NT) {
    d[i] = work[i];
    e[i] = work[n + i];
  }
  for (int idx = tid; idx < rows * ldzs; idx += TQL_NT) {
    const int r = idx / ldzs, c = idx % ldzs;
    Zs[idx] = (r0 + r == c) ? 1.0 : 0.0;
  }
  if (tid == 0) s_fail = 0;
  __syncthreads();
  // producer state (warp 0, the same in every lane): current l and its iterations
  int l = 0, iter = 0;
  // computes the next chase into buffer b: s_cnt[b] rotations ending at
  // column s_m[b], or s_cnt[b] = -1 once every eigenvalue has converged
  auto produce = [&](int b) {
    double* cb = cs + 2 * (size_t)n * b;
    double* sb = cb + n;
    int cnt = -1, m = l;
    while (l < n) {
      // block end: first m >= l with a negligible e[m] (32 candidates at a time)
      m = n - 1;
      for (int base = l; base < n - 1; base += 32) {
        const int mi = base + lane;
        bool small = false;
        if (mi < n - 1) small = fabs(e[mi]) <= 2.220446049250313e-16 * (fabs(d[mi]) + fabs(d[mi + 1]));
        const unsigned bal = __ballot_sync(0xffffffffu, small);
        if (bal) {
          m = base + __ffs(bal) - 1;
          break;
        }
      }
      if (m == l) {
        ++l;
        iter = 0;
        continue;
      }
      if (iter >= 60) {  // no convergence for this eigenvalue: leave it as is
        if (lane == 0) s_fail = 1;
        ++l;
        iter = 0;
        continue;
      }
      if (lane == 0) {
        double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
        double r = hypot(g, 1.0);
        g = d[m] - d[l] + e[l] / (g + (g >= 0 ? fabs(r) : -fabs(r)));
        double s = 1.0, c = 1.0, p = 0.0;
        int nrot = 0;
        bool early = false;
        for (int i = m - 1; i >= l; --i) {
          const double f = s * e[i];
          const double bb = c * e[i];
          double ri;
          if (sqrt_rsqrt_gs(fma(f, f, g * g), &r, &ri)) {
            s = f * ri;
            c = g * ri;
          } else {
            r = hypot(f, g);
            if (r == 0.0) {
              e[i + 1] = 0.0;
              d[i + 1] -= p;
              e[m] = 0.0;
              early = true;
              break;
            }
            s = f / r;
            c = g / r;
          }
          e[i + 1] = r;
          g = d[i + 1] - p;
          r = (d[i] - g) * s + 2.0 * c * bb;
          p = s * r;
          d[i + 1] = g + p;
          g = c * r - bb;
          cb[nrot] = c;
          sb[nrot] = s;
          ++nrot;
        }
        if (!early) {
          d[l] -= p;
          e[l] = g;
          e[m] = 0.0;
        }
        cnt = nrot;
      }
      cnt = __shfl_sync(0xffffffffu, cnt, 0);
      ++iter;
      break;
    }
    if (l >= n) cnt = -1;
    if (lane == 0) {
      s_cnt[b] = cnt;
      s_m[b] = m;
    }
    __syncwarp();
  };
  if (warp == 0) produce(0);
  __syncthreads();
  for (int q = 0;; ++q) {
    const int b = q & 1;
    const int cnt = s_cnt[b];
    if (cnt < 0) break;
    if (warp == 0) {
      produce(b ^ 1);
    } else if (lane < nr && cnt > 0) {
      // rotation t acts on columns (i, i+1), i = m-1-t; the new column i
      // is the next rotation's column i+1, carried in a register
      const double* cb = cs + 2 * (size_t)n * b;
      const double* sb = cb + n;
      const int m = s_m[b];
      double* z = Zs + (size_t)lane * ldzs;
      double carry = z[m];
      for (int t = 0; t < cnt; ++t) {
        const int i = m - 1 - t;
        const double c = cb[t], s = sb[t], zi = z[i];
        z[i + 1] = fma(c, carry, s * zi);
        carry = fma(-s, carry, c * zi);
      }
      z[m - cnt] = carry;
    }
    __syncthreads();
  }
  // rank by decreasing eigenvalue (ties and NaN by index)
  for (int i = tid; i < n; i += TQL_NT) {
    const double di = isnan(d[i]) ? -INFINITY : d[i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double dj = isnan(d[j]) ? -INFINITY : d[j];
      rank += (dj > di) || (dj == di && j < i);
    }
    perm[rank] = i;
  }
  __syncthreads();
  for (int idx = tid; idx < nr * n; idx += TQL_NT) {
    const int r = idx % nr, c = idx / nr;
    Z[(size_t)c * ldz + r0 + r] = Zs[(size_t)r * ldzs + perm[c]];
  }
  if (blockIdx.x == 0) {
    for (int i = tid; i < n; i += TQL_NT) theta[i] = d[perm[i]];
    if (tid == 0 && status) *status = s_fail;
  }
}

// Z[:, c] <- H_0 H_1 ... H_{n-3} Z[:, c], one warp per column, the column in
// shared memory; v_k = A[k+1:, k], tau_k = work[2n + k].
__global__ void __launch_bounds__(32 * BACK_WARPS) k_eig_back(int n, const double* A, int lda,
                                                              const double* work, double* Z, int ldz) {
  extern __shared__ double sm_back[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int col = blockIdx.x * BACK_WARPS + warp;
  if (col >= n) return;
  const double* tau = work + 2 * n;
  double* z = sm_back + (size_t)warp * n;
  double* zg = Z + (size_t)col * ldz;
  for (int i = lane; i < n; i += 32) z[i] = zg[i];
  __syncwarp();
  for (int k = n - 3; k >= 0; --k) {
    const double tk = tau[k];
    if (tk == 0.0) continue;
    const double* v = A + (size_t)k * lda + k + 1;
    const int len = n - k - 1;
    double part = 0.0;
    for (int i = lane; i < len; i += 32) part = fma(v[i], z[k + 1 + i], part);
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    const double w = tk * part;
    for (int i = lane; i < len; i += 32) z[k + 1 + i] = fma(-w, v[i], z[k + 1 + i]);
    __syncwarp();
  }
  for (int i = lane; i < n; i += 32) zg[i] = z[i];
}

// resid[i] = || B (nb x nb upper, col-major) * Z[row0:row0+nb, i] ||, i < k
__global__ void k_ritz_resid(int k, int nb, const double* B, const double* Z, int ldz, int row0,
                             double* resid) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k) return;
  double s2 = 0.0;
  for (int r = 0; r < nb; ++r) {
    double s = 0.0;
    for (int c = 0; c < nb; ++c) s += B[c * nb + r] * Z[(size_t)i * ldz + row0 + c];
    s2 += s * s;
  }
  resid[i] = sqrt(s2);
}

// T[r0:r0+nb, c0:c0+nb] = S (and optionally the transpose block), S col-major nb x nb
__global__ void k_set_block(double* T, int ldt, int r0, int c0, int nb, const double* S, int lds,
                            int symmetrize, int also_transpose) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nb * nb) return;
  const int i = e % nb, j = e / nb;
  double v = S[(size_t)j * lds + i];
  if (symmetrize) v = 0.5 * (v + S[(size_t)i * lds + j]);
  T[(size_t)(c0 + j) * ldt + r0 + i] = v;
  if (also_transpose) T[(size_t)(r0 + i) * ldt + c0 + j] = v;
}


// Pseudo-random values in [-1, 1) from a counter-based hash (splitmix64 of
// seed, column and row); fills columns with flags[c] != 0 (flags NULL = all).
__device__ __forceinline__ double hash_uniform(unsigned long long seed, int col, int row) {
  unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(col + 1) +
                         0xD1B54A32D192ED03ull * (unsigned long long)(row + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

__global__ void k_fill_random(int nx, int nb, double* W, int ldw, const int* flags,
                              unsigned long long seed) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (p >= nx || c >= nb) return;
  if (flags && !flags[c]) return;
  W[(size_t)c * ldw + p] = hash_uniform(seed, c, p);
}

__global__ void k_copy_cols(int nx, int nb, const double* S, int lds, double* D, int ldd) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (p >= nx || c >= nb) return;
  D[(size_t)c * ldd + p] = S[(size_t)c * lds + p];
}

// y[j] = scale * x[j] * f(lambda_j): mode 0 -> d = lam/(lam+1); mode 1 -> (1+lam)^{-1/2} - 1
__global__ void k_diag_scale(int k, int ncols, const double* lam, double lam_scale, int mode,
                             double* C, int ldc) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= k * ncols) return;
  const int i = e % k, j = e / k;
  const double l = lam[i] * lam_scale;
  const double f = (mode == 0) ? l / (l + 1.0) : 1.0 / sqrt(1.0 + l) - 1.0;
  C[(size_t)j * ldc + i] *= f;
}

// var[i] = pdiag[i] - sum_j d_j G[node_i, j]^2
__global__ void k_variance(int np, const int* nodes, const double* pdiag, int k, const double* lam,
                           double lam_scale, const double* G, int ldg, double* var) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const int node = nodes[i];
  double s = 0.0;
  for (int j = 0; j < k; ++j) {
    const double l = lam[j] * lam_scale;
    const double g = G[(size_t)j * ldg + node];
    s += (l / (l + 1.0)) * g * g;
  }
  var[i] = pdiag[i] - s;
}

// E[:, i] = e_{nodes[i]} (columns i0..i0+nc)
__global__ void k_unit_cols(int nx, int nc, const int* nodes, int i0, double* E, int lde) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (p >= nx || c >= nc) return;
  E[(size_t)c * lde + p] = (nodes[i0 + c] == p) ? 1.0 : 0.0;
}

// out[i] = sum_p X[i][p]^2 for columns i < nc (one block per column)
__global__ void k_col_norm2(int nx, int nc, const double* X, int ldx, double* out) {
  __shared__ double s_red[32];
  const int c = blockIdx.x;
  if (c >= nc) return;
  double s = 0.0;
  for (int p = threadIdx.x; p < nx; p += blockDim.x) {
    const double x = X[(size_t)c * ldx + p];
    s += x * x;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_red[w];
    out[c] = t;
  }
}

__global__ void k_axpby(size_t n, double a, const double* x, double b, double* y) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = a * x[i] + (b == 0.0 ? 0.0 : b * y[i]);
}

// Y[:, j] += m (broadcast a vector into every column)
__global__ void k_add_vec_cols(int nx, int nc, const double* m, double* Y, int ldy) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (p >= nx || c >= nc) return;
  Y[(size_t)c * ldy + p] += m[p];
}

// ---------------------------------------------------------------- block Gram-Schmidt
// Rank-revealing orthonormalisation of the s <= 16 columns of B (nx x s, ld
// ldb) in place, one CTA per matrix (blockIdx.x selects B + b*strideB and
// R + b*strideR): column c is orthogonalised against columns 0..c-1 by
// classical Gram-Schmidt twice (a third pass when the norm fell below 1/10),
// then normalised. A column whose remaining norm is at most drop_tol times
// its norm on entry lies numerically in the span of the previous ones: it is
// set to zero and its diagonal entry of R is 0. Output: B = Q R with R
// (s x s, col-major) upper triangular; zero columns of Q have zero rows in R.
#define GS_NT 512
#define GS_MAXC 64
#define GS_MC_MAXG 64   // CTAs of the cooperative variant
#define GS_MC_ROWS 1024  // rows per CTA at least
__global__ void __launch_bounds__(GS_NT) k_block_gs(int nx, int s, double* B, size_t strideB, int ldb,
                                                     double* R, size_t strideR, double drop_tol,
                                                     const double* ref_norm2, int* ndrop) {
  __shared__ double s_part[GS_NT / 32][17];
  __shared__ double s_tot[17];
  __shared__ double s_h[GS_MAXC];   // projections of the current column on the previous ones
  __shared__ double s_rc[GS_MAXC];  // their sum over the passes (column c of R)
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  double* Bb = B + blockIdx.x * strideB;
  double* Rb = R + blockIdx.x * strideR;
  // reduce acc[0..16] over the CTA into s_tot
  auto reduce17 = [&](double* acc) {
#pragma unroll
    for (int i = 0; i < 17; ++i) {
      double v = acc[i];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) s_part[wid][i] = v;
    }
    __syncthreads();
    if (tid < 17) {
      double t = 0.0;
      for (int w = 0; w < GS_NT / 32; ++w) t += s_part[w][tid];
      s_tot[tid] = t;
    }
    __syncthreads();
  };
  int dropped = 0;
  for (int c = 0; c < s; ++c) {
    double* w = Bb + (size_t)c * ldb;
    if (tid < GS_MAXC) s_rc[tid] = 0.0;
    double n0 = 0.0, nprev = 0.0, ncur = 0.0;
    for (int pass = 0; pass < 4; ++pass) {
      // h = Q[:, :c]^T w in chunks of 16 previous columns, |w|^2 with the first
      const int nchunk = c > 0 ? (c + 15) / 16 : 1;
      for (int q = 0; q < nchunk; ++q) {
        const int i0 = q * 16, ni = min(16, c - i0);
        double acc[17];
#pragma unroll
        for (int i = 0; i < 17; ++i) acc[i] = 0.0;
        for (int p = tid; p < nx; p += GS_NT) {
          const double wp = w[p];
#pragma unroll
          for (int i = 0; i < 16; ++i)
            if (i < ni) acc[i] += Bb[(size_t)(i0 + i) * ldb + p] * wp;
          if (q == 0) acc[16] += wp * wp;
        }
        reduce17(acc);
        if (tid < ni) s_h[i0 + tid] = s_tot[tid];
        if (q == 0) ncur = s_tot[16];
      }
      if (pass == 0) n0 = ncur;
      // stop after two projections, or a third one if the norm collapsed
      const bool more = (c > 0) && (pass < 2 || (pass == 2 && ncur < 1e-2 * nprev));
      if (!more) break;
      __syncthreads();  // every s_h entry written
      if (tid < c) s_rc[tid] += s_h[tid];
      for (int p = tid; p < nx; p += GS_NT) {
        double v = w[p];
        for (int i = 0; i < c; ++i) v -= s_h[i] * Bb[(size_t)i * ldb + p];
        w[p] = v;
      }
      __syncthreads();
      nprev = ncur;
    }
    const double nrm = sqrt(ncur);
    // dependent: what is left is at most drop_tol of the column's norm on
    // entry, or of its norm before the caller's earlier projections
    const double nref = ref_norm2 ? fmax(n0, ref_norm2[(size_t)blockIdx.x * s + c]) : n0;
    const bool drop = !(nrm > drop_tol * sqrt(nref)) || !(nrm > 0.0);
    const double scale = drop ? 0.0 : 1.0 / nrm;
    for (int p = tid; p < nx; p += GS_NT) w[p] *= scale;
    __syncthreads();  // s_rc complete
    if (tid == 0) {
      for (int i = 0; i < s; ++i) Rb[(size_t)c * s + i] = (i < c) ? s_rc[i] : (i == c ? (drop ? 0.0 : nrm) : 0.0);
    }
    dropped += drop ? 1 : 0;
    __syncthreads();
  }
  if (tid == 0 && ndrop) ndrop[blockIdx.x] = dropped;
}

// The same rank-revealing block CGS2 of one matrix spread over the CTAs of
// a cooperative grid: CTA g owns rows [g rows, (g+1) rows) of every column,
// so the only cross-CTA data are the projections and norms, reduced through
// per-CTA partial sums in `part` ([2][G][GS_MAXC + 1], the two halves used by
// alternate passes so one grid barrier per pass suffices). Every CTA adds the
// partials in the same order and takes identical decisions.
__global__ void __launch_bounds__(GS_NT) k_block_gs_mc(int nx, int s, double* B, int ldb, double* R,
                                                        double drop_tol, const double* ref_norm2, int* ndrop,
                                                        double* part) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  __shared__ double s_part[GS_NT / 32][17];
  __shared__ double s_tot[17];
  __shared__ double s_h[GS_MAXC], s_rc[GS_MAXC];
  __shared__ double s_n;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int G = gridDim.x, g = blockIdx.x;
  const int rows = (nx + G - 1) / G, p0 = min(nx, g * rows), p1 = min(nx, p0 + rows);
  constexpr int PW = GS_MAXC + 1;
  auto reduce17 = [&](double* acc) {
#pragma unroll
    for (int i = 0; i < 17; ++i) {
      double v = acc[i];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) s_part[wid][i] = v;
    }
    __syncthreads();
    if (tid < 17) {
      double t = 0.0;
      for (int w = 0; w < GS_NT / 32; ++w) t += s_part[w][tid];
      s_tot[tid] = t;
    }
    __syncthreads();
  };
  int dropped = 0, buf = 0;
  for (int c = 0; c < s; ++c) {
    double* w = B + (size_t)c * ldb;
    if (tid < GS_MAXC) s_rc[tid] = 0.0;
    double n0 = 0.0, nprev = 0.0, ncur = 0.0;
    for (int pass = 0; pass < 4; ++pass) {
      double* pb = part + ((size_t)buf * G + g) * PW;
      const int nchunk = c > 0 ? (c + 15) / 16 : 1;
      for (int q = 0; q < nchunk; ++q) {
        const int i0 = q * 16, ni = min(16, c - i0);
        double acc[17];
#pragma unroll
        for (int i = 0; i < 17; ++i) acc[i] = 0.0;
        for (int p = p0 + tid; p < p1; p += GS_NT) {
          const double wp = w[p];
#pragma unroll
          for (int i = 0; i < 16; ++i)
            if (i < ni) acc[i] += B[(size_t)(i0 + i) * ldb + p] * wp;
          if (q == 0) acc[16] += wp * wp;
        }
        reduce17(acc);
        if (tid < ni) pb[i0 + tid] = s_tot[tid];
        if (q == 0 && tid == 0) pb[GS_MAXC] = s_tot[16];
      }
      grid.sync();
      const double* pa = part + (size_t)buf * G * PW;
      if (tid < c) {
        double t = 0.0;
        for (int k = 0; k < G; ++k) t += pa[(size_t)k * PW + tid];
        s_h[tid] = t;
      }
      if (tid == GS_NT - 1) {
        double t = 0.0;
        for (int k = 0; k < G; ++k) t += pa[(size_t)k * PW + GS_MAXC];
        s_n = t;
      }
      __syncthreads();
      ncur = s_n;
      buf ^= 1;
      if (pass == 0) n0 = ncur;
      const bool more = (c > 0) && (pass < 2 || (pass == 2 && ncur < 1e-2 * nprev));
      if (!more) break;
      if (tid < c) s_rc[tid] += s_h[tid];
      for (int p = p0 + tid; p < p1; p += GS_NT) {
        double v = w[p];
        for (int i = 0; i < c; ++i) v -= s_h[i] * B[(size_t)i * ldb + p];
        w[p] = v;
      }
      nprev = ncur;
    }
    const double nrm = sqrt(ncur);
    const double nref = ref_norm2 ? fmax(n0, ref_norm2[c]) : n0;
    const bool drop = !(nrm > drop_tol * sqrt(nref)) || !(nrm > 0.0);
    const double scale = drop ? 0.0 : 1.0 / nrm;
    for (int p = p0 + tid; p < p1; p += GS_NT) w[p] *= scale;
    __syncthreads();  // s_rc complete
    if (g == 0 && tid == 0)
      for (int i = 0; i < s; ++i) R[(size_t)c * s + i] = (i < c) ? s_rc[i] : (i == c ? (drop ? 0.0 : nrm) : 0.0);
    dropped += drop ? 1 : 0;
    __syncthreads();
  }
  if (g == 0 && tid == 0 && ndrop) *ndrop = dropped;
}

size_t block_gs_scratch_doubles() { return (size_t)2 * GS_MC_MAXG * (GS_MAXC + 1); }

// --------------------------------------------------------------------------- host wrappers

cudaError_t gemm_tn(cudaStream_t s, int nx, int m, int nb, const double* A, int lda, const double* B,
                    int ldb, double* C, int ldc, double alpha, double beta, double* part, size_t part_cap) {
  int nchunk = std::min(128, std::max(1, (nx + 4095) / 4096));
  while ((size_t)nchunk * m * 16 > part_cap && nchunk > 1) nchunk /= 2;
  const int rows = ((nx + nchunk - 1) / nchunk + TN_TR - 1) / TN_TR * TN_TR;
  nchunk = (nx + rows - 1) / rows;
  for (int j0 = 0; j0 < nb; j0 += 16) {
    const int nbl = std::min(16, nb - j0);
    dim3 grid((m + TN_TI - 1) / TN_TI, nchunk);
    note_launch();
    k_gemm_tn<<<grid, 256, 0, s>>>(nx, m, nbl, A, lda, B + (size_t)j0 * ldb, ldb, part, rows);
    note_launch();
    k_reduce_parts<<<(m * nbl + 255) / 256, 256, 0, s>>>(m, nbl, nchunk, part, C + (size_t)j0 * ldc,
                                                         ldc, alpha, beta);
  }
  return cudaGetLastError();
}

cudaError_t gemm_nn(cudaStream_t s, int nx, int m, int nc, double alpha, const double* A, int lda,
                    const double* M, int ldm, double beta, double* Y, int ldy) {
  if (m == 0) {
    if (beta == 1.0) return cudaSuccess;
  }
  dim3 grid((nx + 255) / 256, (nc + 15) / 16);
  note_launch();
  k_gemm_nn<<<grid, 256, 0, s>>>(nx, m, nc, alpha, A, lda, M, ldm, beta, Y, ldy);
  return cudaGetLastError();
}

cudaError_t eig_sym(cudaStream_t s, int n, double* A, int lda, double* Z, int ldz, double* theta,
                    double* work, int* status) {
  if (n < 1 || n > 1024) return cudaErrorInvalidValue;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  // one value from every caller: the device's opt-in maximum less the static part
  cudaFuncAttributes fa_tql, fa_back;
  cudaError_t e = cudaFuncGetAttributes(&fa_tql, k_tql);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa_back, k_eig_back);
  if (e != cudaSuccess) return e;
  const size_t cap_tql = (size_t)optin - fa_tql.sharedSizeBytes;
  const size_t cap_back = (size_t)optin - fa_back.sharedSizeBytes;
  // rows of Z per QL CTA: at most TQL_ROWS, fewer when n is large
  const size_t fixed = 6 * (size_t)n * sizeof(double) + (size_t)n * sizeof(int);
  const size_t per_row = (size_t)(n + 1) * sizeof(double);
  if (fixed + per_row > cap_tql) return cudaErrorInvalidValue;
  const int rows = (int)std::min<size_t>(TQL_ROWS, (cap_tql - fixed) / per_row);
  const size_t smem_tql = fixed + rows * per_row;
  const size_t smem_back = (size_t)BACK_WARPS * n * sizeof(double);
  if (smem_back > cap_back) return cudaErrorInvalidValue;
  e = cudaFuncSetAttribute(k_tql, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap_tql);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_eig_back, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap_back);
  if (e != cudaSuccess) return e;
  note_launch();
  k_tridiag<<<1, EIG_NT, 0, s>>>(n, A, lda, work);
  note_launch();
  k_tql<<<(n + rows - 1) / rows, TQL_NT, smem_tql, s>>>(n, work, Z, ldz, theta, status, rows);
  note_launch();
  k_eig_back<<<(n + BACK_WARPS - 1) / BACK_WARPS, 32 * BACK_WARPS, smem_back, s>>>(n, A, lda, work, Z, ldz);
  return cudaGetLastError();
}

cudaError_t ritz_resid(cudaStream_t s, int k, int nb, const double* B, const double* Z, int ldz, int row0,
                       double* resid) {
  note_launch();
  k_ritz_resid<<<(k + 127) / 128, 128, 0, s>>>(k, nb, B, Z, ldz, row0, resid);
  return cudaGetLastError();
}

cudaError_t set_block(cudaStream_t s, double* T, int ldt, int r0, int c0, int nb, const double* S, int lds,
                      bool symmetrize, bool also_transpose) {
  note_launch();
  k_set_block<<<(nb * nb + 255) / 256, 256, 0, s>>>(T, ldt, r0, c0, nb, S, lds, symmetrize ? 1 : 0,
                                                     also_transpose ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t fill_random(cudaStream_t s, int nx, int nb, double* W, int ldw, const int* flags,
                        unsigned long long seed) {
  dim3 grid((nx + 255) / 256, nb);
  note_launch();
  k_fill_random<<<grid, 256, 0, s>>>(nx, nb, W, ldw, flags, seed);
  return cudaGetLastError();
}

cudaError_t copy_cols(cudaStream_t s, int nx, int nb, const double* S, int lds, double* D, int ldd) {
  dim3 grid((nx + 255) / 256, nb);
  note_launch();
  k_copy_cols<<<grid, 256, 0, s>>>(nx, nb, S, lds, D, ldd);
  return cudaGetLastError();
}

cudaError_t diag_scale(cudaStream_t s, int k, int ncols, const double* lam, double lam_scale, int mode,
                       double* C, int ldc) {
  note_launch();
  k_diag_scale<<<(k * ncols + 255) / 256, 256, 0, s>>>(k, ncols, lam, lam_scale, mode, C, ldc);
  return cudaGetLastError();
}

cudaError_t variance(cudaStream_t s, int np, const int* nodes, const double* pdiag, int k, const double* lam,
                     double lam_scale, const double* G, int ldg, double* var) {
  note_launch();
  k_variance<<<(np + 127) / 128, 128, 0, s>>>(np, nodes, pdiag, k, lam, lam_scale, G, ldg, var);
  return cudaGetLastError();
}

cudaError_t unit_cols(cudaStream_t s, int nx, int nc, const int* nodes, int i0, double* E, int lde) {
  dim3 grid((nx + 255) / 256, nc);
  note_launch();
  k_unit_cols<<<grid, 256, 0, s>>>(nx, nc, nodes, i0, E, lde);
  return cudaGetLastError();
}

cudaError_t col_norm2(cudaStream_t s, int nx, int nc, const double* X, int ldx, double* out) {
  note_launch();
  k_col_norm2<<<nc, 256, 0, s>>>(nx, nc, X, ldx, out);
  return cudaGetLastError();
}

cudaError_t axpby(cudaStream_t s, size_t n, double a, const double* x, double b, double* y) {
  note_launch();
  k_axpby<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, a, x, b, y);
  return cudaGetLastError();
}

cudaError_t add_vec_cols(cudaStream_t s, int nx, int nc, const double* m, double* Y, int ldy) {
  dim3 grid((nx + 255) / 256, nc);
  note_launch();
  k_add_vec_cols<<<grid, 256, 0, s>>>(nx, nc, m, Y, ldy);
  return cudaGetLastError();
}

cudaError_t block_gs(cudaStream_t s, int batch, int nx, int ncols, double* B, size_t strideB, int ldb, double* R,
                     size_t strideR, double drop_tol, int* ndrop, const double* ref_norm2, double* coop_scratch) {
  if (ncols > GS_MAXC) return cudaErrorInvalidValue;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  if (batch == 1 && coop_scratch && nx >= 2 * GS_MC_ROWS && cs == cudaStreamCaptureStatusNone) {
    // one matrix: spread over a cooperative grid (co-residency checked by the launch)
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int G = std::max(1, std::min({GS_MC_MAXG, sms, nx / GS_MC_ROWS}));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G);
    cfg.blockDim = dim3(GS_NT);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    note_launch();
    return cudaLaunchKernelEx(&cfg, k_block_gs_mc, nx, ncols, B, ldb, R, drop_tol, ref_norm2, ndrop, coop_scratch);
  }
  note_launch();
  k_block_gs<<<batch, GS_NT, 0, s>>>(nx, ncols, B, strideB, ldb, R, strideR, drop_tol, ref_norm2, ndrop);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Diagonal of the prior covariance R^-2, R = I + alpha L0, with L0 the
// constant-coefficient finite-difference Laplacian on the n^dim interior
// grid of the unit square/cube (zero Dirichlet data). L0 is diagonalised by
// the orthonormal sine transform: S_ik = sqrt(2/(n+1)) sin(pi i k/(n+1)) per
// axis, eigenvalues mu_k = (4/h^2) sin^2(pi k h/2), h = 1/(n+1), summed over
// the axes. Hence diag_i = sum_k w(k) prod_d S_{i_d k_d}^2 with
// w(k) = (1 + alpha sum_d mu_{k_d})^-2, evaluated by contracting one axis at
// a time (dim n^(dim+1) multiply-adds).
__global__ void k_dst_sq(int n, double* A) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  const int i = e / n, k = e % n;
  const double s = sinpi((double)((i + 1) * (k + 1)) / (double)(n + 1));
  A[e] = 2.0 / (double)(n + 1) * s * s;
}

__global__ void k_dst_weight(int dim, int n, double alpha, double* W) {
  const int total = dim == 2 ? n * n : n * n * n;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const double h = 1.0 / (double)(n + 1);
  int k[3] = {e % n, (e / n) % n, dim == 3 ? e / (n * n) : 0};
  double mu = 0.0;
  for (int d = 0; d < dim; ++d) {
    const double sv = sinpi(0.5 * (double)(k[d] + 1) * h);
    mu += 4.0 / (h * h) * sv * sv;
  }
  const double r = 1.0 + alpha * mu;
  W[e] = 1.0 / (r * r);
}

// out(.., i_axis, ..) = sum_k A(i_axis, k) in(.., k, ..); axis 0 is the fastest index.
__global__ void k_dst_contract(int dim, int n, int axis, const double* A, const double* in, double* out) {
  const int total = dim == 2 ? n * n : n * n * n;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const int stride = axis == 0 ? 1 : (axis == 1 ? n : n * n);
  const int ia = (e / stride) % n;
  const int base = e - ia * stride;
  double acc = 0.0;
  for (int k = 0; k < n; ++k) acc += A[ia * n + k] * in[base + k * stride];
  out[e] = acc;
}

cudaError_t prior_diag_dst(cudaStream_t s, int dim, int n, double alpha, double* out, double* work) {
  const int total = dim == 2 ? n * n : n * n * n;
  double* A = work;
  double* W = work + (size_t)n * n;
  double* T = W + total;
  note_launch(2);
  k_dst_sq<<<(n * n + 255) / 256, 256, 0, s>>>(n, A);
  k_dst_weight<<<(total + 255) / 256, 256, 0, s>>>(dim, n, alpha, W);
  const double* src = W;
  for (int axis = 0; axis < dim; ++axis) {
    double* dst = (axis == dim - 1) ? out : (src == W ? T : W);
    note_launch();
    k_dst_contract<<<(total + 255) / 256, 256, 0, s>>>(dim, n, axis, A, src, dst);
    src = dst;
  }
  return cudaGetLastError();
}

__global__ void k_fill_const(size_t n, double v, double* out) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = v;
}

cudaError_t prior_diag(cudaStream_t s, const lrp_problem_desc& d, double* out, double* work) {
  if (d.prior_kind == LRP_PRIOR_IDENTITY) {
    const size_t total = d.dim == 2 ? (size_t)d.n * d.n : (size_t)d.n * d.n * d.n;
    note_launch();
    k_fill_const<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(total, d.prior_gamma, out);
    return cudaGetLastError();
  }
  return prior_diag_dst(s, d.dim, d.n, d.prior_alpha, out, work);
}

// D[0:m, 0:n] += S[0:m, 0:n] (column-major, leading dimensions lds, ldd)
__global__ void k_add_block(int m, int n, const double* S, int lds, double* D, int ldd) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * n) return;
  const int i = e % m, j = e / m;
  D[(size_t)j * ldd + i] += S[(size_t)j * lds + i];
}

cudaError_t add_block(cudaStream_t s, int m, int n, const double* S, int lds, double* D, int ldd) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  note_launch();
  k_add_block<<<(m * n + 255) / 256, 256, 0, s>>>(m, n, S, lds, D, ldd);
  return cudaGetLastError();
}

// T[r0:r0+m, c0:c0+n] = S (m x n, ld lds) and, if also_transpose, the
// mirrored block T[c0:c0+n, r0:r0+m] = S^T.
__global__ void k_set_rect(double* T, int ldt, int r0, int c0, int m, int n, const double* S, int lds,
                           int also_transpose) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * n) return;
  const int i = e % m, j = e / m;
  const double v = S[(size_t)j * lds + i];
  T[(size_t)(c0 + j) * ldt + r0 + i] = v;
  if (also_transpose) T[(size_t)(r0 + i) * ldt + c0 + j] = v;
}

cudaError_t set_rect(cudaStream_t s, double* T, int ldt, int r0, int c0, int m, int n, const double* S, int lds,
                     bool also_transpose) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  note_launch();
  k_set_rect<<<(m * n + 255) / 256, 256, 0, s>>>(T, ldt, r0, c0, m, n, S, lds, also_transpose ? 1 : 0);
  return cudaGetLastError();
}

// out[i] = v[idx[i]]
__global__ void k_gather(int n, const int* idx, const double* v, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = v[idx[i]];
}

cudaError_t gather(cudaStream_t s, int n, const int* idx, const double* v, double* out) {
  if (n <= 0) return cudaSuccess;
  note_launch();
  k_gather<<<(n + 255) / 256, 256, 0, s>>>(n, idx, v, out);
  return cudaGetLastError();
}

}  // namespace lrp
