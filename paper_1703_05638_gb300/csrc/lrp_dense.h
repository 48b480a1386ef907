// Host wrappers of the FP64 dense kernels (lrp_dense.cu). All matrices are
// column-major device arrays; every call is asynchronous on stream s.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "lrp.h"

namespace lrp {

// C (m x nb, ld ldc) = alpha * A^T B + beta * C; A: nx x m (lda), B: nx x nb (ldb).
// part: scratch of part_cap doubles (>= m*16).
cudaError_t gemm_tn(cudaStream_t s, int nx, int m, int nb, const double* A, int lda, const double* B,
                    int ldb, double* C, int ldc, double alpha, double beta, double* part, size_t part_cap);
// Y (nx x nc) = beta Y + alpha A M; A: nx x m, M: m x nc. Y may alias A only if nc <= 16.
cudaError_t gemm_nn(cudaStream_t s, int nx, int m, int nc, double alpha, const double* A, int lda,
                    const double* M, int ldm, double beta, double* Y, int ldy);
// theta decreasing, Z eigenvectors; A destroyed; work >= 6n doubles; n <= 1024.
cudaError_t eig_sym(cudaStream_t s, int n, double* A, int lda, double* Z, int ldz, double* theta,
                    double* work, int* status);
// Rank-revealing block CGS2 of `batch` matrices (nx x ncols, ncols <= 64),
// in place; R (ncols x ncols per matrix) upper triangular; columns numerically
// dependent on the previous ones (relative remainder <= drop_tol) become zero
// with a zero diagonal in R; ndrop[b] (may be NULL) counts them.
// ref_norm2 (may be NULL): squared column norms before the caller's earlier
// projections ([batch][ncols]); a column is then dependent if its remainder
// is at most drop_tol of the larger of that norm and its norm on entry.
// coop_scratch (may be NULL; block_gs_scratch_doubles() doubles): with one
// matrix, the work is spread over a cooperative grid of CTAs.
cudaError_t block_gs(cudaStream_t s, int batch, int nx, int ncols, double* B, size_t strideB, int ldb, double* R,
                     size_t strideR, double drop_tol, int* ndrop, const double* ref_norm2 = nullptr,
                     double* coop_scratch = nullptr);
size_t block_gs_scratch_doubles();
cudaError_t ritz_resid(cudaStream_t s, int k, int nb, const double* B, const double* Z, int ldz, int row0,
                       double* resid);
cudaError_t set_block(cudaStream_t s, double* T, int ldt, int r0, int c0, int nb, const double* S, int lds,
                      bool symmetrize, bool also_transpose);
cudaError_t fill_random(cudaStream_t s, int nx, int nb, double* W, int ldw, const int* flags,
                        unsigned long long seed);
cudaError_t copy_cols(cudaStream_t s, int nx, int nb, const double* S, int lds, double* D, int ldd);
cudaError_t diag_scale(cudaStream_t s, int k, int ncols, const double* lam, double lam_scale, int mode,
                       double* C, int ldc);
cudaError_t variance(cudaStream_t s, int np, const int* nodes, const double* pdiag, int k, const double* lam,
                     double lam_scale, const double* G, int ldg, double* var);
cudaError_t unit_cols(cudaStream_t s, int nx, int nc, const int* nodes, int i0, double* E, int lde);
cudaError_t col_norm2(cudaStream_t s, int nx, int nc, const double* X, int ldx, double* out);
cudaError_t axpby(cudaStream_t s, size_t n, double a, const double* x, double b, double* y);
cudaError_t add_vec_cols(cudaStream_t s, int nx, int nc, const double* m, double* Y, int ldy);

// T[r0:r0+m, c0:c0+n] = S (m x n, ld lds), and the mirrored block if also_transpose.
cudaError_t set_rect(cudaStream_t s, double* T, int ldt, int r0, int c0, int m, int n, const double* S, int lds,
                     bool also_transpose);
// D[0:m, 0:n] += S[0:m, 0:n] (column-major).
cudaError_t add_block(cudaStream_t s, int m, int n, const double* S, int lds, double* D, int ldd);
// out[i] = v[idx[i]], i < n.
cudaError_t gather(cudaStream_t s, int n, const int* idx, const double* v, double* out);
// Diagonal of (I + alpha L0)^-2 on the n^dim grid (constant-coefficient
// Laplacian, zero Dirichlet data) by the sine transform; work >= n^2 + 2 n^dim.
cudaError_t prior_diag_dst(cudaStream_t s, int dim, int n, double alpha, double* out, double* work);
// (Gamma_prior)_ii at every node for either prior kind (work as prior_diag_dst)
cudaError_t prior_diag(cudaStream_t s, const lrp_problem_desc& d, double* out, double* work);

}  // namespace lrp
