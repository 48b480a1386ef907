// Low-rank-in-time trajectory factors (Sec. 3: Y = [y_1 .. y_nt] ~ W V^T with
// small rank; Sec. 4: rank control of factored sums by skinny QR and
// truncated SVD).
//
// The forward sweep runs in chunks of s steps; each chunk's states land in a
// buffer B (nx x s per column). Streaming recompression per column, with the
// current factors Y_old ~ Qw diag(sig) V^T (Qw, V orthonormal columns):
//   C = Qw^T B, B' = B - Qw C (twice: CGS2), B' = Q2 R2 (rank-revealing
//   block Gram-Schmidt), core = [[diag(sig), C], [0, R2]] = U S Zt (SVD),
//   keep the r' leading triplets whose discarded Frobenius tail is at most
//   (tol / K) ||core||_F (K = number of chunks; by the triangle inequality the
//   accumulated error is at most tol ||Y||_F), capped at time_rank_max,
//   Qw <- [Qw Q2] U[:, :r'], V <- blockdiag(V, I_s) Zt^T[:, :r'], sig <- S[:r'].
// The SVD of the small core is one-sided Jacobi in shared memory (k_core_svd),
// which works on the core itself (no squaring) and resolves small singular
// values to high relative accuracy.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "lrp_dense.h"
#include "lrp_internal.h"

namespace lrp {


// SVD of every column's core K = [[diag(sig), C], [0, R]] (m x m, m = r + s;
// the factors' singular values, the chunk's coefficients on them and the
// chunk's own triangular factor) by one-sided Jacobi (Hestenes): the columns
// of A = K V are made pairwise orthogonal by plane rotations, applied to V as
// well, in round-robin order (each round rotates m/2 disjoint column pairs in
// parallel, one warp per pair), until a sweep rotates nothing. Then
// sigma_j = |A e_j|, u_j = A e_j / sigma_j, v_j = V e_j. One CTA per column;
// A and V live in shared memory. Output, sorted by decreasing sigma:
// th[i] = sigma_i, Z = [U | V] (two m x m column-major blocks, ld m).
__global__ void k_core_svd(const int* r_arr, int s, const double* sig, size_t sig_stride, const double* C,
                           size_t c_stride, const double* R, size_t r_stride, double* th, size_t th_stride, double* Z,
                           size_t z_stride, int* status) {
  extern __shared__ double sm_svd[];
  const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  const int r = r_arr[b], m = r + s, mp = m + (m & 1);
  double* A = sm_svd;              // mp x mp, column-major
  double* V = A + (size_t)mp * mp;  // mp x mp
  double* nrm = V + (size_t)mp * mp;
  int* order = (int*)(nrm + mp);
  __shared__ int s_rot;
  const double* sg = sig + b * sig_stride;
  const double* Cb = C + b * c_stride;  // r x s, ld r
  const double* Rb = R + b * r_stride;  // s x s, ld s
  for (int e = tid; e < mp * mp; e += blockDim.x) {
    const int i = e % mp, j = e / mp;
    double v = 0.0;
    if (i < m && j < m) {
      if (i < r && j < r) v = (i == j) ? sg[i] : 0.0;
      else if (i < r && j >= r) v = Cb[(size_t)(j - r) * r + i];
      else if (i >= r && j >= r) v = Rb[(size_t)(j - r) * s + (i - r)];
    }
    A[e] = v;
    V[e] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  // columns below 1e-18 of the core's norm are noise for any truncation this
  // serves (tolerances >= 1e-14): pairs of them are not rotated
  __shared__ double s_f2;
  if (tid == 0) s_f2 = 0.0;
  __syncthreads();
  {
    double f2 = 0.0;
    for (int e = tid; e < mp * mp; e += blockDim.x) f2 += A[e] * A[e];
    for (int o = 16; o > 0; o >>= 1) f2 += __shfl_xor_sync(0xffffffffu, f2, o);
    if (lane == 0) atomicAdd(&s_f2, f2);
  }
  __syncthreads();
  const double floor2 = 1e-36 * s_f2;
  const double tol_rot = 4.0 * mp * 2.220446049250313e-16;
  // round-robin schedule: position 0 holds player 0, position q > 0 holds
  // player ((q - 1 + round) mod (mp - 1)) + 1; positions k and mp-1-k meet
  auto player = [&](int q, int round) { return q == 0 ? 0 : ((q - 1 + round) % (mp - 1)) + 1; };
  int sweep = 0;
  for (; sweep < 40; ++sweep) {
    if (tid == 0) s_rot = 0;
    __syncthreads();
    for (int round = 0; round < mp - 1; ++round) {
      for (int k = warp; k < mp / 2; k += nwarp) {
        const int i = player(k, round), j = player(mp - 1 - k, round);
        double a = 0.0, bb = 0.0, g = 0.0;
        for (int row = lane; row < mp; row += 32) {
          const double x = A[(size_t)i * mp + row], y = A[(size_t)j * mp + row];
          a += x * x;
          bb += y * y;
          g += x * y;
        }
        for (int o = 16; o > 0; o >>= 1) {
          a += __shfl_xor_sync(0xffffffffu, a, o);
          bb += __shfl_xor_sync(0xffffffffu, bb, o);
          g += __shfl_xor_sync(0xffffffffu, g, o);
        }
        // orthogonal to working accuracy once |g| is within the rounding of an
        // mp-term dot product
        if (fabs(g) > tol_rot * sqrt(a * bb) && fmax(a, bb) > floor2 && fabs(g) > 1e-300) {
          const double zeta = (bb - a) / (2.0 * g);
          const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
          for (int row = lane; row < mp; row += 32) {
            const double x = A[(size_t)i * mp + row], y = A[(size_t)j * mp + row];
            A[(size_t)i * mp + row] = c * x - sn * y;
            A[(size_t)j * mp + row] = sn * x + c * y;
            const double vx = V[(size_t)i * mp + row], vy = V[(size_t)j * mp + row];
            V[(size_t)i * mp + row] = c * vx - sn * vy;
            V[(size_t)j * mp + row] = sn * vx + c * vy;
          }
          if (lane == 0) atomicAdd(&s_rot, 1);
        }
      }
      __syncthreads();
    }
    if (s_rot == 0) break;
    __syncthreads();
  }
  if (tid == 0 && sweep >= 40 && status) *status = 1;
  for (int j = warp; j < mp; j += nwarp) {
    double a = 0.0;
    for (int row = lane; row < mp; row += 32) a += A[(size_t)j * mp + row] * A[(size_t)j * mp + row];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) nrm[j] = sqrt(a);
  }
  __syncthreads();
  if (tid == 0) {
    for (int j = 0; j < mp; ++j) order[j] = j;
    for (int j = 1; j < mp; ++j) {  // insertion sort by decreasing norm (mp <= 128)
      const int x = order[j];
      int q = j - 1;
      while (q >= 0 && nrm[order[q]] < nrm[x]) {
        order[q + 1] = order[q];
        --q;
      }
      order[q + 1] = x;
    }
  }
  __syncthreads();
  double* U = Z + b * z_stride;
  double* Vo = U + (size_t)m * m;
  for (int e = tid; e < m * m; e += blockDim.x) {
    const int i = e % m, jj = e / m, j = order[jj];
    const double n_j = nrm[j];
    U[e] = n_j > 0.0 ? A[(size_t)j * mp + i] / n_j : 0.0;
    Vo[e] = V[(size_t)j * mp + i];
  }
  for (int jj = tid; jj < m; jj += blockDim.x) th[b * th_stride + jj] = nrm[order[jj]];
}

// Vn[rows n0..n0+s, :] = Zv[r:r+s, :rn]; (rows 0..n0 come from a GEMM)
__global__ void k_tail_rows(int n0, int s, int r, int m, int rn, const double* Zv, double* Vn, int ldv) {
  const int e = threadIdx.x + blockIdx.x * blockDim.x;
  if (e >= s * rn) return;
  const int i = e % s, j = e / s;
  Vn[(size_t)j * ldv + n0 + i] = Zv[(size_t)j * m + r + i];
}

__global__ void k_scale_cols(int nx, int r, const double* sig, double* W, int ldw) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (p >= nx || c >= r) return;
  W[(size_t)c * ldw + p] *= sig[c];
}

// One time column of factored trajectory Qw diag(sig) V^T:
// out[p] = sum_i Qw[p, i] sig[i] V[row, i] (row = step - 1).
__global__ void k_factor_col(int nx, int r, const double* Qw, const double* sig, const double* V, int ldv,
                             int row, double* out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nx) return;
  double acc = 0.0;
  for (int i = 0; i < r; ++i) acc += Qw[(size_t)i * nx + p] * (sig[i] * V[(size_t)i * ldv + row]);
  out[p] = acc;
}

// Observations of a factored trajectory (the adjoint's data of the truncated
// product): D[k*n_obs + s] = inv_sigma2 * sum_c w_sc (Qw diag(sig) V^T)[node_sc, n_k - 1]
// at the observed steps n_k = (k+1) obs_every, k < n_steps (8 taps per sensor).
__global__ void k_observe_factors(int nx, int r, const double* Qw, const double* sig, const double* V, int ldv,
                                  int n_obs, int n_steps, int obs_every, const int* obs_node, const double* obs_w,
                                  double inv_sigma2, double* D) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_obs * n_steps) return;
  const int k = e / n_obs, so = e % n_obs;
  const int row = (k + 1) * obs_every - 1;
  double y = 0.0;
  for (int c = 0; c < 8; ++c) {
    const int node = obs_node[so * 8 + c];
    if (node < 0) continue;
    double v = 0.0;
    for (int i = 0; i < r; ++i) v += Qw[(size_t)i * nx + node] * (sig[i] * V[(size_t)i * ldv + row]);
    y += obs_w[so * 8 + c] * v;
  }
  D[e] = y * inv_sigma2;
}

#define CKT(call)                                          \
  do {                                                     \
    cudaError_t _e = (call);                               \
    if (_e != cudaSuccess) return cuda_status(_e, #call);  \
  } while (0)

struct DBuf {
  double* p = nullptr;
  ~DBuf() {
    if (p) cudaFree(p);
  }
  cudaError_t alloc(size_t n) { return lrp::dev_malloc((void**)&p, std::max<size_t>(n, 1) * sizeof(double)); }
};

// Factor state of one column: Y_absorbed ~ Qw diag(sig) V^T.
struct TrajCol {
  DBuf Qa, Qb;  // nx x rmax (orthonormal columns)
  DBuf V, Vn;   // nt x rmax
  int r = 0;
  int nrows = 0;  // time steps absorbed
  double err_abs = 0.0;
  double fro2 = 0.0;
};

// Scratch shared by all columns (batched over columns b with fixed strides).
struct TrajWS {
  int nvec, s, rmax, m;  // m = rmax + s
  DBuf traj[2];          // nvec x s x nx: a chunk's states, orthonormalised in place
                         // (two buffers: the next chunk's sweep fills one while
                         // the other is being absorbed)
  DBuf C, C2;            // nvec x (rmax*s)
  DBuf R;                // nvec x s*s
  DBuf part;             // gemm_tn scratch
  size_t part_cap = 0;
  DBuf Zaug;             // nvec x 4m^2: the core's singular vectors [U | V] (2 m^2 used)
  DBuf th;               // nvec x 2m: the core's singular values
  DBuf gs;               // scratch of the cooperative block Gram-Schmidt (one column)
  DBuf sig;              // nvec x rmax singular values of the current factors
  int* iarr = nullptr;   // device: [0, nvec) ranks, [nvec, 2nvec) eig sizes
  ~TrajWS() {
    if (iarr) cudaFree(iarr);
  }
};

// Absorbing one chunk (sk steps, all columns; states in `traj`) into the
// factors takes two parts. The head (steps 1-2) is enqueued on stream `st`
// when no other work of the trajectory is in flight, so that a single
// column's QR may use the cooperative grid.
static lrp_status absorb_head(lrp_problem* P, std::vector<TrajCol>& cols, TrajWS& ws, int sk, cudaStream_t st,
                              double* traj) {
  const int nx = P->nx, nvec = ws.nvec, s = ws.s, rmax = ws.rmax;
  // 1. project the chunk onto the complement of each column's Qw (CGS2)
  for (int b = 0; b < nvec; ++b) {
    TrajCol& tc = cols[b];
    const int r = tc.r;
    double* B = traj + (size_t)b * s * nx;
    double* C = ws.C.p + (size_t)b * rmax * s;
    if (r == 0) continue;
    CKT(cudaMemsetAsync(C, 0, (size_t)r * sk * sizeof(double), st));
    for (int pass = 0; pass < 2; ++pass) {
      CKT(gemm_tn(st, nx, r, sk, tc.Qa.p, nx, B, nx, ws.C2.p, r, 1.0, 0.0, ws.part.p, ws.part_cap));
      CKT(gemm_nn(st, nx, r, sk, -1.0, tc.Qa.p, nx, ws.C2.p, r, 1.0, B, nx));
      CKT(axpby(st, (size_t)r * sk, 1.0, ws.C2.p, 1.0, C));
    }
  }
  // 2. rank-revealing thin QR of the remainders
  CKT(block_gs(st, nvec, nx, sk, traj, (size_t)s * nx, nx, ws.R.p, (size_t)s * s, 1e-13, nullptr, nullptr,
               ws.gs.p));
  return LRP_OK;
}

// The tail (steps 3-4), on stream `st`, may overlap the next chunk's sweep;
// the host waits for the core SVD's singular values.
static lrp_status absorb_tail(lrp_problem* P, std::vector<TrajCol>& cols, TrajWS& ws, int sk, double tol_k,
                              cudaStream_t st, const double* traj) {
  const int nx = P->nx, nt = P->nt, nvec = ws.nvec, s = ws.s, rmax = ws.rmax, M = ws.m;
  // 3. SVD of every column's small core (one-sided Jacobi)
  std::vector<int> iarr(2 * nvec);
  for (int b = 0; b < nvec; ++b) {
    iarr[b] = cols[b].r;
    iarr[nvec + b] = 2 * (cols[b].r + sk);
  }
  CKT(cudaMemcpyAsync(ws.iarr, iarr.data(), 2 * nvec * sizeof(int), cudaMemcpyHostToDevice, st));
  {
    // R of a short last chunk has leading dimension sk
    const int mp = M + (M & 1);
    const size_t smem = (2 * (size_t)mp * mp + mp) * sizeof(double) + mp * sizeof(int);
    {
      // one value from every caller: the device's opt-in maximum less the static part
      int dev = 0, optin = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
      cudaFuncAttributes fa;
      CKT(cudaFuncGetAttributes(&fa, k_core_svd));
      const int cap = optin - (int)fa.sharedSizeBytes;
      if ((long long)smem > cap) {
        set_error("time_rank_max + time_chunk too large for the core SVD in shared memory");
        return LRP_EINVAL;
      }
      CKT(cudaFuncSetAttribute(k_core_svd, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
    }
    note_launch();
    k_core_svd<<<nvec, 512, smem, st>>>(ws.iarr, sk, ws.sig.p, (size_t)rmax, ws.C.p, (size_t)rmax * s, ws.R.p,
                                        (size_t)s * s, ws.th.p, (size_t)2 * M, ws.Zaug.p, (size_t)4 * M * M, nullptr);
    CKT(cudaGetLastError());
  }
  std::vector<double> th((size_t)nvec * 2 * M);
  CKT(cudaMemcpyAsync(th.data(), ws.th.p, th.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  CKT(cudaStreamSynchronize(st));
  // 4. per column: truncation rank, new space factor, new time factor
  for (int b = 0; b < nvec; ++b) {
    TrajCol& tc = cols[b];
    const int r = tc.r, m = r + sk;
    std::vector<double> sv(m);
    for (int i = 0; i < m; ++i) sv[i] = std::max(th[(size_t)b * 2 * M + i], 0.0);
    double fro2 = 0.0;
    for (double x : sv) fro2 += x * x;
    std::vector<double> tail(m + 1, 0.0);
    for (int i = m - 1; i >= 0; --i) tail[i] = tail[i + 1] + sv[i] * sv[i];
    int rn = 0;
    while (rn < m && tail[rn] > tol_k * tol_k * fro2) ++rn;
    if (rn == 0 && m > 0 && sv[0] > 0) rn = 1;
    rn = std::min(rn, rmax);
    tc.err_abs += std::sqrt(tail[rn]);
    tc.fro2 = fro2;
    if (rn == 0) {
      tc.r = 0;
      tc.nrows += sk;
      continue;
    }
    // left (spatial) and right (time) singular vectors of the core, ld m
    const double* Ub = ws.Zaug.p + (size_t)b * 4 * M * M;
    const double* Zvb = Ub + (size_t)m * m;
    // Qw <- [Qw Q2] U
    const double* Q2 = traj + (size_t)b * s * nx;
    if (r > 0) {
      CKT(gemm_nn(st, nx, r, rn, 1.0, tc.Qa.p, nx, Ub, m, 0.0, tc.Qb.p, nx));
      CKT(gemm_nn(st, nx, sk, rn, 1.0, Q2, nx, Ub + r, m, 1.0, tc.Qb.p, nx));
    } else {
      CKT(gemm_nn(st, nx, sk, rn, 1.0, Q2, nx, Ub, m, 0.0, tc.Qb.p, nx));
    }
    std::swap(tc.Qa.p, tc.Qb.p);
    // V <- blockdiag(V, I) Zv
    if (r == 0 && tc.nrows > 0) CKT(cudaMemsetAsync(tc.Vn.p, 0, (size_t)nt * rn * sizeof(double), st));
    if (r > 0) CKT(gemm_nn(st, tc.nrows, r, rn, 1.0, tc.V.p, nt, Zvb, m, 0.0, tc.Vn.p, nt));
    note_launch();
    k_tail_rows<<<(sk * rn + 255) / 256, 256, 0, st>>>(tc.nrows, sk, r, m, rn, Zvb, tc.Vn.p, nt);
    CKT(cudaGetLastError());
    std::swap(tc.V.p, tc.Vn.p);
    CKT(cudaMemcpyAsync(ws.sig.p + (size_t)b * rmax, ws.th.p + (size_t)b * 2 * M, rn * sizeof(double),
                        cudaMemcpyDeviceToDevice, st));
    tc.r = rn;
    tc.nrows += sk;
  }
  return LRP_OK;
}

// Second stream, events and pinned sweep statistics of the chunk pipeline.
// Destruction waits for both streams, so that no buffer is freed under work
// still in flight after an early return.
struct TrajPipe {
  cudaStream_t main = nullptr, s2 = nullptr;
  cudaEvent_t sw0[2] = {}, sw1[2] = {}, head_done[2] = {}, absorbed[2] = {};
  Stats* h_stats = nullptr;  // pinned, two
  SweepLaunch info[2];
  cudaError_t init(cudaStream_t m) {
    main = m;
    cudaError_t e = cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
      e = cudaEventCreate(&sw0[i]);
      if (e == cudaSuccess) e = cudaEventCreate(&sw1[i]);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&head_done[i], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&absorbed[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaMallocHost(&h_stats, 2 * sizeof(Stats));
    return e;
  }
  ~TrajPipe() {
    if (s2) {
      cudaStreamSynchronize(s2);
      cudaStreamSynchronize(main);
      cudaStreamDestroy(s2);
    }
    for (int i = 0; i < 2; ++i) {
      if (sw0[i]) cudaEventDestroy(sw0[i]);
      if (sw1[i]) cudaEventDestroy(sw1[i]);
      if (head_done[i]) cudaEventDestroy(head_done[i]);
      if (absorbed[i]) cudaEventDestroy(absorbed[i]);
    }
    if (h_stats) cudaFreeHost(h_stats);
  }
};

// Factors and scratch of one streamed compression of nvec trajectories.
static lrp_status traj_alloc(lrp_problem* P, int nvec, std::vector<TrajCol>& cols, TrajWS& ws) {
  const int nx = P->nx, nt = P->nt;
  const int s = std::min(64, std::max(1, P->desc.time_chunk));  // the block QR handles up to 64 columns
  const int rmax = P->desc.time_rank_max;
  cols.resize(nvec);
  for (auto& c : cols) {
    CKT(c.Qa.alloc((size_t)nx * rmax));
    CKT(c.Qb.alloc((size_t)nx * rmax));
    CKT(c.V.alloc((size_t)nt * rmax));
    CKT(c.Vn.alloc((size_t)nt * rmax));
  }
  ws.nvec = nvec;
  ws.s = s;
  ws.rmax = rmax;
  ws.m = rmax + s;
  const int M = ws.m;
  CKT(ws.traj[0].alloc((size_t)nvec * s * nx));
  CKT(ws.traj[1].alloc((size_t)nvec * s * nx));
  CKT(ws.C.alloc((size_t)nvec * rmax * s));
  CKT(ws.C2.alloc((size_t)rmax * s));
  CKT(ws.R.alloc((size_t)nvec * s * s));
  ws.part_cap = (size_t)std::max(M, 16) * 16 * 128;
  CKT(ws.part.alloc(ws.part_cap));
  CKT(ws.Zaug.alloc((size_t)nvec * 4 * M * M));
  CKT(ws.th.alloc((size_t)nvec * 2 * M));
  CKT(ws.gs.alloc(block_gs_scratch_doubles()));
  CKT(ws.sig.alloc((size_t)nvec * rmax));
  CKT(lrp::dev_malloc(&ws.iarr, 2 * nvec * sizeof(int)));
  return LRP_OK;
}

// Statistics of the sweeps of one call, folded launch by launch.
struct SweepAcc {
  lrp_apply_stats acc;
  double iters_sum = 0.0;
  long long solves = 0;
  lrp_status result = LRP_OK;
  SweepAcc() { std::memset(&acc, 0, sizeof(acc)); }
  // folds one launch's statistics; returns its status unless it is LRP_ENOCONV
  // (kept as the call's result: the outputs are still written)
  lrp_status fold(lrp_status sres, const lrp_apply_stats& st) {
    if (sres != LRP_OK && sres != LRP_ENOCONV) return sres;
    if (sres == LRP_ENOCONV) result = sres;
    acc.pcg_iters_max = std::max(acc.pcg_iters_max, st.pcg_iters_max);
    acc.refine_max = std::max(acc.refine_max, st.refine_max);
    acc.max_rel_residual = std::max(acc.max_rel_residual, st.max_rel_residual);
    iters_sum += st.pcg_iters_mean * st.n_solves;
    solves += st.n_solves;
    return LRP_OK;
  }
  void fill(lrp_apply_stats* out) const {
    *out = acc;
    out->n_solves = (int)solves;
    out->pcg_iters_mean = solves ? iters_sum / solves : 0.0;
  }
};

// The forward sweep of nvec columns (optionally after the prior solve) in
// chunks of s steps over all nt steps, every chunk absorbed into the
// columns' factors.
// On the problem stream, per chunk j: its sweep, then (once chunk j-1 is
// fully absorbed) the head of its absorption. On the second stream: the
// tail, which overlaps chunk j+1's sweep (the sweep only continues its own
// state; the tail only reads chunk j's buffer and the small factors).
// Chunk j+1's sweep refills the buffer of chunk j-1, whose tail the head
// of chunk j has waited for. Returns with the problem stream ordered after
// the last absorption.
static lrp_status stream_forward(lrp_problem* P, int nvec, const double* U, int ldu, bool prior_in,
                                 std::vector<TrajCol>& cols, TrajWS& ws, double tol_k, SweepAcc& sa) {
  const int nt = P->nt, s = ws.s;
  const int K = (nt + s - 1) / s;
  TrajPipe pp;
  CKT(pp.init(P->stream));
  auto enqueue_sweep = [&](int j) -> lrp_status {
    const int b = j & 1, c0 = j * s, c1 = std::min(nt, c0 + s);
    unsigned stages = ST_FORWARD | ST_TRAJ;
    if (j == 0) stages |= ST_LOAD_X | (prior_in ? ST_PRIOR_IN : 0);
    CKT(cudaEventRecord(pp.sw0[b], P->stream));
    lrp_status r = sweep_enqueue(P, stages, nvec, U, ldu, nullptr, 0, nullptr, 0, nullptr, 0, c0, c1,
                                 ws.traj[b].p, s, pp.h_stats + b, pp.info + b);
    if (r != LRP_OK) return r;
    CKT(cudaEventRecord(pp.sw1[b], P->stream));
    return LRP_OK;
  };
  auto enqueue_head = [&](int j) -> lrp_status {
    const int b = j & 1, c0 = j * s, c1 = std::min(nt, c0 + s);
    if (j > 0) CKT(cudaStreamWaitEvent(P->stream, pp.absorbed[b ^ 1], 0));
    lrp_status r = absorb_head(P, cols, ws, c1 - c0, P->stream, ws.traj[b].p);
    if (r != LRP_OK) return r;
    CKT(cudaEventRecord(pp.head_done[b], P->stream));
    return LRP_OK;
  };
  {
    lrp_status r = enqueue_sweep(0);
    if (r == LRP_OK) r = enqueue_head(0);
    if (r != LRP_OK) return r;
  }
  for (int j = 0; j < K; ++j) {
    const int b = j & 1, c0 = j * s, c1 = std::min(nt, c0 + s);
    if (j + 1 < K) {
      lrp_status r = enqueue_sweep(j + 1);
      if (r != LRP_OK) return r;
    }
    CKT(cudaStreamWaitEvent(pp.s2, pp.head_done[b], 0));
    lrp_status a = absorb_tail(P, cols, ws, c1 - c0, tol_k, pp.s2, ws.traj[b].p);
    if (a != LRP_OK) return a;
    CKT(cudaEventRecord(pp.absorbed[b], pp.s2));
    // chunk j's sweep has completed (its head followed it)
    CKT(cudaEventSynchronize(pp.sw1[b]));
    float ms = 0.f;
    CKT(cudaEventElapsedTime(&ms, pp.sw0[b], pp.sw1[b]));
    ledger_add(P, pp.h_stats[b], pp.info[b], ms);
    lrp_apply_stats st;
    lrp_status sres = sweep_status(pp.h_stats[b], pp.info[b], &st, ms);
    if ((sres = sa.fold(sres, st)) != LRP_OK) return sres;
    if (j + 1 < K) {
      lrp_status r = enqueue_head(j + 1);
      if (r != LRP_OK) return r;
    }
  }
  // the trailing GEMMs of the last absorption precede everything after
  CKT(cudaStreamWaitEvent(P->stream, pp.absorbed[(K - 1) & 1], 0));
  return LRP_OK;
}

// Absorbs a stored trajectory (nvec x nt x nx: column b's step n at
// traj + (b*nt + n-1)*nx) into cols, chunk by chunk in time order, on the
// problem stream.
static lrp_status absorb_stored(lrp_problem* P, int nvec, const double* traj, std::vector<TrajCol>& cols,
                                TrajWS& ws, double tol_k) {
  const size_t nx = P->nx, nt = P->nt;
  const int s = ws.s;
  for (int c0 = 0; c0 < (int)nt; c0 += s) {
    const int sk = std::min<int>(s, (int)nt - c0);
    // chunk buffer layout: [column][step in chunk][nx] (absorb_head works on it in place)
    CKT(cudaMemcpy2DAsync(ws.traj[0].p, (size_t)s * nx * sizeof(double), traj + (size_t)c0 * nx,
                          nt * nx * sizeof(double), (size_t)sk * nx * sizeof(double), nvec,
                          cudaMemcpyDeviceToDevice, P->stream));
    lrp_status r = absorb_head(P, cols, ws, sk, P->stream, ws.traj[0].p);
    if (r == LRP_OK) r = absorb_tail(P, cols, ws, sk, tol_k, P->stream, ws.traj[0].p);
    if (r != LRP_OK) return r;
  }
  return LRP_OK;
}

// Largest rank and largest certified relative truncation error of the factors.
static void factor_summary(const std::vector<TrajCol>& cols, int* rank_max, double* err_max, int* ranks) {
  *rank_max = 0;
  *err_max = 0.0;
  for (size_t j = 0; j < cols.size(); ++j) {
    const TrajCol& tc = cols[j];
    *rank_max = std::max(*rank_max, tc.r);
    const double fro = std::sqrt(tc.fro2);
    *err_max = std::max(*err_max, fro > 0 ? tc.err_abs / fro : 0.0);
    if (ranks) ranks[j] = tc.r;
  }
}

lrp_status trajectory_factors_impl(lrp_problem* P, int nvec, const double* U, int ldu, double* Wout,
                                   double* Vout, int* ranks, lrp_apply_stats* stats, bool with_hessian,
                                   double* Yout, int ldy) {
  auto t0 = std::chrono::steady_clock::now();
  const int nx = P->nx, nt = P->nt;
  std::vector<TrajCol> cols;
  TrajWS ws;
  {
    lrp_status r = traj_alloc(P, nvec, cols, ws);
    if (r != LRP_OK) return r;
  }
  const int rmax = ws.rmax;
  const int K = (nt + ws.s - 1) / ws.s;
  const double tol_k = P->desc.time_trunc_tol / K;
  SweepAcc sa;
  {
    lrp_status r = stream_forward(P, nvec, U, ldu, with_hessian, cols, ws, tol_k, sa);
    if (r != LRP_OK) return r;
  }
  if (with_hessian) {
    lrp_apply_stats st;
    lrp_status sres = run_sweep_ex(P, ST_ADJOINT | ST_PRIOR_OUT | ST_STORE_Y, nvec, nullptr, 0, Yout, ldy,
                                   nullptr, 0, nullptr, 0, &st, 0, 0, nullptr, 0);
    if ((sres = sa.fold(sres, st)) != LRP_OK) return sres;
  }
  int rank_max = 0;
  double err_max = 0.0;
  factor_summary(cols, &rank_max, &err_max, ranks);
  for (int j = 0; j < nvec; ++j) {
    TrajCol& tc = cols[j];
    if (Wout && tc.r > 0) {
      double* W = Wout + (size_t)j * nx * rmax;
      CKT(cudaMemcpyAsync(W, tc.Qa.p, (size_t)nx * tc.r * sizeof(double), cudaMemcpyDeviceToDevice, P->stream));
      dim3 grid((nx + 255) / 256, tc.r);
      note_launch();
      k_scale_cols<<<grid, 256, 0, P->stream>>>(nx, tc.r, ws.sig.p + (size_t)j * rmax, W, nx);
      CKT(cudaGetLastError());
    }
    if (Vout && tc.r > 0)
      CKT(cudaMemcpyAsync(Vout + (size_t)j * nt * rmax, tc.V.p, (size_t)nt * tc.r * sizeof(double),
                          cudaMemcpyDeviceToDevice, P->stream));
  }
  CKT(cudaStreamSynchronize(P->stream));
  if (stats) {
    sa.fill(stats);
    stats->time_rank_max = rank_max;
    stats->time_trunc_err = err_max;
    stats->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return sa.result;
}

// The matrix-vector product of Sec. 4 Algorithm 1 "up to the truncation
// tolerance", with the initial condition as parameter: the space-time
// solutions it passes through (the state and the adjoint trajectory) are
// kept in low-rank-in-time form truncated to time_trunc_tol (rank cap
// time_rank_max), and every later step uses the truncated form:
//   z = Gamma_prior^{1/2} x (not for H_mis); Y = [y_1 .. y_nt] of z ~ W_Y V_Y^T
//   (chunked forward sweep, streaming recompression); d_n = B (W_Y V_Y^T) e_n
//   / sigma^2 at the observed steps; adjoint sweep with that source, storing
//   Q = [q_1 .. q_nt] ~ W_Q V_Q^T (same recompression); result
//   Gamma_prior^{1/2} (W_Q V_Q^T) e_1.
// The product is then no longer symmetric (by about the tolerance), which is
// why Algorithm 1 is an Arnoldi process. X and Y are device arrays.
lrp_status lowrank_hessian_impl(lrp_problem* P, int nvec, const double* X, int ldx, double* Y, int ldy,
                                bool misfit, lrp_apply_stats* stats) {
  auto t0 = std::chrono::steady_clock::now();
  const int nx = P->nx, nt = P->nt;
  std::vector<TrajCol> cy, cq;
  TrajWS ws;
  {
    lrp_status r = traj_alloc(P, nvec, cy, ws);
    if (r != LRP_OK) return r;
  }
  cq.resize(nvec);
  for (auto& c : cq) {
    CKT(c.Qa.alloc((size_t)nx * ws.rmax));
    CKT(c.Qb.alloc((size_t)nx * ws.rmax));
    CKT(c.V.alloc((size_t)nt * ws.rmax));
    CKT(c.Vn.alloc((size_t)nt * ws.rmax));
  }
  const int rmax = ws.rmax;
  const int K = (nt + ws.s - 1) / ws.s;
  const double tol_k = P->desc.time_trunc_tol / K;
  DBuf D, Q, Z;
  CKT(D.alloc((size_t)nvec * std::max(1, P->n_data)));
  CKT(Q.alloc((size_t)nvec * nt * nx));
  CKT(Z.alloc((size_t)nvec * nx));
  SweepAcc sa;
  // 1-2: (prior solve and) forward sweep, state factors
  {
    lrp_status r = stream_forward(P, nvec, X, ldx, !misfit, cy, ws, tol_k, sa);
    if (r != LRP_OK) return r;
  }
  // 3: the adjoint's data from the truncated state
  CKT(cudaMemsetAsync(D.p, 0, (size_t)nvec * std::max(1, P->n_data) * sizeof(double), P->stream));
  const double inv_s2 = 1.0 / (P->desc.sigma * P->desc.sigma);
  for (int b = 0; b < nvec; ++b) {
    if (cy[b].r == 0 || P->n_data == 0) continue;
    note_launch();
    k_observe_factors<<<(P->n_data + 127) / 128, 128, 0, P->stream>>>(
        nx, cy[b].r, cy[b].Qa.p, ws.sig.p + (size_t)b * rmax, cy[b].V.p, nt, P->n_obs, P->n_steps,
        P->desc.obs_every, P->obs_node, P->obs_w, inv_s2, D.p + (size_t)b * P->n_data);
    CKT(cudaGetLastError());
  }
  // 4: adjoint sweep storing its trajectory (q_n = 0 after the last observation)
  CKT(cudaMemsetAsync(Q.p, 0, (size_t)nvec * nt * nx * sizeof(double), P->stream));
  {
    lrp_apply_stats st;
    lrp_status sres = run_sweep_ex(P, ST_LOAD_D | ST_ADJOINT | ST_TRAJ_ADJ, nvec, nullptr, 0, nullptr, 0, D.p,
                                   std::max(1, P->n_data), nullptr, 0, &st, 0, 0, Q.p, nt);
    if ((sres = sa.fold(sres, st)) != LRP_OK) return sres;
  }
  int rank_y = 0, rank_q = 0;
  double err_y = 0.0, err_q = 0.0;
  factor_summary(cy, &rank_y, &err_y, nullptr);
  // the state's singular values in ws.sig are no longer needed: the adjoint's
  // compression reuses the scratch
  {
    lrp_status r = absorb_stored(P, nvec, Q.p, cq, ws, tol_k);
    if (r != LRP_OK) return r;
  }
  factor_summary(cq, &rank_q, &err_q, nullptr);
  // 5: the truncated q_1, then the prior factor
  for (int b = 0; b < nvec; ++b) {
    double* zb = Z.p + (size_t)b * nx;
    if (cq[b].r == 0) {
      CKT(cudaMemsetAsync(zb, 0, (size_t)nx * sizeof(double), P->stream));
      continue;
    }
    note_launch();
    k_factor_col<<<(nx + 255) / 256, 256, 0, P->stream>>>(nx, cq[b].r, cq[b].Qa.p, ws.sig.p + (size_t)b * rmax,
                                                         cq[b].V.p, nt, 0, zb);
    CKT(cudaGetLastError());
  }
  if (misfit) {
    CKT(cudaMemcpy2DAsync(Y, (size_t)ldy * sizeof(double), Z.p, (size_t)nx * sizeof(double),
                          (size_t)nx * sizeof(double), nvec, cudaMemcpyDeviceToDevice, P->stream));
  } else {
    lrp_apply_stats st;
    lrp_status sres = run_sweep_ex(P, ST_LOAD_X | ST_PRIOR_OUT | ST_STORE_Y, nvec, Z.p, nx, Y, ldy, nullptr, 0,
                                   nullptr, 0, &st, 0, 0, nullptr, 0);
    if ((sres = sa.fold(sres, st)) != LRP_OK) return sres;
  }
  CKT(cudaStreamSynchronize(P->stream));
  if (stats) {
    sa.fill(stats);
    stats->time_rank_max = rank_y;
    stats->time_trunc_err = err_y;
    stats->adj_rank_max = rank_q;
    stats->adj_trunc_err = err_q;
    stats->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return sa.result;
}


// SVD of a general m x m matrix M (column-major, ld m; 1 <= m <= 112) by the
// one-sided Jacobi kernel of the trajectory compression (a core with no
// carried singular values): th (device, >= 2m) gets the singular values in
// decreasing order, Z (device, >= 4 m^2) = [U | V] (two m x m blocks, ld m).
// The values are also returned on the host (the stream is synchronised).
lrp_status core_svd(cudaStream_t s, int m, const double* M, double* th, double* Z, int* iarr, int* stat,
                    std::vector<double>* th_host) {
  const int mp = m + (m & 1);
  const size_t smem = (2 * (size_t)mp * mp + mp) * sizeof(double) + mp * sizeof(int);
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  CKT(cudaFuncGetAttributes(&fa, k_core_svd));
  const int cap = optin - (int)fa.sharedSizeBytes;
  if ((long long)smem > cap) {
    set_error("core SVD larger than shared memory");
    return LRP_EINVAL;
  }
  CKT(cudaFuncSetAttribute(k_core_svd, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
  CKT(cudaMemsetAsync(iarr, 0, sizeof(int), s));
  CKT(cudaMemsetAsync(stat, 0, sizeof(int), s));
  note_launch();
  k_core_svd<<<1, 512, smem, s>>>(iarr, m, nullptr, 0, nullptr, 0, M, 0, th, 0, Z, 0, stat);
  CKT(cudaGetLastError());
  th_host->assign(m, 0.0);
  CKT(cudaMemcpyAsync(th_host->data(), th, m * sizeof(double), cudaMemcpyDeviceToHost, s));
  CKT(cudaStreamSynchronize(s));
  for (double& x : *th_host) x = std::max(x, 0.0);
  return LRP_OK;
}

cudaError_t scale_cols(cudaStream_t s, int nx, int r, const double* sig, double* W, int ldw) {
  if (r <= 0) return cudaSuccess;
  dim3 grid((nx + 255) / 256, r);
  note_launch();
  k_scale_cols<<<grid, 256, 0, s>>>(nx, r, sig, W, ldw);
  return cudaGetLastError();
}

// Compresses a stored trajectory of one column (nt x nx, step n at
// traj + (n-1)*nx) into W diag(sig) V^T by the streaming recompression;
// writes W diag(sig) (nx x r, ld nx) to Wout and V (nt x r, ld nt) to Vout,
// *r_out = r, *err = the certified relative truncation error bound.
lrp_status compress_trajectory(lrp_problem* P, const double* traj, double* Wout, double* Vout, int* r_out,
                               double* err) {
  std::vector<TrajCol> cols;
  TrajWS ws;
  {
    lrp_status r = traj_alloc(P, 1, cols, ws);
    if (r != LRP_OK) return r;
  }
  const int nx = P->nx, nt = P->nt;
  const int K = (nt + ws.s - 1) / ws.s;
  {
    lrp_status r = absorb_stored(P, 1, traj, cols, ws, P->desc.time_trunc_tol / K);
    if (r != LRP_OK) return r;
  }
  int rank = 0;
  factor_summary(cols, &rank, err, nullptr);
  const TrajCol& tc = cols[0];
  if (tc.r > 0) {
    CKT(cudaMemcpyAsync(Wout, tc.Qa.p, (size_t)nx * tc.r * sizeof(double), cudaMemcpyDeviceToDevice, P->stream));
    dim3 grid((nx + 255) / 256, tc.r);
    note_launch();
    k_scale_cols<<<grid, 256, 0, P->stream>>>(nx, tc.r, ws.sig.p, Wout, nx);
    CKT(cudaGetLastError());
    CKT(cudaMemcpyAsync(Vout, tc.V.p, (size_t)nt * tc.r * sizeof(double), cudaMemcpyDeviceToDevice, P->stream));
  }
  CKT(cudaStreamSynchronize(P->stream));
  *r_out = tc.r;
  return LRP_OK;
}

// The space-time parameter's Hessian on a factored vector U = W V^T
// (W: nx x r, V: nt x r; device): Z = Gamma_x^{1/2} W (prior solves on the
// r columns), the forward sweep with the source tau u_n = tau Z V[n-1, :]^T
// added before each step's solve (y_0 = 0) and the fused observation, the
// adjoint sweep storing q_1 .. q_nt, its streaming truncation W_Q V_Q^T,
// and the result factors (tau Gamma_x^{1/2} W_Q, V_Q). Wout: nx x
// time_rank_max, Vout: nt x time_rank_max (device).
lrp_status st_hessian_impl(lrp_problem* P, int r, const double* W, int ldw, const double* V, int ldv, double* Wout,
                           double* Vout, int* r_out, lrp_apply_stats* stats) {
  auto t0 = std::chrono::steady_clock::now();
  const int nx = P->nx, nt = P->nt;
  DBuf Z, Q, X0, Wq;
  CKT(Z.alloc((size_t)nx * std::max(r, 1)));
  CKT(Q.alloc((size_t)nt * nx));
  CKT(X0.alloc(nx));
  CKT(Wq.alloc((size_t)nx * P->desc.time_rank_max));
  SweepAcc sa;
  if (r > 0) {
    lrp_apply_stats st;
    lrp_status sres = run_sweep_ex(P, ST_LOAD_X | ST_PRIOR_IN | ST_STORE_Y, r, W, ldw, Z.p, nx, nullptr, 0, nullptr,
                                   0, &st, 0, 0, nullptr, 0);
    if ((sres = sa.fold(sres, st)) != LRP_OK) return sres;
  }
  CKT(cudaMemsetAsync(X0.p, 0, (size_t)nx * sizeof(double), P->stream));
  CKT(cudaMemsetAsync(Q.p, 0, (size_t)nt * nx * sizeof(double), P->stream));
  P->src_W = Z.p;
  P->src_V = V;
  P->src_r = r;
  P->src_ldv = ldv;
  {
    lrp_apply_stats st;
    lrp_status sres = run_sweep_ex(P, ST_LOAD_X | ST_SOURCE | ST_FORWARD | ST_ADJOINT | ST_TRAJ_ADJ, 1, X0.p, nx,
                                   nullptr, 0, nullptr, 0, nullptr, 0, &st, 0, -1, Q.p, nt);
    P->src_W = nullptr;
    P->src_V = nullptr;
    P->src_r = 0;
    if ((sres = sa.fold(sres, st)) != LRP_OK) return sres;
  }
  int rq = 0;
  double err = 0.0;
  {
    lrp_status c = compress_trajectory(P, Q.p, Wq.p, Vout, &rq, &err);
    if (c != LRP_OK) return c;
  }
  if (rq > 0) {
    lrp_apply_stats st;
    lrp_status sres = run_sweep_ex(P, ST_LOAD_X | ST_PRIOR_IN | ST_STORE_Y, rq, Wq.p, nx, Wout, nx, nullptr, 0,
                                   nullptr, 0, &st, 0, 0, nullptr, 0);
    if ((sres = sa.fold(sres, st)) != LRP_OK) return sres;
    CKT(axpby(P->stream, (size_t)nx * rq, 0.0, Wout, P->tau, Wout));
  }
  CKT(cudaStreamSynchronize(P->stream));
  *r_out = rq;
  if (stats) {
    sa.fill(stats);
    stats->adj_rank_max = rq;
    stats->adj_trunc_err = err;
    stats->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return sa.result;
}

}  // namespace lrp

using namespace lrp;

extern "C" lrp_status lrp_trajectory_factors(lrp_problem* P, int nvec, const double* U, int ldu, double* W,
                                             double* V, int* ranks, lrp_apply_stats* st) {
  if (!P || !U || !W || !V || !ranks || nvec < 0 || ldu < (P ? P->nx : 0)) {
    set_error("lrp_trajectory_factors: invalid argument");
    return LRP_EINVAL;
  }
  if (nvec == 0) return LRP_OK;
  for (const void* a : {(const void*)U, (const void*)W, (const void*)V}) {
    lrp_status sd = check_on_device(P->device, a, "lrp_trajectory_factors");
    if (sd != LRP_OK) return sd;
  }
  cudaSetDevice(P->device);
  if (!is_device_ptr(U) || !is_device_ptr(W) || !is_device_ptr(V)) {
    // stage through the device
    const size_t nx = P->nx, nt = P->nt, rmax = P->desc.time_rank_max;
    double *dU = nullptr, *dW = nullptr, *dV = nullptr;
    cudaError_t e = lrp::dev_malloc(&dU, nx * nvec * sizeof(double));
    if (e == cudaSuccess) e = lrp::dev_malloc(&dW, nx * rmax * nvec * sizeof(double));
    if (e == cudaSuccess) e = lrp::dev_malloc(&dV, nt * rmax * nvec * sizeof(double));
    if (e != cudaSuccess) {
      cudaFree(dU);
      cudaFree(dW);
      cudaFree(dV);
      return cuda_status(e, "trajectory staging");
    }
    const cudaMemcpyKind ku = is_device_ptr(U) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    e = cudaMemcpy2D(dU, nx * sizeof(double), U, (size_t)ldu * sizeof(double), nx * sizeof(double), nvec, ku);
    if (e == cudaSuccess) e = cudaMemset(dW, 0, nx * rmax * nvec * sizeof(double));
    if (e == cudaSuccess) e = cudaMemset(dV, 0, nt * rmax * nvec * sizeof(double));
    lrp_status s = e == cudaSuccess
                       ? trajectory_factors_impl(P, nvec, dU, (int)nx, dW, dV, ranks, st, false, nullptr, 0)
                       : cuda_status(e, "trajectory staging");
    if (s == LRP_OK || s == LRP_ENOCONV) {
      const cudaMemcpyKind kw = is_device_ptr(W) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
      const cudaMemcpyKind kv = is_device_ptr(V) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
      e = cudaMemcpy(W, dW, nx * rmax * nvec * sizeof(double), kw);
      if (e == cudaSuccess) e = cudaMemcpy(V, dV, nt * rmax * nvec * sizeof(double), kv);
      if (e != cudaSuccess) s = cuda_status(e, "trajectory results");
    }
    cudaFree(dU);
    cudaFree(dW);
    cudaFree(dV);
    return s;
  }
  return trajectory_factors_impl(P, nvec, U, ldu, W, V, ranks, st, false, nullptr, 0);
}
