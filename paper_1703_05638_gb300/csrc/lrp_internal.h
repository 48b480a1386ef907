// Internal structures of the GB300 low-rank posterior library.
//
// Layout in HBM (per problem):
//  * geometry of the multigrid hierarchy: n_l = (n+1)/2^l - 1 nodes per axis,
//    level 0 the finest; face diffusivities per level (FP64 and FP32 copies)
//    for the time-step operator I + tau L; the prior operator I + alpha L0 has
//    kappa = 1 and needs no arrays;
//  * sensors: per sensor 2^dim (node, weight) pairs (node -1 = unused) and the
//    transpose as CSR over fine nodes (sensor, weight) for the adjoint source;
//  * solver workspace: one slab per "team" (a thread-block cluster owning a
//    group of BV columns); inside a slab every grid vector stores BV columns
//    interleaved, element (p, j) at p*BV + j, so a thread reading item
//    (p, j) and its neighbours reads whole BV-wide rows.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "lrp.h"

#define LRP_MAXLEV 10
#define LRP_MAXBV 16

namespace lrp {

// Division by a runtime constant d (dividend < 2^31): q = (umulhi(x,m)+x) >> s.
struct FastDiv {
  uint32_t d, m, s;
};

inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  f.d = d;
  uint32_t l = 0;
  while ((1ull << l) < d) ++l;
  f.s = l;
  f.m = (uint32_t)((((uint64_t)1 << 32) * (((uint64_t)1 << l) - d)) / d + 1);
  return f;
}

// One multigrid level of one operator I + c L_l.
struct OpLevel {
  int n;        // nodes per axis
  int N;        // n^dim
  FastDiv dn;   // division by n
  double ch2;   // c / h_l^2
  double dinv;  // 1 / diagonal when kappa = 1
  const double* kd[3];  // face diffusivity (NULL -> 1), see kappa layout in lrp.h
  const float* kf[3];
  const double* dinvd;  // per-node 1 / diagonal when kappa is given
  const float* dinvf;
  double cw[3];         // convection-diffusion: c w_a / h (signed; the diffusion part is in ch2)
};

struct Op {
  int L;        // number of levels
  int Ls;       // levels Ls..L-1 are solved by every CTA of a team in its shared memory
  int has_kappa;
  int conv;     // 1: the convection-diffusion operator (not symmetric; BiCGStab, FP64)
  OpLevel lv[LRP_MAXLEV];
};

// Stage mask of one sweep-kernel launch.
enum : unsigned {
  ST_LOAD_X = 1u << 0,      // load column-major X into the start buffer
  ST_PRIOR_IN = 1u << 1,    // solve (I + alpha L0) z = x
  ST_FORWARD = 1u << 2,     // forward implicit-Euler sweep with observation
  ST_LOAD_D = 1u << 3,      // load column-major D (observations) into the team's D buffer
  ST_ADJOINT = 1u << 4,     // adjoint sweep with the B^T source
  ST_PRIOR_OUT = 1u << 5,   // solve (I + alpha L0) y = q
  ST_STORE_Y = 1u << 6,     // store the result buffer to column-major Y
  ST_STORE_D = 1u << 7,     // store the observations (unweighted) to column-major D
  ST_TRAJ = 1u << 8,        // copy every forward state into the trajectory chunk buffer
  ST_TRAJ_ADJ = 1u << 9,    // copy every adjoint state q_n into column n-1 of the trajectory buffer
  ST_SOURCE = 1u << 10,     // forward steps solve (I + tau L) y_n = y_{n-1} + s_scale W V[n-1, :]^T (one column)
  ST_SHIFTED = 1u << 11     // one solve per column with that column's operator team_ops[team] (one column per team)
};

enum : int { STAT_NOCONV = 1, STAT_NONFINITE = 2 };

struct SolveCfg {
  double rtol;        // outer relative residual
  double inner_rtol;  // mixed: FP32 inner relative residual
  int maxit;          // PCG iterations per (inner) solve
  int maxref;         // mixed: refinement sweeps
  int nu;             // Jacobi sweeps pre and post (finest level)
  int nu_coarse;      // Jacobi sweeps pre and post on the coarser levels
  double omega;       // Jacobi damping
  int mg_levels;      // levels of the time-step operator's hierarchy (0 = all)
};

struct Stats {
  unsigned long long solves;
  unsigned long long iters;
  unsigned long long refines;
  int iters_max;
  int refine_max;
  unsigned long long max_rel_res_bits;  // double bits (non-negative)
  int status;
};

struct SweepParams {
  Op step, prior;
  int dim;
  int nt;             // steps of the forward sweep (last observed step unless the trajectory is kept)
  int t_begin, t_end; // forward steps handled by this launch: t_begin+1 .. t_end
  int adj_begin;      // adjoint: first (largest) step
  int obs_every, n_obs, n_steps;
  double inv_sigma2;
  double prior_scale;      // > 0: Gamma_prior^{1/2} = prior_scale I (no prior solve); 0: MG solve with I + alpha L0
  const int* obs_node;     // [n_obs][8]
  const double* obs_w;     // [n_obs][8]
  const int* bt_ptr;       // [N0+1]
  const int* bt_idx;       // sensor index
  const double* bt_w;
  // launch geometry
  int C, NT, BV, bv_shift, nvec, n_teams;
  unsigned stages;
  // column-major inputs/outputs
  const double* X; int ldx;
  double* Y; int ldy;
  const double* Din; int lddin;
  double* Dout; int lddout;
  const double* src_W; const double* src_V; int src_r, src_ldw, src_ldv; double src_scale;  // ST_SOURCE factors
  const Op* team_ops; int shift_transpose;    // ST_SHIFTED: per-column operators (device), solve with the transpose
  double* traj; int traj_ld; int traj_cols;  // trajectory buffer: [team col][step in chunk (forward) or step-1 (adjoint)][nx]
  // workspace
  char* ws;
  size_t team_bytes;
  size_t off_dbuf[3], off_bd, off_obs;        // double vectors
  size_t off_r, off_p, off_q, off_c, off_e0[2];  // inner vectors (T)
  size_t off_e[LRP_MAXLEV][2], off_f[LRP_MAXLEV]; // coarse levels (T)
  size_t smem_off[LRP_MAXLEV][3];  // shared-memory coarse levels: e0, e1, f offsets (bytes)
  size_t smem_bytes;
  int fast_band_len;  // band kernel: floats per band array (halos and padding included)
  int fast_split1;    // band kernel: level 1 split across the cluster (each CTA owns >= 2 of its rows)
  unsigned long long* section_cycles;  // optional section timers (LRP_SECTION_TIMERS builds)
  int poison;         // fill the dynamic shared memory with NaN first (read-before-write check)
  int start_buf;      // index of the buffer that holds the sweep state at launch
  int* end_buf;       // device: buffer index holding the state at exit (per team)
  SolveCfg cfg;
  Stats* stats;
};

// host-side helpers shared by the translation units
struct DeviceBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
};

}  // namespace lrp

// The opaque problem handle.
struct lrp_problem {
  lrp_problem_desc desc;
  int dim, n, nx, nt, L;
  int n_obs, n_steps, n_data, last_obs;
  double tau, h;
  cudaStream_t stream;
  int device;
  // device arrays
  std::vector<void*> allocs;
  lrp::Op step, prior;
  int* obs_node;
  double* obs_w;
  int* bt_ptr;
  int* bt_idx;
  double* bt_w;
  // solver workspace (grown on demand)
  char* ws;
  size_t ws_bytes;
  lrp::Stats* stats;
  int* end_buf;
  int sm_count;
  // tuned launch parameters
  int team_ctas, team_cols, nthreads, coarse_items, smem_cap, kernel_variant;
  int last_kernel = 0, last_team_ctas = 0;  // what the last sweep launch used
  int allow_waves = 0;  // 1: keep the requested cluster size even if not all teams are resident at once
  // cluster size for launches whose teams at this size all fit on the GPU at
  // once (few columns: a sweep is then latency-bound and more CTAs per
  // column shorten every step); 0 = team_ctas
  int team_ctas_narrow = 0;
  int poison;  // LRP_POISON set: new workspace and shared memory start as NaN
  // caller-provided sweep workspace (set only for the duration of an
  // allocation-free call; NULL otherwise)
  char* ws_fixed;
  size_t ws_fixed_bytes;
  // factored source of the forward sweep (set only for the duration of a
  // space-time Hessian product; NULL otherwise)
  const double* src_W = nullptr;
  const double* src_V = nullptr;
  int src_r = 0, src_ldv = 0;
  // per-column operators of an ST_SHIFTED launch (set only for the duration
  // of an alternating space-time solve): host templates (one per column;
  // the launcher sets their shared-memory level split) and their device copy
  std::vector<lrp::Op> shift_ops;
  lrp::Op* shift_ops_dev = nullptr;
  int shift_transpose = 0;
  lrp::SolveCfg cfg;
  uint64_t hash;
  // sweep-kernel ledger (lrp_sweep_profile): CUDA-event time and algorithmic
  // bytes of every sweep launch while enabled
  // (index 0: all launches; 1: generic team kernel; 2: band kernel)
  int prof_on;
  cudaEvent_t prof_ev[2];
  // (3: generic kernel, 4: band kernel, launches that run a whole Hessian
  // apply: both prior solves, the forward and the adjoint sweep)
  double prof_ms[5];
  double prof_bytes[5];
  unsigned long long prof_launches[5];
  size_t dev_bytes = 0;  // device bytes of the problem's own arrays (not the workspace)
};

struct lrp_posterior {
  lrp_problem* prob;
  int k;             // number of eigenpairs kept
  int nx;
  double sigma0;
  double* lambda;    // device [k]
  double* V;         // device nx x k
  double* G;         // device nx x k, R^{-1} V
  std::vector<double> lambda_host;
  // prior variance at every node (sine-transform closed form), computed by the
  // first variance query
  double* diag;      // device, nx
  int diag_cap;
};

namespace lrp {
void note_launch(unsigned n = 1);
void set_error(const std::string& msg);
lrp_status cuda_status(cudaError_t e, const char* where);
bool is_device_ptr(const void* p);
// Every device allocation of the library goes through here (cudaMalloc, plus
// the failure injection of lrp_debug_fail_alloc).
cudaError_t dev_malloc_raw(void** p, size_t bytes);
template <class T>
inline cudaError_t dev_malloc(T** p, size_t bytes) {
  return dev_malloc_raw((void**)p, bytes);
}
lrp_status check_on_device(int device, const void* p, const char* what);

// sweep launcher (lrp_sweep.cu)
struct SweepLaunch {
  bool fast = false, mixed = false, bf16 = false;
  int BV = 1, n_teams = 0;
  unsigned stages = 0;
};
lrp_status sweep_enqueue(lrp_problem* Pr, unsigned stages, int nvec, const double* X, int ldx, double* Y, int ldy,
                         const double* Din, int lddin, double* Dout, int lddout, int t_begin, int t_end,
                         double* traj, int traj_cols, Stats* hs_dst, SweepLaunch* info);
lrp_status sweep_status(const Stats& hs, const SweepLaunch& info, lrp_apply_stats* st, double ms);
void ledger_add(lrp_problem* Pr, const Stats& hs, const SweepLaunch& info, double ms);
lrp_status run_sweep(lrp_problem* P, unsigned stages, int nvec, const double* X, int ldx,
                     double* Y, int ldy, const double* Din, int lddin, double* Dout,
                     int lddout, lrp_apply_stats* st, bool misfit_only);
lrp_status run_sweep_ex(lrp_problem* Pr, unsigned stages, int nvec, const double* X, int ldx, double* Y,
                        int ldy, const double* Din, int lddin, double* Dout, int lddout, lrp_apply_stats* st,
                        int t_begin, int t_end, double* traj, int traj_cols);
lrp_status trajectory_factors_impl(lrp_problem* P, int nvec, const double* U, int ldu, double* Wout,
                                   double* Vout, int* ranks, lrp_apply_stats* stats, bool with_hessian,
                                   double* Yout, int ldy);
lrp_status ensure_workspace(lrp_problem* P, size_t bytes);
// Y = the truncated product of Algorithm 1 (LRP_LOWRANK_SOURCE); X, Y device arrays.
lrp_status lowrank_hessian_impl(lrp_problem* P, int nvec, const double* X, int ldx, double* Y, int ldy,
                                bool misfit, lrp_apply_stats* stats);
// Y = Htilde X (H_mis X if misfit) with the forward and adjoint space-time
// systems solved by the alternating low-rank solver (LRP_ALS_SOLVES); X, Y
// device arrays.
lrp_status als_hessian_impl(lrp_problem* P, int nvec, const double* X, int ldx, double* Y, int ldy, bool misfit,
                            lrp_apply_stats* stats);
// Stored one-column trajectory -> W diag(sig), V (streaming truncation).
lrp_status compress_trajectory(lrp_problem* P, const double* traj, double* Wout, double* Vout, int* r_out,
                               double* err);
// The space-time parameter's Hessian on factors (W, V) -> (Wout, Vout, *r_out).
lrp_status st_hessian_impl(lrp_problem* P, int r, const double* W, int ldw, const double* V, int ldv, double* Wout,
                           double* Vout, int* r_out, lrp_apply_stats* stats);
// General m x m SVD by one-sided Jacobi (th: singular values, Z = [U | V]).
lrp_status core_svd(cudaStream_t s, int m, const double* M, double* th, double* Z, int* iarr, int* stat,
                    std::vector<double>* th_host);
cudaError_t scale_cols(cudaStream_t s, int nx, int r, const double* sig, double* W, int ldw);
}  // namespace lrp
