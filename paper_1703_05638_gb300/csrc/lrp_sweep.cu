// Host launcher of the persistent sweep kernel (lrp_sweep_kernel.cuh): team
// workspace layout, levels worked by the whole team, cluster launch, stats.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <string>

#include "lrp_internal.h"

namespace lrp {

constexpr int FAST_HALO_ROWS = 2;  // halo rows of the band kernel

template <typename T, int DIM, bool MIXED, typename ES = T>
cudaError_t launch_sweep(const SweepParams& prm, cudaStream_t stream);
extern template cudaError_t launch_sweep<double, 2, false>(const SweepParams&, cudaStream_t);
extern template cudaError_t launch_sweep<double, 3, false>(const SweepParams&, cudaStream_t);
extern template cudaError_t launch_sweep<float, 2, true>(const SweepParams&, cudaStream_t);
extern template cudaError_t launch_sweep<float, 3, true>(const SweepParams&, cudaStream_t);
extern template cudaError_t launch_sweep<float, 2, true, __nv_bfloat16>(const SweepParams&, cudaStream_t);
extern template cudaError_t launch_sweep<float, 3, true, __nv_bfloat16>(const SweepParams&, cudaStream_t);
template <typename T, int DIM, bool MIXED, typename ES = T>
int max_resident_teams(int C, int NT, size_t smem, int sm_count);
extern template int max_resident_teams<double, 2, false>(int, int, size_t, int);
extern template int max_resident_teams<double, 3, false>(int, int, size_t, int);
extern template int max_resident_teams<float, 2, true>(int, int, size_t, int);
extern template int max_resident_teams<float, 3, true>(int, int, size_t, int);
extern template int max_resident_teams<float, 2, true, __nv_bfloat16>(int, int, size_t, int);
extern template int max_resident_teams<float, 3, true, __nv_bfloat16>(int, int, size_t, int);

cudaError_t launch_fast2d(const SweepParams& prm, cudaStream_t stream);
int fast2d_resident_teams(int C, int NT, size_t smem, int sm_count);

static int resident_teams(bool mixed, bool bf16, int dim, int C, int NT, size_t smem, int sm_count) {
  if (mixed && bf16)
    return dim == 2 ? max_resident_teams<float, 2, true, __nv_bfloat16>(C, NT, smem, sm_count)
                    : max_resident_teams<float, 3, true, __nv_bfloat16>(C, NT, smem, sm_count);
  if (dim == 2)
    return mixed ? max_resident_teams<float, 2, true>(C, NT, smem, sm_count)
                 : max_resident_teams<double, 2, false>(C, NT, smem, sm_count);
  return mixed ? max_resident_teams<float, 3, true>(C, NT, smem, sm_count)
               : max_resident_teams<double, 3, false>(C, NT, smem, sm_count);
}


static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

// Algorithmic bytes of one sweep launch from the solver's own counts: the
// passes over fine-level vectors each phase makes (coarse levels add 1/3 in
// 2D, 1/7 in 3D), per point and column:
//   PCG iteration: phase A 5, phase B 7, V-cycle 3(nu-1) pre-sweeps +
//     2.5 restriction + 2.25 prolongation + 3 nu post-sweeps + 1 (r.z),
//     in words of the inner type;
//   solve set-up: 3 FP64 + 2 inner words; FP64 refinement: 3 FP64 + 3 inner.
double algorithmic_bytes(const lrp_problem* Pr, const Stats& hs, int BV, bool mixed, bool bf16) {
  const double T = mixed ? 4.0 : 8.0, D = 8.0;
  const double E = bf16 ? 2.0 : T;  // multigrid vectors of the global-memory levels
  const double nu = Pr->cfg.nu;
  const double g = Pr->dim == 2 ? 4.0 / 3.0 : 8.0 / 7.0;
  // phases A and B: 10 words of PCG vectors, 2 of multigrid vectors (z read,
  // the first smoother iterate written); the V-cycle: multigrid vectors
  // (r, read once, counted in T)
  const double c_it_bytes = 10.0 * T + 2.0 * E + (3.0 * (nu - 1.0) + 2.5 + 2.25 + 3.0 * nu) * g * E + g * T;
  const double per_point = (double)hs.iters * c_it_bytes + (double)hs.refines * (3.0 * D + 3.0 * T) +
                           (double)hs.solves * (3.0 * D + 2.0 * T);
  return per_point * (double)Pr->nx * BV;
}

lrp_status run_sweep(lrp_problem* Pr, unsigned stages, int nvec, const double* X, int ldx,
                     double* Y, int ldy, const double* Din, int lddin, double* Dout, int lddout,
                     lrp_apply_stats* st, bool misfit_only) {
  (void)misfit_only;
  return run_sweep_ex(Pr, stages, nvec, X, ldx, Y, ldy, Din, lddin, Dout, lddout, st, 0, -1, nullptr, 0);
}

// Enqueues one sweep launch on the problem's stream without host
// synchronisation (so it can be captured into a CUDA graph): the stats are
// reset before the launch and copied to *hs_dst (host memory; pinned for an
// asynchronous copy) after it. t_end < 0: the forward sweep runs to the last
// observed step. The workspace must already be large enough when the stream
// is being captured (it cannot be reallocated then).
lrp_status sweep_enqueue(lrp_problem* Pr, unsigned stages, int nvec, const double* X, int ldx, double* Y, int ldy,
                         const double* Din, int lddin, double* Dout, int lddout, int t_begin, int t_end,
                         double* traj, int traj_cols, Stats* hs_dst, SweepLaunch* info) {
  const bool mixed = Pr->desc.precision == LRP_MIXED;
  // per-column operators: one column per team
  const int BV = (stages & ST_SHIFTED) ? 1 : Pr->team_cols;
  if ((stages & ST_SHIFTED) && ((int)Pr->shift_ops.size() < nvec || !Pr->shift_ops_dev)) {
    set_error("shifted solves without per-column operators");
    return LRP_EINVAL;
  }
  int bvs = 0;
  while ((1 << bvs) < BV) ++bvs;
  const int n_teams = (nvec + BV - 1) / BV;
  const size_t tsz = mixed ? sizeof(float) : sizeof(double);
  // BF16 storage of the multigrid vectors: the generic kernel only (the band
  // kernel keeps its vectors in shared memory in FP32); decided with the
  // kernel below, the workspace is laid out for the larger element size
  const bool bf16_req = mixed && Pr->desc.mg_bf16 != 0;
  if (bf16_req && (Pr->kernel_variant == 2 || Pr->kernel_variant == 3)) {
    set_error("the band kernel has no BF16 form (mg_bf16 runs the generic kernel)");
    return LRP_EINVAL;
  }
  const size_t N0 = (size_t)Pr->nx;
  SweepParams prm;
  std::memset(&prm, 0, sizeof(prm));
  cudaError_t e0 = cudaSuccess;
  size_t off = 0;
  for (int k = 0; k < 3; ++k) {
    prm.off_dbuf[k] = off;
    off = align_up(off + N0 * BV * sizeof(double));
  }
  prm.off_bd = off;
  off = align_up(off + (mixed ? N0 * BV * sizeof(double) : 0));
  prm.off_obs = off;
  off = align_up(off + (size_t)Pr->n_obs * Pr->n_steps * BV * sizeof(double));
  prm.off_r = off;
  off = align_up(off + N0 * BV * tsz);
  prm.off_p = off;
  off = align_up(off + N0 * BV * tsz);
  prm.off_q = off;
  off = align_up(off + N0 * BV * tsz);
  prm.off_c = off;
  // mixed: the inner correction; convection-diffusion: BiCGStab's shadow residual
  off = align_up(off + ((mixed || Pr->step.conv) ? N0 * BV * tsz : 0));
  const size_t esz = bf16_req ? sizeof(__nv_bfloat16) : tsz;
  prm.off_e0[0] = off;
  off = align_up(off + N0 * BV * esz);
  prm.off_e0[1] = off;
  off = align_up(off + N0 * BV * esz);
  for (int l = 1; l < Pr->L; ++l) {
    const size_t Nl = (size_t)Pr->step.lv[l].N;
    prm.off_e[l][0] = off;
    off = align_up(off + Nl * BV * esz);
    prm.off_e[l][1] = off;
    off = align_up(off + Nl * BV * esz);
    prm.off_f[l] = off;
    off = align_up(off + Nl * BV * esz);
  }
  prm.team_bytes = off;
  if (Pr->ws_fixed) {
    if (off * n_teams > Pr->ws_fixed_bytes) {
      set_error("the fixed workspace holds " + std::to_string(Pr->ws_fixed_bytes) + " bytes; this call needs " +
                std::to_string(off * n_teams));
      return LRP_EINVAL;
    }
    prm.ws = Pr->ws_fixed;
  } else {
    if (off * n_teams > Pr->ws_bytes) {
      cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
      cudaStreamIsCapturing(Pr->stream, &cs);
      if (cs != cudaStreamCaptureStatusNone) {
        set_error("sweep workspace too small while the stream is being captured");
        return LRP_EINVAL;
      }
    }
    lrp_status s = ensure_workspace(Pr, off * n_teams);
    if (s != LRP_OK) return s;
    prm.ws = Pr->ws;
  }
  prm.step = Pr->step;
  prm.prior = Pr->prior;
  // coarse levels solved redundantly in every CTA's shared memory: the first
  // level l >= 1 with at most coarse_items items whose levels l..L-1 fit the
  // shared-memory budget
  int Ls = Pr->L > 1 ? Pr->L - 1 : 1;
  for (int l = Pr->L - 1; l >= 1; --l) {
    size_t bytes = 0;
    for (int c = l; c < Pr->L; ++c) bytes += 3 * (((size_t)Pr->step.lv[c].N * BV * tsz + 15) & ~(size_t)15);
    if ((long long)Pr->step.lv[l].N * BV <= Pr->coarse_items && bytes <= (size_t)Pr->smem_cap) Ls = l;
  }
  // the time-step operator's hierarchy may stop above the one-node level;
  // its coarsest kept level then lives in shared memory too (if it fits)
  int Ls_step = Ls;
  if (Pr->cfg.mg_levels >= 3 && Pr->cfg.mg_levels < Pr->L) {
    const int Lst = Pr->cfg.mg_levels;
    const int cand = std::min(Ls, Lst - 1);
    size_t bytes = 0;
    for (int c = cand; c < Pr->L; ++c) bytes += 3 * (((size_t)Pr->step.lv[c].N * BV * tsz + 15) & ~(size_t)15);
    if (bytes <= (size_t)Pr->smem_cap) {
      prm.step.L = Lst;
      Ls_step = cand;
    }
  }
  const int Ls_all = std::min(Ls, Ls_step);
  size_t soff = 0;
  for (int l = 0; l < LRP_MAXLEV; ++l) {
    for (int k = 0; k < 3; ++k) prm.smem_off[l][k] = 0;
    if (l >= Ls_all && l < Pr->L) {
      const size_t b = ((size_t)Pr->step.lv[l].N * BV * tsz + 15) & ~(size_t)15;
      for (int k = 0; k < 3; ++k) {
        prm.smem_off[l][k] = soff;
        soff += b;
      }
    }
  }
  prm.smem_bytes = soff;
  prm.poison = Pr->poison;
  prm.step.Ls = Ls_step;
  prm.prior.Ls = Ls;
  // team size: the largest C <= the requested one whose teams all stay
  // resident; few teams take the narrow-launch size when they all fit at it
  int C = Pr->team_ctas;
  if (Pr->team_ctas_narrow > 0 && (long long)n_teams * Pr->team_ctas_narrow <= Pr->sm_count)
    C = Pr->team_ctas_narrow;
  // Band kernel (2D, kappa = 1, one column per team, FP32 inner): every CTA
  // keeps its band of the finest level and all coarse levels in shared memory.
  bool fast = false;
  if (Pr->kernel_variant != 1 && !bf16_req && !(stages & (ST_SOURCE | ST_SHIFTED)) && Pr->dim == 2 && mixed && BV == 1 && !Pr->step.has_kappa &&
      !Pr->step.conv &&
      Pr->L >= 2 &&
      Pr->n <= 128) {
    const int n = Pr->n;
    for (int Cf = C; Cf >= 1; Cf >>= 1) {
      if (n / Cf < FAST_HALO_ROWS) continue;
      const int rows_max = (n + Cf - 1) / Cf;
      const int band_len = (rows_max + 2 * FAST_HALO_ROWS) * (n + 1) + 2;
      size_t bytes = ((size_t)6 * band_len * sizeof(float) + 15) & ~(size_t)15;
      size_t offs[LRP_MAXLEV][3] = {};
      for (int l = 1; l < Pr->L; ++l)
        for (int k = 0; k < 3; ++k) {
          offs[l][k] = bytes;
          const size_t nl = Pr->step.lv[l].n;  // padded copy: (n+2) rows of pitch n+1, plus 2
          bytes += (((nl + 2) * (nl + 1) + 2) * sizeof(float) + 15) & ~(size_t)15;
        }
      if (bytes > (size_t)215 * 1024) continue;
      if (!Pr->allow_waves && fast2d_resident_teams(Cf, Pr->nthreads, bytes, Pr->sm_count) < n_teams && Cf > 1)
        continue;
      fast = true;
      C = Cf;
      prm.fast_band_len = band_len;
      prm.smem_bytes = bytes;
      for (int l = 0; l < LRP_MAXLEV; ++l)
        for (int k = 0; k < 3; ++k) prm.smem_off[l][k] = offs[l][k];
      break;
    }
    if (!fast && (Pr->kernel_variant == 2 || Pr->kernel_variant == 3)) {
      set_error("the band kernel does not apply to or fit this problem");
      return LRP_EINVAL;
    }
    // level 1 split across the cluster: every CTA must own at least two of
    // its rows (the rows J with 2J+1 in the CTA's band: J in [r0/2, r1/2))
    prm.fast_split1 = 0;
    if (fast && Pr->kernel_variant != 2 && Pr->L >= 3 && C > 1) {
      bool ok = true;
      for (int k = 0; k < C; ++k) {
        const int r0 = k * n / C, r1 = (k + 1) * n / C;
        if (r1 / 2 - r0 / 2 < 2) ok = false;
      }
      prm.fast_split1 = ok ? 1 : 0;
    }
    if (Pr->kernel_variant == 3 && !prm.fast_split1) {
      set_error("the split-level band kernel does not apply to this problem and cluster size");
      return LRP_EINVAL;
    }
  }
  if (!fast && !Pr->allow_waves)
    while (C > 1 && resident_teams(mixed, bf16_req, Pr->dim, C, Pr->nthreads, soff, Pr->sm_count) < n_teams) C >>= 1;
  Pr->last_kernel = fast ? 2 : 1;
  Pr->last_team_ctas = C;
  prm.dim = Pr->dim;
  prm.nt = Pr->nt;
  prm.t_begin = t_begin;
  prm.t_end = t_end >= 0 ? t_end : Pr->last_obs;
  prm.traj = traj;
  prm.traj_ld = Pr->nx;
  prm.src_W = Pr->src_W;
  prm.src_V = Pr->src_V;
  prm.src_r = (stages & ST_SOURCE) ? Pr->src_r : 0;
  prm.src_ldw = Pr->nx;
  prm.src_ldv = Pr->src_ldv;
  prm.src_scale = Pr->tau;
  prm.traj_cols = traj_cols;
  if (stages & ST_SHIFTED) {
    // the per-column operators keep the whole hierarchy (their coefficient
    // can be much larger than tau) with the prior's shared-memory split
    for (int j = 0; j < nvec; ++j) {
      Pr->shift_ops[j].L = Pr->L;
      Pr->shift_ops[j].Ls = Ls;
    }
    e0 = cudaMemcpyAsync(Pr->shift_ops_dev, Pr->shift_ops.data(), sizeof(Op) * nvec, cudaMemcpyHostToDevice,
                         Pr->stream);
    if (e0 != cudaSuccess) return cuda_status(e0, "per-column operators");
    prm.team_ops = Pr->shift_ops_dev;
    prm.shift_transpose = Pr->shift_transpose;
  }
  prm.adj_begin = Pr->last_obs;
  prm.obs_every = Pr->desc.obs_every;
  prm.n_obs = Pr->n_obs;
  prm.n_steps = Pr->n_steps;
  prm.inv_sigma2 = 1.0 / (Pr->desc.sigma * Pr->desc.sigma);
  prm.prior_scale = Pr->desc.prior_kind == LRP_PRIOR_IDENTITY ? std::sqrt(Pr->desc.prior_gamma) : 0.0;
  prm.obs_node = Pr->obs_node;
  prm.obs_w = Pr->obs_w;
  prm.bt_ptr = Pr->bt_ptr;
  prm.bt_idx = Pr->bt_idx;
  prm.bt_w = Pr->bt_w;
  prm.C = C;
  prm.NT = Pr->nthreads;
  prm.BV = BV;
  prm.bv_shift = bvs;
  prm.nvec = nvec;
  prm.n_teams = n_teams;
  prm.stages = stages;
  prm.X = X;
  prm.ldx = ldx;
  prm.Y = Y;
  prm.ldy = ldy;
  prm.Din = Din;
  prm.lddin = lddin;
  prm.Dout = Dout;
  prm.lddout = lddout;
  prm.end_buf = Pr->end_buf;
  prm.cfg = Pr->cfg;
  prm.stats = Pr->stats;
  cudaError_t e = cudaMemsetAsync(Pr->stats, 0, sizeof(Stats), Pr->stream);
  if (e != cudaSuccess) return cuda_status(e, "stats reset");
  if (info) {
    info->fast = fast;
    info->stages = stages;
    info->BV = BV;
    info->n_teams = n_teams;
    info->mixed = mixed;
    info->bf16 = bf16_req && !fast;
  }
  if (Pr->prof_on) cudaEventRecord(Pr->prof_ev[0], Pr->stream);
#ifdef LRP_SECTION_TIMERS
  static unsigned long long* sec_buf = nullptr;
  if (!sec_buf) lrp::dev_malloc(&sec_buf, 12 * sizeof(unsigned long long));
  cudaMemsetAsync(sec_buf, 0, 12 * sizeof(unsigned long long), Pr->stream);
  prm.section_cycles = sec_buf;
#endif
  if (fast) {
    e = launch_fast2d(prm, Pr->stream);
  } else if (bf16_req) {
    e = Pr->dim == 2 ? launch_sweep<float, 2, true, __nv_bfloat16>(prm, Pr->stream)
                     : launch_sweep<float, 3, true, __nv_bfloat16>(prm, Pr->stream);
  } else if (Pr->dim == 2) {
    e = mixed ? launch_sweep<float, 2, true>(prm, Pr->stream)
              : launch_sweep<double, 2, false>(prm, Pr->stream);
  } else {
    e = mixed ? launch_sweep<float, 3, true>(prm, Pr->stream)
              : launch_sweep<double, 3, false>(prm, Pr->stream);
  }
  if (e != cudaSuccess) return cuda_status(e, "sweep launch");
  note_launch();
  if (Pr->prof_on) cudaEventRecord(Pr->prof_ev[1], Pr->stream);
  if (hs_dst) {
    e = cudaMemcpyAsync(hs_dst, Pr->stats, sizeof(Stats), cudaMemcpyDeviceToHost, Pr->stream);
    if (e != cudaSuccess) return cuda_status(e, "stats copy");
  }
#ifdef LRP_SECTION_TIMERS
  {
    cudaStreamSynchronize(Pr->stream);
    unsigned long long sc[12];
    cudaMemcpy(sc, prm.section_cycles, sizeof(sc), cudaMemcpyDeviceToHost);
    std::fprintf(stderr,
                 "[sections %s] finest %.3e sync %.3e coarse %.3e coarse2/smem %.3e restrict0 %.3e refine %.3e "
                 "reduce %.3e pcg-vectors %.3e total %.3e cycles\n",
                 fast ? "band" : "generic", (double)sc[0], (double)sc[1], (double)sc[2], (double)sc[6],
                 (double)sc[7], (double)sc[3], (double)sc[4], (double)sc[5], (double)sc[11]);
  }
#endif
  return LRP_OK;
}

// Adds a completed launch to the problem's sweep ledger (when recording).
void ledger_add(lrp_problem* Pr, const Stats& hs, const SweepLaunch& info, double ms) {
  if (!Pr->prof_on) return;
  const double ab = algorithmic_bytes(Pr, hs, info.BV, info.mixed, info.bf16);
  const unsigned hess = ST_PRIOR_IN | ST_FORWARD | ST_ADJOINT | ST_PRIOR_OUT;
  const bool whole = (info.stages & hess) == hess;
  for (int v : {0, info.fast ? 2 : 1, whole ? (info.fast ? 4 : 3) : -1}) {
    if (v < 0) continue;
    Pr->prof_ms[v] += ms;
    Pr->prof_launches[v] += 1;
    Pr->prof_bytes[v] += ab;
  }
}

// Status of a completed sweep launch from its stats (and the caller's stats
// record, if st is not NULL).
lrp_status sweep_status(const Stats& hs, const SweepLaunch& info, lrp_apply_stats* st, double ms) {
  if (st) {
    std::memset(st, 0, sizeof(*st));
    st->n_solves = (int)(hs.solves / (unsigned long long)std::max(1, info.n_teams));
    st->pcg_iters_max = hs.iters_max;
    st->pcg_iters_mean = hs.solves ? (double)hs.iters / (double)hs.solves : 0.0;
    st->refine_max = hs.refine_max;
    double mr;
    std::memcpy(&mr, &hs.max_rel_res_bits, sizeof(double));
    st->max_rel_residual = mr;
    st->ms = ms;
  }
  if (hs.status & STAT_NONFINITE) {
    set_error("non-finite value in a spatial solve");
    return LRP_ENONFINITE;
  }
  if (hs.status & STAT_NOCONV) {
    set_error("a spatial solve missed its tolerance within the iteration cap");
    return LRP_ENOCONV;
  }
  return LRP_OK;
}

lrp_status run_sweep_ex(lrp_problem* Pr, unsigned stages, int nvec, const double* X, int ldx, double* Y, int ldy,
                        const double* Din, int lddin, double* Dout, int lddout, lrp_apply_stats* st, int t_begin,
                        int t_end, double* traj, int traj_cols) {
  auto t0 = std::chrono::steady_clock::now();
  Stats hs;
  SweepLaunch info;
  lrp_status s = sweep_enqueue(Pr, stages, nvec, X, ldx, Y, ldy, Din, lddin, Dout, lddout, t_begin, t_end, traj,
                               traj_cols, &hs, &info);
  if (s != LRP_OK) return s;
  cudaError_t e = cudaStreamSynchronize(Pr->stream);
  if (e != cudaSuccess) return cuda_status(e, "sweep");
  if (Pr->prof_on) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, Pr->prof_ev[0], Pr->prof_ev[1]);
    ledger_add(Pr, hs, info, ms);
  }
  return sweep_status(hs, info, st,
                      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count());
}

}  // namespace lrp
