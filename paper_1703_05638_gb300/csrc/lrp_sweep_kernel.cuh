#pragma once
// Persistent sweep kernel: one launch runs, for every group of BV columns,
// the prior half-apply, the forward implicit-Euler sweep with the fused
// observation, the adjoint sweep with the fused B^T source and the second
// prior half-apply (the Hessian apply of Sec. 2 Eq. (prior_pre) /
// Sec. 6.1 Eq. (misfit)), or any subset of these stages.
//
// Work decomposition: a "team" is one thread-block cluster of C CTAs that owns
// BV columns; it steps through all 2*nt spatial solves on its own, separated
// from its phases by hardware cluster barriers, and never waits on another
// team. Each spatial solve is preconditioned CG on I + c L with one V-cycle
// per iteration; LRP_MIXED runs the PCG in FP32 inside FP64 iterative
// refinement (residual and solution in FP64).
#include <cuda_runtime.h>

#include <type_traits>

#include "lrp_team.cuh"

namespace lrp {

// Team vectors. The multigrid vectors on the levels held in global memory
// (smoother iterates e, coarse right-hand sides f) are stored as ES (T, or
// BF16 with arithmetic in FP32); level 0's right-hand side is the PCG
// residual r (T).
template <typename T, typename ES = T>
struct WSV {
  double* dbuf[3];
  double* bd;
  double* obs;
  T* r;
  T* p;
  T* q;
  T* c;
  ES* e[LRP_MAXLEV][2];  // level 0: the two finest smoother buffers
  ES* f[LRP_MAXLEV];     // levels >= 1 (level 0: r)
};

struct Ctr {
  long long iters = 0, refines = 0, solves = 0;
  int iters_max = 0, refine_max = 0;
  double max_res = 0.0;
  int status = 0;
  double mix_scale = 1.0;  // power-of-two scale of the next FP32 inner problem (this column)
};

// 2^-round(log2(x)) for x > 0 (exact power of two; 1 for x = 0 or non-finite)
__device__ __forceinline__ double pow2_inv(double x) {
  if (!(x > 0.0) || !isfinite(x)) return 1.0;
  int e;
  frexp(x, &e);
  return ldexp(1.0, -e);
}

// Pointers of the shared-memory copies of the coarse levels Ls..L-1.
template <typename T>
struct SmemLv {
  T* e[LRP_MAXLEV][2];
  T* f[LRP_MAXLEV];
};

// Calls fn with level l's right-hand side: w.f[l], which for level 0 is r
// itself when the multigrid vectors have the arithmetic type (one code path,
// as before BF16 storage existed); with BF16 storage level 0's is r (T) and
// the others' are BF16, two instantiations of the phase.
template <typename T, typename ES, class Fn>
__device__ __forceinline__ void with_rhs(const WSV<T, ES>& w, int l, Fn&& fn) {
  if constexpr (std::is_same<ES, T>::value) {
    fn(w.f[l]);
  } else {
    if (l == 0)
      fn((const T*)w.r);
    else
      fn((const ES*)w.f[l]);
  }
}

// V-cycle: z = M r. On entry f[0] = r is complete and e[0][0] holds the first
// (pointwise) smoother sweep of level 0. Levels 0..Ls-1 live in global memory
// and are worked by the whole team (phases separated by team barriers);
// levels Ls..L-1 are small: every CTA restricts level Ls-1 into its own
// shared-memory copy of level Ls and runs the rest of the cycle there with
// block barriers only, so no CTA idles and no team barrier is needed before
// the prolongation back to level Ls-1 (all copies are bit-identical). On exit
// z = e[0][returned index] and the team total r.z is in slot SL_RZ.
template <typename T, typename ES, int DIM, bool KAPPA>
__device__ LRP_SOLVER_FN int vcycle(const Team& t, const Op& op, const WSV<T, ES>& w, const SmemLv<T>& sm, T omega,
                                    int nu) {
  int ecur[LRP_MAXLEV];
  for (int l = 0; l < LRP_MAXLEV; ++l) ecur[l] = 0;
  const int L = op.L;
  if (L == 1) return 0;  // z = r/d was formed exactly in the fused phase (rz too)
  const int Ls = op.Ls;  // 1 <= Ls <= L-1
  double rz = 0.0;
  SEC_T0();
  // down: team levels 0..Ls-2 (pre-smoothing, restriction in global memory)
  for (int l = 0; l < Ls - 1; ++l) {
    for (int s = 1; s < nu; ++s) {
      with_rhs(w, l, [&](auto fl) {
        mg_sweep<T, DIM, KAPPA>(op.lv[l], w.e[l][ecur[l] ^ 1], w.e[l][ecur[l]], fl, t.g, t.S, t.bvs, t.col, omega,
                                (const T*)nullptr, rz);
      });
      ecur[l] ^= 1;
      SEC_ADD(l == 0 ? SEC_BAND : SEC_COARSE);
      team_sync(t);
      SEC_ADD(SEC_SYNC);
    }
    with_rhs(w, l, [&](auto fl) {
      mg_restrict<T, DIM, KAPPA>(op.lv[l], op.lv[l + 1], w.e[l][ecur[l]], fl, w.f[l + 1], w.e[l + 1][0], t.g, t.S,
                                 t.bvs, t.col, omega);
    });
    ecur[l + 1] = 0;
    SEC_ADD(l == 0 ? SEC_RESTRICT : SEC_COARSE);
    team_sync(t);
    SEC_ADD(SEC_SYNC);
  }
  // level Ls-1: pre-smoothing by the team
  {
    const int l = Ls - 1;
    for (int s = 1; s < nu; ++s) {
      with_rhs(w, l, [&](auto fl) {
        mg_sweep<T, DIM, KAPPA>(op.lv[l], w.e[l][ecur[l] ^ 1], w.e[l][ecur[l]], fl, t.g, t.S, t.bvs, t.col, omega,
                                (const T*)nullptr, rz);
      });
      ecur[l] ^= 1;
      SEC_ADD(l == 0 ? SEC_BAND : SEC_COARSE);
      team_sync(t);
      SEC_ADD(SEC_SYNC);
    }
  }
  // every CTA: restriction into its shared-memory level Ls, coarse cycle there
  {
    // the coarsest level: one node is solved exactly (e = f / d); a
    // hierarchy cut above it smooths its coarsest level by 2 nu damped
    // Jacobi sweeps from zero instead (a fixed symmetric polynomial)
    const bool exact = op.lv[L - 1].n == 1;
    const int l = Ls - 1;
    const T sc_ls = (Ls == L - 1 && exact) ? T(1) : omega;
    with_rhs(w, l, [&](auto fl) {
      mg_restrict<T, DIM, KAPPA>(op.lv[l], op.lv[Ls], w.e[l][ecur[l]], fl, sm.f[Ls], sm.e[Ls][0], t.tid, t.NT,
                                 t.bvs, t.col, sc_ls);
    });
    ecur[Ls] = 0;
    __syncthreads();
    for (int c = Ls; c < L - 1; ++c) {
      for (int s = 1; s < nu; ++s) {
        mg_sweep<T, DIM, KAPPA>(op.lv[c], sm.e[c][ecur[c] ^ 1], sm.e[c][ecur[c]], sm.f[c], t.tid, t.NT,
                                t.bvs, t.col, omega, (const T*)nullptr, rz);
        ecur[c] ^= 1;
        __syncthreads();
      }
      mg_restrict<T, DIM, KAPPA>(op.lv[c], op.lv[c + 1], sm.e[c][ecur[c]], sm.f[c], sm.f[c + 1],
                                 sm.e[c + 1][0], t.tid, t.NT, t.bvs, t.col, (c + 1 == L - 1 && exact) ? T(1) : omega);
      ecur[c + 1] = 0;
      __syncthreads();
    }
    if (!exact) {
      const int c = L - 1;
      for (int s = 1; s < 2 * nu; ++s) {
        mg_sweep<T, DIM, KAPPA>(op.lv[c], sm.e[c][ecur[c] ^ 1], sm.e[c][ecur[c]], sm.f[c], t.tid, t.NT,
                                t.bvs, t.col, omega, (const T*)nullptr, rz);
        ecur[c] ^= 1;
        __syncthreads();
      }
    }
    for (int c = L - 2; c >= Ls; --c) {
      mg_prolong<T, DIM>(op.lv[c], op.lv[c + 1], sm.e[c][ecur[c]], sm.e[c + 1][ecur[c + 1]], t.tid, t.NT,
                         t.bvs, t.col);
      __syncthreads();
      for (int s = 0; s < nu; ++s) {
        mg_sweep<T, DIM, KAPPA>(op.lv[c], sm.e[c][ecur[c] ^ 1], sm.e[c][ecur[c]], sm.f[c], t.tid, t.NT,
                                t.bvs, t.col, omega, (const T*)nullptr, rz);
        ecur[c] ^= 1;
        __syncthreads();
      }
    }
  }
  SEC_ADD(Ls == 1 ? SEC_RESTRICT : SEC_COARSE2);
  // up: prolongation from the CTA's own shared-memory level Ls, then the team levels
  for (int l = Ls - 1; l >= 0; --l) {
    if (l == Ls - 1) {
      // out of place: other CTAs may still be restricting from e[l][ecur]
      mg_prolong<T, DIM>(op.lv[l], op.lv[l + 1], w.e[l][ecur[l] ^ 1], sm.e[Ls][ecur[Ls]], t.g, t.S, t.bvs,
                         t.col, w.e[l][ecur[l]]);
      ecur[l] ^= 1;
    } else {
      mg_prolong<T, DIM>(op.lv[l], op.lv[l + 1], w.e[l][ecur[l]], w.e[l + 1][ecur[l + 1]], t.g, t.S, t.bvs,
                         t.col);
    }
    SEC_ADD(l == 0 ? SEC_BAND : SEC_COARSE);
    team_sync(t);
    SEC_ADD(SEC_SYNC);
    for (int s = 0; s < nu; ++s) {
      const bool last = (l == 0 && s == nu - 1);
      with_rhs(w, l, [&](auto fl) {
        mg_sweep<T, DIM, KAPPA>(op.lv[l], w.e[l][ecur[l] ^ 1], w.e[l][ecur[l]], fl, t.g, t.S, t.bvs, t.col, omega,
                                last ? (const T*)w.r : (const T*)nullptr, rz);
      });
      ecur[l] ^= 1;
      SEC_ADD(l == 0 ? SEC_BAND : SEC_COARSE);
      if (last) contribute(t, SL_RZ, (T)rz);
      SEC_ADD(SEC_REDUCE);
      team_sync(t);
      SEC_ADD(SEC_SYNC);
    }
  }
  return ecur[0];
}

// PCG iterations on (I + c L) x = b from a prepared state: f[0] = r holds the
// initial residual, e[0][0] its first smoother sweep, `done` whether this
// thread's column is already converged. Updates xt (+= alpha p; = alpha p on
// the first iteration if zero_init).
template <typename T, typename ES, typename TX, int DIM, bool KAPPA>
__device__ LRP_SOLVER_FN void pcg_iterate(const Team& t, const Op& op, const WSV<T, ES>& w, const SmemLv<T>& sm, TX* xt,
                            bool zero_init,
                            double tol2bb, bool& done, const SolveCfg& cfg, T omega, T scale0,
                            Ctr& ctr, double& rr_last) {
  const OpLevel& l0 = op.lv[0];
  const int items = l0.N << t.bvs;
  int it_count = 0;
  double rz_old = 0.0;
  bool all = __syncthreads_and(done);
  while (!all) {
    const int zc = vcycle<T, ES, DIM, KAPPA>(t, op, w, sm, omega, cfg.nu);
    SEC_T0();
    const ES* z = w.e[0][zc];
    const double rz = total_t<T>(t, SL_RZ);
    SEC_ADD(SEC_REDUCE);
    const T beta = (T)((it_count == 0 || done || !(rz_old > 0.0)) ? 0.0 : rz / rz_old);
    // phase A: p = z + beta p, q = A z + beta q, accumulate p.q
    double pq = 0.0;
    {
      LdT<ES, T> ld{z, t.bvs, t.col};
      T pqp = T(0);  // per-thread partial in the inner type
      batched_loop<V2<T>>(
          t.g, items, t.S,
          [&](int it) {
            const int p = it >> t.bvs;
            int i0, i1, i2;
            decomp<DIM>(l0, p, i0, i1, i2);
            T d;
            const T az = op_at<T, DIM, KAPPA>(l0, ld, p, i0, i1, i2, d);
            V2<T> r;
            if (it_count == 0) {
              r.a = cvt<T>(z[it]);
              r.b = az;
            } else {
              r.a = cvt<T>(z[it]) + beta * w.p[it];
              r.b = az + beta * w.q[it];
            }
            return r;
          },
          [&](int it, const V2<T>& r) {
            w.p[it] = r.a;
            w.q[it] = r.b;
            pqp += r.a * r.b;
          });
      pq = (double)pqp;
    }
    SEC_ADD(SEC_OTHER);
    contribute(t, SL_PQ, (T)pq);
    SEC_ADD(SEC_REDUCE);
    team_sync(t);
    SEC_ADD(SEC_SYNC);
    const double pqt = total_t<T>(t, SL_PQ);
    SEC_ADD(SEC_REDUCE);
    const T alpha = (T)((done || !(pqt > 0.0)) ? 0.0 : rz / pqt);
    // phase B: x += alpha p, r -= alpha q, first smoother sweep of the next V-cycle
    double rr = 0.0, rz1 = 0.0;
    {
      T rrp = T(0), rz1p = T(0);
      const bool fresh = zero_init && it_count == 0;
      struct XRE {
        TX x;
        T r, e;
      };
      batched_loop<XRE>(
          t.g, items, t.S,
          [&](int it) {
            const int p = it >> t.bvs;
            XRE v;
            v.x = fresh ? (TX)(alpha * w.p[it]) : (TX)(xt[it] + (TX)(alpha * w.p[it]));
            v.r = w.r[it] - alpha * w.q[it];
            v.e = scale0 * v.r * dinv_at<T, KAPPA>(l0, p);
            return v;
          },
          [&](int it, const XRE& v) {
            xt[it] = v.x;
            w.r[it] = v.r;
            rrp += v.r * v.r;
            w.e[0][0][it] = cst<ES>(v.e);
            if (op.L == 1) rz1p += v.r * v.e;
          });
      rr = (double)rrp;
      rz1 = (double)rz1p;
    }
    SEC_ADD(SEC_OTHER);
    contribute(t, SL_RR, (T)rr);
    if (op.L == 1) contribute(t, SL_RZ, (T)rz1);
    SEC_ADD(SEC_REDUCE);
    team_sync(t);
    SEC_ADD(SEC_SYNC);
    const double rrt = total_t<T>(t, SL_RR);
    SEC_ADD(SEC_REDUCE);
    if (!isfinite(rrt)) {
      ctr.status |= STAT_NONFINITE;
      done = true;
    }
    if (!done) rr_last = rrt;
    done = done || (rrt <= tol2bb);
    ++it_count;
    rz_old = rz;
    const bool capped = it_count >= cfg.maxit;
    all = __syncthreads_and(done) || capped;
    // the cap is a failure of the FP64 solve; an FP32 inner solve that stops
    // at it leaves the decision to the FP64 refinement around it
    if (capped && sizeof(TX) == sizeof(double) && !__syncthreads_and(done)) ctr.status |= STAT_NOCONV;
  }
  ctr.iters += it_count;
  ctr.iters_max = max(ctr.iters_max, it_count);
}

// Right-hand side at node p: bsrc (or 0) plus the adjoint source B^T d.
__device__ __forceinline__ double rhs_at(const SweepParams& P, const Team& t, const double* bsrc,
                                         const double* dsrc, int p, int it) {
  double b = bsrc ? bsrc[it] : 0.0;
  if (dsrc) {
    const int e0 = P.bt_ptr[p], e1 = P.bt_ptr[p + 1];
    for (int e = e0; e < e1; ++e) b += P.bt_w[e] * dsrc[(P.bt_idx[e] << t.bvs) + t.col];
  }
  return b;
}

// Solve (I + c L) x = b in FP64 (x0 = warm start or NULL = 0). Returns the
// index (in w.dbuf) of the solution buffer X1.
template <int DIM, bool KAPPA>
__device__ LRP_SOLVER_FN double* solve_fp64(const Team& t, const SweepParams& P, const Op& op,
                              const WSV<double>& w, const SmemLv<double>& sm, const double* bsrc,
                              const double* dsrc, const double* x0, double* X1, Ctr& ctr) {
  const OpLevel& l0 = op.lv[0];
  const int items = l0.N << t.bvs;
  const double omega = P.cfg.omega;
  const double scale0 = (op.L == 1) ? 1.0 : omega;
  double rr = 0.0, bb = 0.0, rz1 = 0.0;
  Ld<double> ld{x0, t.bvs, t.col};
  for (int it = t.g; it < items; it += t.S) {
    const int p = it >> t.bvs;
    int i0, i1, i2;
    decomp<DIM>(l0, p, i0, i1, i2);
    const double bp = rhs_at(P, t, bsrc, dsrc, p, it);
    double d, ax = 0.0;
    if (x0) ax = op_at<double, DIM, KAPPA>(l0, ld, p, i0, i1, i2, d);
    const double rv = bp - ax;
    w.r[it] = rv;
    X1[it] = x0 ? x0[it] : 0.0;
    const double e = scale0 * rv * dinv_at<double, KAPPA>(l0, p);
    w.e[0][0][it] = e;
    rr += rv * rv;
    bb += bp * bp;
    if (op.L == 1) rz1 += rv * e;
  }
  contribute(t, SL_RR, rr);
  contribute(t, SL_BB, bb);
  if (op.L == 1) contribute(t, SL_RZ, rz1);
  team_sync(t);
  const double rrt = total(t, SL_RR), bbt = total(t, SL_BB);
  const double tol2bb = P.cfg.rtol * P.cfg.rtol * bbt;
  bool done = rrt <= tol2bb;
  if (!(bbt > 0.0)) {
    for (int it = t.g; it < items; it += t.S) X1[it] = 0.0;
    done = true;
  }
  if (!isfinite(rrt) || !isfinite(bbt)) {
    ctr.status |= STAT_NONFINITE;
    done = true;
  }
  double rr_last = rrt;
  pcg_iterate<double, double, double, DIM, KAPPA>(t, op, w, sm, X1, false, tol2bb, done, P.cfg, omega,
                                          scale0, ctr, rr_last);
  ctr.max_res = fmax(ctr.max_res, bbt > 0.0 ? sqrt(rr_last / bbt) : 0.0);
  ctr.solves += 1;
  return X1;
}

// Solve (I + c L) x = b by FP64 iterative refinement around FP32 MG-PCG.
// Each FP32 inner problem is scaled by an exact power of two chosen so that
// its entries are O(1): deep in a sweep the state has decayed by many orders
// and the refinement residual by more, and unscaled FP32 products of such
// values underflow. The scale of refinement k is predicted from the residual
// of refinement k-1 (the inner solve reduces it by about inner_rtol); that of
// the first refinement from the previous solve's right-hand side.
template <int DIM, bool KAPPA, typename ES>
__device__ LRP_SOLVER_FN double* solve_mixed(const Team& t, const SweepParams& P, const Op& op,
                               const WSV<float, ES>& w, const SmemLv<float>& sm, const double* bsrc,
                               const double* dsrc, const double* x0, double* X1, double* X2,
                               Ctr& ctr) {
  const OpLevel& l0 = op.lv[0];
  const int items = l0.N << t.bvs;
  const float omega = (float)P.cfg.omega;
  const float scale0 = (op.L == 1) ? 1.f : omega;
  const double* xa = x0;
  double* tgt = X1;
  double* oth = X2;
  bool done = false;
  double bbt = 0.0;
  int ref = 0;
  const double inv_n = 1.0 / (double)l0.N;
  double sc = ctr.mix_scale;  // scale of the float residual written in this refinement
  double inv_sc_c = 1.0;      // 1 / scale of the current inner correction c
  for (;; ++ref) {
    const bool first = (ref == 0);
    double rr = 0.0, bb = 0.0, rz1 = 0.0;
    SEC_T0();
    LdSum<float> ls{xa, first ? (const float*)nullptr : w.c, t.bvs, t.col, inv_sc_c};
    struct Ref {
      double bp, rd, x;
    };
    batched_loop<Ref>(
        t.g, items, t.S,
        [&](int it) {
          const int p = it >> t.bvs;
          int i0, i1, i2;
          decomp<DIM>(l0, p, i0, i1, i2);
          Ref v;
          if (first)
            v.bp = rhs_at(P, t, bsrc, dsrc, p, it);
          else
            v.bp = dsrc ? w.bd[it] : (bsrc ? bsrc[it] : 0.0);
          double d, ax = 0.0;
          if (xa || !first) ax = op_at<double, DIM, KAPPA>(l0, ls, p, i0, i1, i2, d);
          v.rd = v.bp - ax;
          v.x = ls(p);
          return v;
        },
        [&](int it, const Ref& v) {
          const int p = it >> t.bvs;
          if (first) {
            if (dsrc) w.bd[it] = v.bp;
            bb += v.bp * v.bp;
          }
          tgt[it] = v.x;
          const float rf = (float)(v.rd * sc);
          w.r[it] = rf;
          const float e = scale0 * rf * dinv_at<float, KAPPA>(l0, p);
          w.e[0][0][it] = cst<ES>(e);
          rr += v.rd * v.rd;
          if (op.L == 1) rz1 += (double)(rf * e);
        });
    SEC_ADD(SEC_REFINE);
    contribute(t, SL_RRD, rr);
    if (first) contribute(t, SL_BBD, bb);
    if (op.L == 1) contribute(t, SL_RZ, (float)rz1);
    SEC_ADD(SEC_REDUCE);
    team_sync(t);
    SEC_ADD(SEC_SYNC);
    const double rrt = total(t, SL_RRD);
    if (first) {
      bbt = total(t, SL_BBD);
      if (!(bbt > 0.0)) {
        for (int it = t.g; it < items; it += t.S) tgt[it] = 0.0;
        done = true;
      }
      ctr.mix_scale = pow2_inv(sqrt(bbt * inv_n));
    }
    if (!isfinite(rrt)) {
      ctr.status |= STAT_NONFINITE;
      done = true;
    }
    done = done || (rrt <= P.cfg.rtol * P.cfg.rtol * bbt);
    if (done) ctr.max_res = fmax(ctr.max_res, bbt > 0.0 ? sqrt(rrt / bbt) : 0.0);
    const bool all = __syncthreads_and(done);
    if (all) break;
    if (ref >= P.cfg.maxref) {
      // the refinement cap: the residual reached is reported with the status
      if (!done) ctr.max_res = fmax(ctr.max_res, bbt > 0.0 ? sqrt(rrt / bbt) : 0.0);
      ctr.status |= STAT_NOCONV;
      break;
    }
    bool idone = done;
    const double itol2 = P.cfg.inner_rtol * P.cfg.inner_rtol * rrt * sc * sc;
    double rr_in = rrt * sc * sc;
    pcg_iterate<float, ES, float, DIM, KAPPA>(t, op, w, sm, w.c, true, itol2, idone, P.cfg, omega, scale0,
                                          ctr, rr_in);
    xa = tgt;
    double* tmp = tgt;
    tgt = oth;
    oth = tmp;
    inv_sc_c = 1.0 / sc;
    sc = pow2_inv(P.cfg.inner_rtol * sqrt(rrt * inv_n));
  }
  ctr.refines += ref;
  ctr.refine_max = max(ctr.refine_max, ref);
  ctr.solves += 1;
  return tgt;
}

// ((I + c L) v)_p for the convection-diffusion operator, L = nu (-Laplace) +
// w . grad with first-order upwind differences (Sec. 6.2, upwind in place of
// the paper's SUPG): the diffusion part as op_at (ch2 = c nu / h^2), and per
// axis with wind, |c w_a / h| on the diagonal and -|c w_a / h| at the
// upstream neighbour (the low side for w_a > 0). transpose: (I + c L)^T, the
// same coefficient at the downstream neighbour (the adjoint sweep).
template <int DIM, class LD>
__device__ __forceinline__ double op_conv_at(const OpLevel& lv, const LD& ld, int p, int i0, int i1, int i2,
                                             bool transpose, double& diag) {
  double v = op_at<double, DIM, false>(lv, ld, p, i0, i1, i2, diag);
  const int n = lv.n;
  const int ii[3] = {i0, i1, i2};
  int stride = 1;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    const double cw = lv.cw[a];
    if (cw != 0.0) {
      const double c = fabs(cw);
      // upstream side: low (-1) for w_a > 0; the transpose reads the other side
      const bool low = (cw > 0.0) != transpose;
      const bool inside = low ? ii[a] > 0 : ii[a] < n - 1;
      v += c * ld(p) - (inside ? c * ld(low ? p - stride : p + stride) : 0.0);
      diag += c;
    }
    stride *= n;
  }
  return v;
}

// Solve (I + c L) x = b for the nonsymmetric convection-diffusion step by
// BiCGStab (van der Vorst, 1992) with the Jacobi preconditioner applied on
// the right, in FP64: five phases and team barriers per iteration (the two
// operator applications need their input's neighbours). Vectors: x in X1,
// r in w.r, shadow residual r^ = r_0 in w.c, p in w.p, v in w.q,
// D^-1 p and D^-1 s in the two finest smoother buffers, s in place of r,
// t in X2.
template <int DIM>
__device__ LRP_SOLVER_FN double* solve_bicgstab(const Team& t, const SweepParams& P, const Op& op,
                                                const WSV<double>& w, const double* bsrc, const double* dsrc,
                                                const double* x0, double* X1, double* X2, bool transpose,
                                                Ctr& ctr) {
  const OpLevel& l0 = op.lv[0];
  const int items = l0.N << t.bvs;
  const double dinv = l0.dinv;
  double* r = w.r;
  double* rh = w.c;
  double* pv = w.p;
  double* vv = w.q;
  double* ph = w.e[0][0];
  double* sh = w.e[0][1];
  double* tv = X2;
  auto decomp_at = [&](int it, int& p, int& i0, int& i1, int& i2) {
    p = it >> t.bvs;
    decomp<DIM>(l0, p, i0, i1, i2);
  };
  // r0 = b - A x0, r^ = r0, x = x0
  double rr = 0.0, bb = 0.0;
  {
    Ld<double> ld{x0, t.bvs, t.col};
    for (int it = t.g; it < items; it += t.S) {
      int p, i0, i1, i2;
      decomp_at(it, p, i0, i1, i2);
      const double bp = rhs_at(P, t, bsrc, dsrc, p, it);
      double d, ax = 0.0;
      if (x0) ax = op_conv_at<DIM>(l0, ld, p, i0, i1, i2, transpose, d);
      const double rv = bp - ax;
      r[it] = rv;
      rh[it] = rv;
      X1[it] = x0 ? x0[it] : 0.0;
      pv[it] = 0.0;
      vv[it] = 0.0;
      rr += rv * rv;
      bb += bp * bp;
    }
  }
  contribute(t, SL_RR, rr);
  contribute(t, SL_BBD, bb);
  team_sync(t);
  double rrt = total(t, SL_RR);
  const double bbt = total(t, SL_BBD);
  const double tol2 = P.cfg.rtol * P.cfg.rtol * bbt;
  bool done = !(bbt > 0.0) || rrt <= tol2;
  if (!isfinite(rrt) || !isfinite(bbt)) {
    ctr.status |= STAT_NONFINITE;
    done = true;
  }
  double rho = rrt;  // (r^, r0) = ||r0||^2
  double alpha = 1.0, omg = 1.0, rho_old = 1.0;
  int it_count = 0;
  bool all = __syncthreads_and(done);
  while (!all) {
    const double beta = (it_count == 0 || done) ? 0.0 : (rho / rho_old) * (alpha / omg);
    const double omg_p = (it_count == 0 || done) ? 0.0 : omg;
    // phase A: p = r + beta (p - omega v); p^ = D^-1 p
    for (int it = t.g; it < items; it += t.S) {
      const double pn = r[it] + beta * (pv[it] - omg_p * vv[it]);
      pv[it] = pn;
      ph[it] = dinv * pn;
    }
    team_sync(t);
    // phase B: v = A p^, (r^, v)
    double rhv = 0.0;
    {
      Ld<double> ld{ph, t.bvs, t.col};
      for (int it = t.g; it < items; it += t.S) {
        int p, i0, i1, i2;
        decomp_at(it, p, i0, i1, i2);
        double d;
        const double v = op_conv_at<DIM>(l0, ld, p, i0, i1, i2, transpose, d);
        vv[it] = v;
        rhv += rh[it] * v;
      }
    }
    contribute(t, SL_PQ, rhv);
    team_sync(t);
    const double rhvt = total(t, SL_PQ);
    if (!done && !(fabs(rhvt) > 0.0)) {  // breakdown
      ctr.status |= STAT_NOCONV;
      done = true;
    }
    alpha = done ? 0.0 : rho / rhvt;
    // phase C: s = r - alpha v (in place of r); s^ = D^-1 s
    for (int it = t.g; it < items; it += t.S) {
      const double sv = r[it] - alpha * vv[it];
      r[it] = sv;
      sh[it] = dinv * sv;
    }
    team_sync(t);
    // phase D: t = A s^, (t, s), (t, t)
    double ts = 0.0, tt = 0.0;
    {
      Ld<double> ld{sh, t.bvs, t.col};
      for (int it = t.g; it < items; it += t.S) {
        int p, i0, i1, i2;
        decomp_at(it, p, i0, i1, i2);
        double d;
        const double tvv = op_conv_at<DIM>(l0, ld, p, i0, i1, i2, transpose, d);
        tv[it] = tvv;
        ts += tvv * r[it];
        tt += tvv * tvv;
      }
    }
    contribute(t, 6, ts);
    contribute(t, 7, tt);
    team_sync(t);
    const double tst = total(t, 6), ttt = total(t, 7);
    omg = (done || !(ttt > 0.0)) ? 0.0 : tst / ttt;
    // phase E: x += alpha p^ + omega s^, r = s - omega t, (r^, r), (r, r)
    double rhr = 0.0;
    rr = 0.0;
    for (int it = t.g; it < items; it += t.S) {
      X1[it] += alpha * ph[it] + omg * sh[it];
      const double rn = r[it] - omg * tv[it];
      r[it] = rn;
      rhr += rh[it] * rn;
      rr += rn * rn;
    }
    contribute(t, SL_RZ, rhr);
    contribute(t, SL_RR, rr);
    team_sync(t);
    const double rhrt = total(t, SL_RZ);
    rrt = total(t, SL_RR);
    if (!isfinite(rrt)) {
      ctr.status |= STAT_NONFINITE;
      done = true;
    }
    const bool conv = rrt <= tol2;
    if (!done && !conv && !(omg != 0.0 && fabs(rhrt) > 0.0)) {  // breakdown
      ctr.status |= STAT_NOCONV;
      done = true;
    }
    done = done || conv;
    rho_old = rho;
    rho = rhrt;
    ++it_count;
    const bool capped = it_count >= P.cfg.maxit;
    all = __syncthreads_and(done) || capped;
    if (capped && !__syncthreads_and(done)) ctr.status |= STAT_NOCONV;
  }
  ctr.iters += it_count;
  ctr.iters_max = max(ctr.iters_max, it_count);
  ctr.max_res = fmax(ctr.max_res, bbt > 0.0 ? sqrt(rrt / bbt) : 0.0);
  ctr.solves += 1;
  return X1;
}

template <typename T, int DIM, bool MIXED, typename ES>
__device__ __forceinline__ double* solve_any(const Team& t, const SweepParams& P, const Op& op,
                                             const WSV<T, ES>& w, const SmemLv<T>& sm, const double* bsrc,
                                             const double* dsrc, const double* x0, double* X1,
                                             double* X2, Ctr& ctr, bool transpose = false) {
  if constexpr (MIXED) {
    if (op.has_kappa)
      return solve_mixed<DIM, true, ES>(t, P, op, w, sm, bsrc, dsrc, x0, X1, X2, ctr);
    return solve_mixed<DIM, false, ES>(t, P, op, w, sm, bsrc, dsrc, x0, X1, X2, ctr);
  } else {
    if (op.conv) return solve_bicgstab<DIM>(t, P, op, w, bsrc, dsrc, x0, X1, X2, transpose, ctr);
    if (op.has_kappa) return solve_fp64<DIM, true>(t, P, op, w, sm, bsrc, dsrc, x0, X1, ctr);
    return solve_fp64<DIM, false>(t, P, op, w, sm, bsrc, dsrc, x0, X1, ctr);
  }
}

__device__ __forceinline__ int buf_index(const double* const* b, const double* x) {
  return x == b[0] ? 0 : (x == b[1] ? 1 : 2);
}

// Gamma_prior^{1/2} x = sqrt(gamma) x for the identity prior: the next state
// buffer receives the scaled copy; returns its index.
__device__ __forceinline__ int prior_scale_copy(const Team& t, const SweepParams& P, double* const* dbuf, int cur,
                                                int items) {
  const int nxt = (cur + 1) % 3;
  for (int it = t.g; it < items; it += t.S) dbuf[nxt][it] = P.prior_scale * dbuf[cur][it];
  team_sync(t);
  return nxt;
}

template <typename T, int DIM, bool MIXED, typename ES = T>
__global__ void __launch_bounds__(512, 1) sweep_kernel(const SweepParams P) {
  __shared__ double s_red[2 * NSLOT * LRP_MAXBV];
  __shared__ double s_redw[32 * LRP_MAXBV];
  __shared__ float s_redf[2 * NSLOT * LRP_MAXBV];
  __shared__ float s_redwf[32 * LRP_MAXBV];
  extern __shared__ __align__(16) unsigned char s_dyn[];
  Team t;
  t.C = P.C;
  t.rank = (P.C > 1) ? (int)cg::this_cluster().block_rank() : 0;
  t.NT = blockDim.x;
  t.tid = threadIdx.x;
  t.g = t.rank * t.NT + t.tid;
  t.S = t.C * t.NT;
  t.BV = P.BV;
  t.bvs = P.bv_shift;
  t.col = t.g & (P.BV - 1);
  t.red = s_red;
  t.redw = s_redw;
  t.redf = s_redf;
  t.redwf = s_redwf;
  t.phase = 0;
  const int team = blockIdx.x / P.C;
#ifdef LRP_SECTION_TIMERS
  if (threadIdx.x < 12) s_sec[threadIdx.x] = 0;
  const long long k_t0 = clock64();
#endif
  char* base = P.ws + (size_t)team * P.team_bytes;
  WSV<T, ES> w;
  for (int k = 0; k < 3; ++k) w.dbuf[k] = (double*)(base + P.off_dbuf[k]);
  w.bd = (double*)(base + P.off_bd);
  w.obs = (double*)(base + P.off_obs);
  w.r = (T*)(base + P.off_r);
  w.p = (T*)(base + P.off_p);
  w.q = (T*)(base + P.off_q);
  w.c = (T*)(base + P.off_c);
  w.e[0][0] = (ES*)(base + P.off_e0[0]);
  w.e[0][1] = (ES*)(base + P.off_e0[1]);
  if constexpr (std::is_same<ES, T>::value)
    w.f[0] = w.r;  // level 0's right-hand side is r
  else
    w.f[0] = nullptr;
  for (int l = 1; l < LRP_MAXLEV; ++l) {
    w.e[l][0] = (ES*)(base + P.off_e[l][0]);
    w.e[l][1] = (ES*)(base + P.off_e[l][1]);
    w.f[l] = (ES*)(base + P.off_f[l]);
  }
  if (P.poison) {
    for (size_t i = t.tid; i < P.smem_bytes / sizeof(T); i += t.NT) ((T*)s_dyn)[i] = T(NAN);
    __syncthreads();
  }
  SmemLv<T> sm;
  for (int l = 0; l < LRP_MAXLEV; ++l) {
    sm.e[l][0] = (T*)(s_dyn + P.smem_off[l][0]);
    sm.e[l][1] = (T*)(s_dyn + P.smem_off[l][1]);
    sm.f[l] = (T*)(s_dyn + P.smem_off[l][2]);
  }
  const int gcol = team * P.BV + t.col;
  const bool valid = gcol < P.nvec;
  const int N0 = P.step.lv[0].N;
  const int items0 = N0 << t.bvs;
  Ctr ctr;
  int cur = (P.stages & ST_LOAD_X) ? 0 : min(max(P.end_buf[team], 0), 2);

  if (P.stages & ST_LOAD_X) {
    for (int it = t.g; it < items0; it += t.S) {
      const int p = it >> t.bvs;
      w.dbuf[0][it] = valid ? P.X[(size_t)gcol * P.ldx + p] : 0.0;
    }
    team_sync(t);
  }
  if (P.stages & ST_LOAD_D) {
    const int nd = (P.n_obs * P.n_steps) << t.bvs;
    for (int it = t.g; it < nd; it += t.S) {
      const int e = it >> t.bvs;
      w.obs[it] = valid ? P.Din[(size_t)gcol * P.lddin + e] : 0.0;
    }
    team_sync(t);
  }
  if (P.stages & ST_PRIOR_IN) {
    double* X1 = w.dbuf[(cur + 1) % 3];
    double* X2 = w.dbuf[(cur + 2) % 3];
    if (P.prior_scale > 0.0) {
      cur = prior_scale_copy(t, P, w.dbuf, cur, items0);
    } else {
      double* res = solve_any<T, DIM, MIXED, ES>(t, P, P.prior, w, sm, w.dbuf[cur], nullptr, nullptr, X1,
                                             X2, ctr);
      cur = buf_index(w.dbuf, res);
    }
  }
  if (P.stages & ST_SHIFTED) {
    // one solve with this column's own operator (one column per team): the
    // block-diagonal preconditioner of the alternating space-time solver
    double* X1 = w.dbuf[(cur + 1) % 3];
    double* X2 = w.dbuf[(cur + 2) % 3];
    double* res = solve_any<T, DIM, MIXED, ES>(t, P, P.team_ops[team], w, sm, w.dbuf[cur], nullptr, nullptr, X1, X2,
                                           ctr, P.shift_transpose != 0);
    cur = buf_index(w.dbuf, res);
  }
  if (P.stages & ST_FORWARD) {
    for (int n = P.t_begin + 1; n <= P.t_end; ++n) {
      if (P.stages & ST_SOURCE) {
        // y_{n-1} + tau u_n with u_n = W V[n-1, :]^T (also the solve's
        // start). The previous step's fused observation reads y_{n-1} with no
        // barrier after it: wait for it before y_{n-1} is overwritten.
        team_sync(t);
        for (int it = t.g; it < items0; it += t.S) {
          const int p = it >> t.bvs;
          double u = 0.0;
          for (int i = 0; i < P.src_r; ++i)
            u += P.src_W[(size_t)i * P.src_ldw + p] * P.src_V[(size_t)i * P.src_ldv + n - 1];
          w.dbuf[cur][it] += P.src_scale * u;
        }
        team_sync(t);
      }
      double* X1 = w.dbuf[(cur + 1) % 3];
      double* X2 = w.dbuf[(cur + 2) % 3];
      double* res = solve_any<T, DIM, MIXED, ES>(t, P, P.step, w, sm, w.dbuf[cur], nullptr, w.dbuf[cur],
                                             X1, X2, ctr);
      cur = buf_index(w.dbuf, res);
      // fused observation d_n = B y_n (/ sigma^2 for the Hessian); no barrier
      // needed: the next phase only reads y_n as well
      if ((P.stages & ST_FORWARD) && P.n_steps > 0 && (n % P.obs_every) == 0 &&
          n / P.obs_every <= P.n_steps) {
        const int k = n / P.obs_every - 1;
        const int no = P.n_obs << t.bvs;
        for (int it = t.g; it < no; it += t.S) {
          const int s = it >> t.bvs;
          double y = 0.0;
          for (int c = 0; c < 8; ++c) {
            const int node = P.obs_node[s * 8 + c];
            if (node >= 0) y += P.obs_w[s * 8 + c] * res[(node << t.bvs) + t.col];
          }
          w.obs[((size_t)k * P.n_obs << t.bvs) + it] = y * P.inv_sigma2;
          if ((P.stages & ST_STORE_D) && valid) P.Dout[(size_t)gcol * P.lddout + k * P.n_obs + s] = y;
        }
      }
      if (P.stages & ST_TRAJ) {
        const int chunk_pos = n - P.t_begin - 1;
        if (valid) {
          double* dst = P.traj + ((size_t)gcol * P.traj_cols + chunk_pos) * P.traj_ld;
          for (int it = t.g; it < items0; it += t.S) dst[it >> t.bvs] = res[it];
        }
      }
    }
  }
  if (P.stages & ST_FORWARD) {
    // the last observation phase has no barrier of its own: the adjoint
    // source reads those values next
    team_sync(t);
  }
  if (P.stages & ST_ADJOINT) {
    const double* q = nullptr;  // q_{nt+1} = 0
    for (int n = P.adj_begin; n >= 1; --n) {
      const bool obs = (n % P.obs_every) == 0 && n / P.obs_every <= P.n_steps;
      if (!q && !obs) continue;
      const double* dsrc = obs ? w.obs + ((size_t)(n / P.obs_every - 1) * P.n_obs << t.bvs) : nullptr;
      const int qi = q ? buf_index(w.dbuf, q) : cur;
      double* X1 = w.dbuf[(qi + 1) % 3];
      double* X2 = w.dbuf[(qi + 2) % 3];
      double* res = solve_any<T, DIM, MIXED, ES>(t, P, P.step, w, sm, q, dsrc, q, X1, X2, ctr, true);
      q = res;
      if ((P.stages & ST_TRAJ_ADJ) && valid) {
        // steps after the last observation hold q_n = 0: the caller zeroes the buffer
        double* dst = P.traj + ((size_t)gcol * P.traj_cols + (n - 1)) * P.traj_ld;
        for (int it = t.g; it < items0; it += t.S) dst[it >> t.bvs] = res[it];
      }
    }
    if (q) {
      cur = buf_index(w.dbuf, q);
    } else {
      for (int it = t.g; it < items0; it += t.S) w.dbuf[cur][it] = 0.0;
      team_sync(t);
    }
  }
  if (P.stages & ST_PRIOR_OUT) {
    double* X1 = w.dbuf[(cur + 1) % 3];
    double* X2 = w.dbuf[(cur + 2) % 3];
    if (P.prior_scale > 0.0) {
      cur = prior_scale_copy(t, P, w.dbuf, cur, items0);
    } else {
      double* res = solve_any<T, DIM, MIXED, ES>(t, P, P.prior, w, sm, w.dbuf[cur], nullptr, nullptr, X1,
                                             X2, ctr);
      cur = buf_index(w.dbuf, res);
    }
  }
  if ((P.stages & ST_STORE_Y) && valid) {
    for (int it = t.g; it < items0; it += t.S) P.Y[(size_t)gcol * P.ldy + (it >> t.bvs)] = w.dbuf[cur][it];
  }
  // keep every CTA's shared memory alive until all DSMEM readers are done
  team_sync(t);
  if (t.rank == 0 && t.tid == 0) {
    P.end_buf[team] = cur;
    atomicAdd(&P.stats->solves, (unsigned long long)ctr.solves);
    atomicAdd(&P.stats->iters, (unsigned long long)ctr.iters);
    atomicAdd(&P.stats->refines, (unsigned long long)ctr.refines);
    atomicMax(&P.stats->iters_max, ctr.iters_max);
    atomicMax(&P.stats->refine_max, ctr.refine_max);
    if (ctr.status) atomicOr(&P.stats->status, ctr.status);
  }
  if (t.rank == 0 && t.tid < t.BV && valid) {
    atomicMax(&P.stats->max_rel_res_bits, (unsigned long long)__double_as_longlong(ctr.max_res));
  }
#ifdef LRP_SECTION_TIMERS
  if (team == 0 && t.rank == 0 && t.tid == 0 && P.section_cycles) {
    for (int k = 0; k < 11; ++k) P.section_cycles[k] = s_sec[k];
    P.section_cycles[11] = (unsigned long long)(clock64() - k_t0);
  }
#endif
}

// The shared-memory cap of a kernel is one value per function: it is always
// set to the device's opt-in maximum (the same value from every thread), so
// concurrent launchers with different shared-memory sizes cannot lower it
// under one another; each launch states its own size.
// (the opt-in per-block maximum less the kernel's static shared memory)
template <class K>
inline int smem_dynamic_max(K kern) {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) return 0;
  return v - (int)fa.sharedSizeBytes;
}

template <typename T, int DIM, bool MIXED, typename ES = T>
static cudaError_t prepare_sweep(size_t smem) {
  auto kern = sweep_kernel<T, DIM, MIXED, ES>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  const int cap = smem_dynamic_max(kern);
  if ((long long)smem > cap) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
}

template <typename T, int DIM, bool MIXED, typename ES = T>
cudaError_t launch_sweep(const SweepParams& prm, cudaStream_t stream) {
  auto kern = sweep_kernel<T, DIM, MIXED, ES>;
  cudaError_t e = prepare_sweep<T, DIM, MIXED, ES>(prm.smem_bytes);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(prm.n_teams * prm.C);
  cfg.blockDim = dim3(prm.NT);
  cfg.dynamicSmemBytes = prm.smem_bytes;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  int na = 0;
  if (prm.C > 1) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = prm.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    na = 1;
  }
  cfg.attrs = attr;
  cfg.numAttrs = na;
  return cudaLaunchKernelEx(&cfg, kern, prm);
}

// How many teams of C CTAs (NT threads, smem dynamic bytes each) can be
// resident at once: the sweep keeps every team resident for its whole
// lifetime, so a launch with more teams than this runs in waves.
template <typename T, int DIM, bool MIXED, typename ES = T>
int max_resident_teams(int C, int NT, size_t smem, int sm_count) {
  auto kern = sweep_kernel<T, DIM, MIXED, ES>;
  if (prepare_sweep<T, DIM, MIXED, ES>(smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (C == 1) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return per_sm * sm_count;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C * 64);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

}  // namespace lrp
