// Shared-memory-resident sweep kernel for 2D grids with kappa = 1, one column
// per team, FP32 multigrid-PCG inside FP64 iterative refinement.
//
// A team is a thread-block cluster of C CTAs. CTA k owns the band of rows
// [r0_k, r1_k) of the finest grid, r0_k = k n / C. Its share of every inner
// vector of the finest level (smoother iterates E0/E1, residual R, search
// direction P, A P = Q, inner solution X) lives in its shared memory, as rows
// of pitch n+1 with HALO rows above and below; after computing its own rows a
// CTA copies its first and last HALO rows into the halos of its neighbours
// through distributed shared memory (st.shared::cluster), so the next phase
// reads every neighbour value locally. Columns -1 and n of a row are a zero
// padding element (one leading pad element before the first row); halo rows
// outside the grid stay zero: the Dirichlet data need no index checks.
// All coarse levels are solved by every CTA redundantly in its own shared
// memory: the restriction of the finest residual is computed band by band
// and all-gathered into every CTA's coarse right-hand side.
// Phases are separated by cluster barriers (release/acquire), and each phase
// that writes a halo-exchanged vector writes the other one of a ping-pong pair
// (or a vector nobody reads in that phase), so no neighbour reads a halo that
// is being overwritten.
// The FP64 state of the implicit-Euler sweep (solution, right-hand side,
// observations) stays in global memory: it is touched once per refinement.
#pragma once

#include "lrp_sweep_kernel.cuh"

namespace lrp {

constexpr int FAST_HALO = 2;

// Optional section timers (build with -DLRP_SECTION_TIMERS): thread 0 of each
// CTA accumulates clock64() cycles per section into shared memory; CTA 0 of
// team 0 writes them to SweepParams::section_cycles at exit.
#ifdef LRP_SECTION_TIMERS
__shared__ unsigned long long s_sec[8];
#define SEC_T0() long long _sec_t0 = clock64()
#define SEC_ADD(k)                                   \
  do {                                               \
    if (threadIdx.x == 0) {                          \
      long long _t = clock64();                      \
      s_sec[k] += (unsigned long long)(_t - _sec_t0); \
      _sec_t0 = _t;                                  \
    }                                                \
  } while (0)
#define SEC_RESET() _sec_t0 = clock64()
#else
#define SEC_T0()
#define SEC_ADD(k)
#define SEC_RESET()
#endif
enum { SEC_BAND = 0, SEC_SYNC = 1, SEC_COARSE = 2, SEC_REFINE = 3, SEC_REDUCE = 4, SEC_OTHER = 5 };

struct Band {
  int n, r0, r1, pitch;  // grid size, own rows, row pitch (n + 1)
  int rank, C;
  int r0p, r0n;          // first row of the previous / next CTA's band
  int warp, lane, nwarp;
};

// Address of (row, col) in a band array whose band starts at row b0.
__device__ __forceinline__ int bidx(const Band& b, int b0, int row, int col) {
  return (row - b0 + FAST_HALO) * b.pitch + col;
}

// A band array with the addresses of the same array in the previous and next
// CTA of the team (NULL at the ends), for halo stores.
struct BArr {
  float* a;
  float* prev;
  float* next;
};

__device__ __forceinline__ BArr barr(const Band& b, float* A) {
  BArr r;
  r.a = A;
  r.prev = b.rank > 0 ? cg::this_cluster().map_shared_rank(A, b.rank - 1) : nullptr;
  r.next = b.rank < b.C - 1 ? cg::this_cluster().map_shared_rank(A, b.rank + 1) : nullptr;
  return r;
}

// Store v at (row, col) locally and, for boundary rows, into the halo of the
// neighbour that needs it.
__device__ __forceinline__ void bstore(const Band& b, const BArr& A, int row, int col, float v) {
  A.a[bidx(b, b.r0, row, col)] = v;
  if (A.prev && row < b.r0 + FAST_HALO) A.prev[bidx(b, b.r0p, row, col)] = v;
  if (A.next && row >= b.r1 - FAST_HALO) A.next[bidx(b, b.r0n, row, col)] = v;
}

// (I + c L) v at (row, col) for a band array (kappa = 1).
__device__ __forceinline__ float band_op(const Band& b, const float* A, int row, int col, float ch2,
                                         float d) {
  const int i = bidx(b, b.r0, row, col);
  return d * A[i] - ch2 * (A[i - 1] + A[i + 1] + A[i - b.pitch] + A[i + b.pitch]);
}

template <class F>
__device__ __forceinline__ void for_own(const Band& b, F f) {
  for (int row = b.r0 + b.warp; row < b.r1; row += b.nwarp)
    for (int col = b.lane; col < b.n; col += 32) f(row, col);
}

struct FastVec {
  float* E[2];
  float* R;
  float* P;
  float* Q;
  float* X;
};

// One damped Jacobi sweep on the band: Eo = Ei + omega (R - A Ei) / d.
__device__ __forceinline__ void fast_sweep(const Band& b, const FastVec& v, int cur, float ch2, float d,
                                           float dinv, float omega, bool acc_rz, double& rz) {
  const float* Ei = v.E[cur];
  const BArr Eo = barr(b, v.E[cur ^ 1]);
  float acc = 0.f;  // per-thread partial in FP32 (FP64 is a slow pipe here)
  for_own(b, [&](int row, int col) {
    const int i = bidx(b, b.r0, row, col);
    const float e = Ei[i] + omega * (v.R[i] - band_op(b, Ei, row, col, ch2, d)) * dinv;
    bstore(b, Eo, row, col, e);
    if (acc_rz) acc += v.R[i] * e;
  });
  rz += (double)acc;
}

// ---- coarse levels: dense copies in every CTA's shared memory, padded
// layout: pitch n+1, one zero row above and below, one leading pad element,
// so (row, col) sits at (row + 1) * (n + 1) + col + 1 and every stencil
// neighbour of an interior node is addressable without checks.
__device__ __forceinline__ int cidx(int n, int row, int col) { return (row + 1) * (n + 1) + col + 1; }

template <class F>
__device__ __forceinline__ void for_all(int n, int warp, int lane, int nwarp, F f) {
  for (int row = warp; row < n; row += nwarp)
    for (int col = lane; col < n; col += 32) f(row, col);
}

__device__ __forceinline__ float cop(const float* A, int n, int i, float ch2, float d) {
  return d * A[i] - ch2 * (A[i - 1] + A[i + 1] + A[i - (n + 1)] + A[i + (n + 1)]);
}

// Jacobi sweep on a coarse level: eo = ei + omega (f - A ei) / d
__device__ __forceinline__ void csweep(const Band& b, const OpLevel& lv, float* eo, const float* ei, const float* f,
                                       float omega) {
  const int n = lv.n;
  const float ch2 = (float)lv.ch2, d = 1.f + 4.f * ch2, dinv = (float)lv.dinv;
  for_all(n, b.warp, b.lane, b.nwarp, [&](int row, int col) {
    const int i = cidx(n, row, col);
    eo[i] = ei[i] + omega * (f[i] - cop(ei, n, i, ch2, d)) * dinv;
  });
}

// Full-weighting restriction of f - A e from level lf to lc, and ec = sc fc / d
__device__ __forceinline__ void crestrict(const Band& b, const OpLevel& lf, const OpLevel& lc, const float* ef,
                                          const float* ff, float* fc, float* ec, float sc) {
  const int nf = lf.n, nc = lc.n;
  const float ch2 = (float)lf.ch2, d = 1.f + 4.f * ch2, dinvc = (float)lc.dinv;
  for_all(nc, b.warp, b.lane, b.nwarp, [&](int J, int I) {
    float acc = 0.f;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int i = cidx(nf, 2 * J + 1 + dy, 2 * I + 1 + dx);
        acc += (dx == 0 ? 0.5f : 0.25f) * (dy == 0 ? 0.5f : 0.25f) * (ff[i] - cop(ef, nf, i, ch2, d));
      }
    const int k = cidx(nc, J, I);
    fc[k] = acc;
    ec[k] = sc * acc * dinvc;
  });
}

// Bilinear value of the coarse field ec (level with nc nodes, padded) at fine
// node (row, col) of the level below it (pads give the zero boundary).
__device__ __forceinline__ float cinterp(const float* ec, int nc, int row, int col) {
  const int cy0 = (row - 1) >> 1, cx0 = (col - 1) >> 1;  // floor((row-1)/2): -1 for row 0
  const float* base = ec + cidx(nc, cy0, cx0);
  if (row & 1) {
    if (col & 1) return base[0];
    return 0.5f * (base[0] + base[1]);
  }
  if (col & 1) return 0.5f * (base[0] + base[nc + 1]);
  return 0.25f * (base[0] + base[1] + base[nc + 1] + base[nc + 2]);
}

// e += P ec on a coarse level (in place)
__device__ __forceinline__ void cprolong(const Band& b, const OpLevel& lf, const OpLevel& lc, float* ef,
                                         const float* ec) {
  const int nf = lf.n, nc = lc.n;
  for_all(nf, b.warp, b.lane, b.nwarp, [&](int row, int col) { ef[cidx(nf, row, col)] += cinterp(ec, nc, row, col); });
}

// Coarse rows J whose fine centre row 2J+1 lies in this band: full-weighting
// restriction of the residual R - A E into every CTA's copy of f1 (padded
// coarse layout).
__device__ __forceinline__ void fast_restrict(const Band& b, const FastVec& v, int cur, float ch2, float d,
                                              float* f1, int n1) {
  const float* E = v.E[cur];
  int J0 = b.r0 / 2;  // smallest J with 2J+1 >= r0
  if (2 * J0 + 1 < b.r0) ++J0;
  for (int J = J0 + b.warp; 2 * J + 1 < b.r1 && J < n1; J += b.nwarp) {
    for (int I = b.lane; I < n1; I += 32) {
      float acc = 0.f;
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy) {
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
          const int row = 2 * J + 1 + dy, col = 2 * I + 1 + dx;
          const float res = v.R[bidx(b, b.r0, row, col)] - band_op(b, E, row, col, ch2, d);
          acc += (dx == 0 ? 0.5f : 0.25f) * (dy == 0 ? 0.5f : 0.25f) * res;
        }
      }
      const int k = cidx(n1, J, I);
      for (int r = 0; r < b.C; ++r) {
        float* dst = (r == b.rank) ? f1 : cg::this_cluster().map_shared_rank(f1, r);
        dst[k] = acc;
      }
    }
  }
}

// Eo = Ei + P e1 on the band (bilinear interpolation from the padded coarse copy).
__device__ __forceinline__ void fast_prolong(const Band& b, const FastVec& v, int cur, const float* e1,
                                             int n1) {
  const float* Ei = v.E[cur];
  const BArr Eo = barr(b, v.E[cur ^ 1]);
  for_own(b, [&](int row, int col) {
    bstore(b, Eo, row, col, Ei[bidx(b, b.r0, row, col)] + cinterp(e1, n1, row, col));
  });
}

// Multigrid V-cycle z = M R on the band. Entry: R and E[0] (first smoother
// sweep, pointwise) complete with halos. Exit: z in E[returned], r.z total in
// slot SL_RZ.
__device__ int fast_vcycle(const Team& t, const Band& b, const FastVec& v, const Op& op,
                           const SmemLv<float>& sm, float omega, int nu, int nuc) {
  const int L = op.L;
  if (L == 1) return 0;
  const OpLevel& l0 = op.lv[0];
  const float ch2 = (float)l0.ch2, d = 1.f + 4.f * ch2, dinv = (float)l0.dinv;
  double rz = 0.0;
  int cur = 0;
  SEC_T0();
  for (int s = 1; s < nu; ++s) {
    fast_sweep(b, v, cur, ch2, d, dinv, omega, false, rz);
    cur ^= 1;
    SEC_ADD(SEC_BAND);
    team_sync(t);
    SEC_ADD(SEC_SYNC);
  }
  const int n1 = op.lv[1].n;
  fast_restrict(b, v, cur, ch2, d, sm.f[1], n1);
  SEC_ADD(SEC_BAND);
  team_sync(t);
  SEC_ADD(SEC_SYNC);
  // every CTA: the coarse levels in its own shared memory
  {
    const OpLevel& l1 = op.lv[1];
    const float sc = (L == 2) ? 1.f : omega;
    const float d1inv = (float)l1.dinv;
    for_all(n1, b.warp, b.lane, b.nwarp, [&](int row, int col) {
      const int i = cidx(n1, row, col);
      sm.e[1][0][i] = sc * sm.f[1][i] * d1inv;
    });
    __syncthreads();
    unsigned ecur = 0;  // bit l: current smoother buffer of level l
    auto E = [&](int l) { return sm.e[l][(ecur >> l) & 1]; };
    auto Eo = [&](int l) { return sm.e[l][((ecur >> l) & 1) ^ 1]; };
    for (int c = 1; c < L - 1; ++c) {
      for (int s = 1; s < nuc; ++s) {
        csweep(b, op.lv[c], Eo(c), E(c), sm.f[c], omega);
        ecur ^= 1u << c;
        __syncthreads();
      }
      crestrict(b, op.lv[c], op.lv[c + 1], E(c), sm.f[c], sm.f[c + 1], sm.e[c + 1][0],
                (c + 1 == L - 1) ? 1.f : omega);
      ecur &= ~(1u << (c + 1));
      __syncthreads();
    }
    for (int c = L - 2; c >= 1; --c) {
      cprolong(b, op.lv[c], op.lv[c + 1], E(c), E(c + 1));
      __syncthreads();
      for (int s = 0; s < nuc; ++s) {
        csweep(b, op.lv[c], Eo(c), E(c), sm.f[c], omega);
        ecur ^= 1u << c;
        __syncthreads();
      }
    }
    SEC_ADD(SEC_COARSE);
    fast_prolong(b, v, cur, E(1), n1);
    cur ^= 1;
    SEC_ADD(SEC_BAND);
    team_sync(t);
    SEC_ADD(SEC_SYNC);
  }
  for (int s = 0; s < nu; ++s) {
    const bool last = (s == nu - 1);
    fast_sweep(b, v, cur, ch2, d, dinv, omega, last, rz);
    cur ^= 1;
    SEC_ADD(SEC_BAND);
    if (last) contribute(t, SL_RZ, rz);
    SEC_ADD(SEC_REDUCE);
    team_sync(t);
    SEC_ADD(SEC_SYNC);
  }
  return cur;
}

// FP32 PCG on the band from a prepared state (R, E[0] set), updating X.
__device__ void fast_pcg(const Team& t, const Band& b, const FastVec& v, const Op& op, const SmemLv<float>& sm,
                         double tol2, bool& done, const SolveCfg& cfg, Ctr& ctr) {
  const OpLevel& l0 = op.lv[0];
  const float ch2 = (float)l0.ch2, d = 1.f + 4.f * ch2, dinv = (float)l0.dinv;
  const float omega = (float)cfg.omega;
  const float scale0 = (op.L == 1) ? 1.f : omega;
  int it_count = 0;
  double rz_old = 0.0;
  bool all = __syncthreads_and(done);
  while (!all) {
    const int zc = fast_vcycle(t, b, v, op, sm, omega, cfg.nu, cfg.nu_coarse);
    SEC_T0();
    const float* z = v.E[zc];
    const double rz = total(t, SL_RZ);
    SEC_ADD(SEC_REDUCE);
    const float beta = (float)((it_count == 0 || done || !(rz_old > 0.0)) ? 0.0 : rz / rz_old);
    float pqf = 0.f;
    const bool first = (it_count == 0);
    for_own(b, [&](int row, int col) {
      const int i = bidx(b, b.r0, row, col);
      const float az = band_op(b, z, row, col, ch2, d);
      const float pv = first ? z[i] : z[i] + beta * v.P[i];
      const float qv = first ? az : az + beta * v.Q[i];
      v.P[i] = pv;
      v.Q[i] = qv;
      pqf += pv * qv;
    });
    const double pq = (double)pqf;
    SEC_ADD(SEC_BAND);
    contribute(t, SL_PQ, pq);
    SEC_ADD(SEC_REDUCE);
    team_sync(t);
    SEC_ADD(SEC_SYNC);
    const double pqt = total(t, SL_PQ);
    SEC_ADD(SEC_REDUCE);
    const float alpha = (float)((done || !(pqt > 0.0)) ? 0.0 : rz / pqt);
    float rrf = 0.f, rz1f = 0.f;
    // E[0] is written below; z may be E[0] but phase A has consumed it
    {
      const BArr Xa = barr(b, v.X), Ra = barr(b, v.R), Ea = barr(b, v.E[0]);
      for_own(b, [&](int row, int col) {
        const int i = bidx(b, b.r0, row, col);
        const float xv = first ? alpha * v.P[i] : v.X[i] + alpha * v.P[i];
        const float rv = v.R[i] - alpha * v.Q[i];
        bstore(b, Xa, row, col, xv);
        bstore(b, Ra, row, col, rv);
        rrf += rv * rv;
        const float e = scale0 * rv * dinv;
        bstore(b, Ea, row, col, e);
        if (op.L == 1) rz1f += rv * e;
      });
    }
    const double rr = (double)rrf, rz1 = (double)rz1f;
    SEC_ADD(SEC_BAND);
    contribute(t, SL_RR, rr);
    if (op.L == 1) contribute(t, SL_RZ, rz1);
    SEC_ADD(SEC_REDUCE);
    team_sync(t);
    SEC_ADD(SEC_SYNC);
    const double rrt = total(t, SL_RR);
    SEC_ADD(SEC_REDUCE);
    if (!isfinite(rrt)) {
      ctr.status |= STAT_NONFINITE;
      done = true;
    }
    done = done || (rrt <= tol2);
    ++it_count;
    rz_old = rz;
    const bool capped = it_count >= cfg.maxit;
    all = __syncthreads_and(done) || capped;
    if (capped && !__syncthreads_and(done)) ctr.status |= STAT_NOCONV;
  }
  ctr.iters += it_count;
  ctr.iters_max = max(ctr.iters_max, it_count);
}

// Solve (I + c L) x = b (FP64 state in global memory) by FP64 iterative
// refinement around the band FP32 MG-PCG; inner problems scaled by powers of
// two as in the generic kernel.
__device__ double* fast_solve(const Team& t, const Band& b, const SweepParams& P, const Op& op,
                              const WSV<float>& w, const FastVec& v, const SmemLv<float>& sm, const double* bsrc,
                              const double* dsrc, const double* x0, double* X1, double* X2, Ctr& ctr) {
  const OpLevel& l0 = op.lv[0];
  const int n = b.n;
  const double ch2d = l0.ch2, dd = 1.0 + 4.0 * ch2d;
  const float dinvf = (float)l0.dinv;
  const float omega = (float)P.cfg.omega;
  const float scale0 = (op.L == 1) ? 1.f : omega;
  const double* xa = x0;
  double* tgt = X1;
  double* oth = X2;
  bool done = false;
  double bbt = 0.0;
  int ref = 0;
  const double inv_n = 1.0 / (double)l0.N;
  double sc = ctr.mix_scale;
  double inv_sc_c = 1.0;
  for (;; ++ref) {
    const bool first = (ref == 0);
    double rr = 0.0, bb = 0.0, rz1 = 0.0;
    SEC_T0();
    const BArr Ra = barr(b, v.R), Ea = barr(b, v.E[0]);
    for_own(b, [&](int row, int col) {
      const int p = row * n + col;
      double bp;
      if (first) {
        bp = rhs_at(P, t, bsrc, dsrc, p, p);
        if (dsrc) w.bd[p] = bp;
        bb += bp * bp;
      } else {
        bp = dsrc ? w.bd[p] : (bsrc ? bsrc[p] : 0.0);
      }
      // x + c at the node and its four neighbours (c from the band, halos included)
      auto xc = [&](int rr_, int cc_) -> double {
        if (rr_ < 0 || rr_ >= n || cc_ < 0 || cc_ >= n) return 0.0;
        double s = xa ? xa[rr_ * n + cc_] : 0.0;
        if (!first) s += (double)v.X[bidx(b, b.r0, rr_, cc_)] * inv_sc_c;
        return s;
      };
      double ax = 0.0, xcen = 0.0;
      if (xa || !first) {
        xcen = xc(row, col);
        ax = dd * xcen - ch2d * (xc(row, col - 1) + xc(row, col + 1) + xc(row - 1, col) + xc(row + 1, col));
      }
      const double rd = bp - ax;
      tgt[p] = xcen;
      const float rf = (float)(rd * sc);
      bstore(b, Ra, row, col, rf);
      const float e = scale0 * rf * dinvf;
      bstore(b, Ea, row, col, e);
      rr += rd * rd;
      if (op.L == 1) rz1 += (double)(rf * e);
    });
    SEC_ADD(SEC_REFINE);
    contribute(t, SL_RRD, rr);
    if (first) contribute(t, SL_BBD, bb);
    if (op.L == 1) contribute(t, SL_RZ, rz1);
    SEC_ADD(SEC_REDUCE);
    team_sync(t);
    SEC_ADD(SEC_SYNC);
    const double rrt = total(t, SL_RRD);
    if (first) {
      bbt = total(t, SL_BBD);
      if (!(bbt > 0.0)) {
        for_own(b, [&](int row, int col) { tgt[row * n + col] = 0.0; });
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
    if (__syncthreads_and(done)) break;
    if (ref >= P.cfg.maxref) {
      ctr.status |= STAT_NOCONV;
      break;
    }
    bool idone = done;
    fast_pcg(t, b, v, op, sm, P.cfg.inner_rtol * P.cfg.inner_rtol * rrt * sc * sc, idone, P.cfg, ctr);
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

__global__ void __launch_bounds__(512, 1) fast2d_kernel(const SweepParams P) {
  __shared__ double s_red[2 * NSLOT * LRP_MAXBV];
  __shared__ double s_redw[32 * LRP_MAXBV];
  extern __shared__ __align__(16) unsigned char s_dyn[];
  Team t;
  t.C = P.C;
  t.rank = (P.C > 1) ? (int)cg::this_cluster().block_rank() : 0;
  t.NT = blockDim.x;
  t.tid = threadIdx.x;
  t.g = t.rank * t.NT + t.tid;
  t.S = t.C * t.NT;
  t.BV = 1;
  t.bvs = 0;
  t.col = 0;
  t.red = s_red;
  t.redw = s_redw;
  t.phase = 0;
  const int team = blockIdx.x / P.C;
  const int n = P.step.lv[0].n;
#ifdef LRP_SECTION_TIMERS
  if (threadIdx.x < 8) s_sec[threadIdx.x] = 0;
  const long long k_t0 = clock64();
#endif
  Band b;
  b.n = n;
  b.pitch = n + 1;
  b.rank = t.rank;
  b.C = t.C;
  b.r0 = (t.rank * n) / t.C;
  b.r1 = ((t.rank + 1) * n) / t.C;
  b.r0p = ((t.rank - 1) * n) / t.C;
  b.r0n = b.r1;
  b.warp = t.tid >> 5;
  b.lane = t.tid & 31;
  b.nwarp = t.NT >> 5;
  // band arrays (each with one leading zero pad element) and coarse levels
  FastVec v;
  float* fb = (float*)s_dyn;
  const int band_len = P.fast_band_len;
  v.E[0] = fb + 0 * band_len + 1;
  v.E[1] = fb + 1 * band_len + 1;
  v.R = fb + 2 * band_len + 1;
  v.P = fb + 3 * band_len + 1;
  v.Q = fb + 4 * band_len + 1;
  v.X = fb + 5 * band_len + 1;
  for (size_t i = t.tid; i < P.smem_bytes / sizeof(float); i += t.NT) fb[i] = 0.f;
  SmemLv<float> sm;
  for (int l = 0; l < LRP_MAXLEV; ++l) {
    sm.e[l][0] = (float*)(s_dyn + P.smem_off[l][0]);
    sm.e[l][1] = (float*)(s_dyn + P.smem_off[l][1]);
    sm.f[l] = (float*)(s_dyn + P.smem_off[l][2]);
  }
  // no neighbour may write into this CTA's halos before they are zeroed
  team_sync(t);
  char* base = P.ws + (size_t)team * P.team_bytes;
  WSV<float> w;
  for (int k = 0; k < 3; ++k) w.dbuf[k] = (double*)(base + P.off_dbuf[k]);
  w.bd = (double*)(base + P.off_bd);
  w.obs = (double*)(base + P.off_obs);
  const int gcol = team;
  const bool valid = gcol < P.nvec;
  const int N0 = n * n;
  Ctr ctr;
  int cur = (P.stages & ST_LOAD_X) ? 0 : min(max(P.end_buf[team], 0), 2);
  if (P.stages & ST_LOAD_X) {
    for_own(b, [&](int row, int col) {
      const int p = row * n + col;
      w.dbuf[0][p] = valid ? P.X[(size_t)gcol * P.ldx + p] : 0.0;
    });
    team_sync(t);
  }
  if (P.stages & ST_LOAD_D) {
    const int nd = P.n_obs * P.n_steps;
    for (int it = t.g; it < nd; it += t.S) w.obs[it] = valid ? P.Din[(size_t)gcol * P.lddin + it] : 0.0;
    team_sync(t);
  }
  if (P.stages & ST_PRIOR_IN) {
    double* res = fast_solve(t, b, P, P.prior, w, v, sm, w.dbuf[cur], nullptr, nullptr, w.dbuf[(cur + 1) % 3],
                             w.dbuf[(cur + 2) % 3], ctr);
    cur = buf_index(w.dbuf, res);
  }
  if (P.stages & ST_FORWARD) {
    for (int step = P.t_begin + 1; step <= P.t_end; ++step) {
      double* res = fast_solve(t, b, P, P.step, w, v, sm, w.dbuf[cur], nullptr, w.dbuf[cur],
                               w.dbuf[(cur + 1) % 3], w.dbuf[(cur + 2) % 3], ctr);
      cur = buf_index(w.dbuf, res);
      if (P.n_steps > 0 && (step % P.obs_every) == 0 && step / P.obs_every <= P.n_steps) {
        const int k = step / P.obs_every - 1;
        for (int s = t.g; s < P.n_obs; s += t.S) {
          double y = 0.0;
          for (int c = 0; c < 8; ++c) {
            const int node = P.obs_node[s * 8 + c];
            if (node >= 0) y += P.obs_w[s * 8 + c] * res[node];
          }
          w.obs[(size_t)k * P.n_obs + s] = y * P.inv_sigma2;
          if ((P.stages & ST_STORE_D) && valid) P.Dout[(size_t)gcol * P.lddout + k * P.n_obs + s] = y;
        }
      }
      if ((P.stages & ST_TRAJ) && valid) {
        double* dst = P.traj + ((size_t)gcol * P.traj_cols + (step - P.t_begin - 1)) * P.traj_ld;
        for_own(b, [&](int row, int col) { dst[row * n + col] = res[row * n + col]; });
      }
    }
    team_sync(t);
  }
  if (P.stages & ST_ADJOINT) {
    const double* q = nullptr;
    for (int step = P.adj_begin; step >= 1; --step) {
      const bool obs = (step % P.obs_every) == 0 && step / P.obs_every <= P.n_steps;
      if (!q && !obs) continue;
      const double* dsrc = obs ? w.obs + (size_t)(step / P.obs_every - 1) * P.n_obs : nullptr;
      const int qi = q ? buf_index(w.dbuf, q) : cur;
      q = fast_solve(t, b, P, P.step, w, v, sm, q, dsrc, q, w.dbuf[(qi + 1) % 3], w.dbuf[(qi + 2) % 3], ctr);
    }
    if (q) {
      cur = buf_index(w.dbuf, q);
    } else {
      for_own(b, [&](int row, int col) { w.dbuf[cur][row * n + col] = 0.0; });
      team_sync(t);
    }
  }
  if (P.stages & ST_PRIOR_OUT) {
    double* res = fast_solve(t, b, P, P.prior, w, v, sm, w.dbuf[cur], nullptr, nullptr, w.dbuf[(cur + 1) % 3],
                             w.dbuf[(cur + 2) % 3], ctr);
    cur = buf_index(w.dbuf, res);
  }
  if ((P.stages & ST_STORE_Y) && valid) {
    for_own(b, [&](int row, int col) {
      const int p = row * n + col;
      P.Y[(size_t)gcol * P.ldy + p] = w.dbuf[cur][p];
    });
  }
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
  if (t.rank == 0 && t.tid == 0 && valid)
    atomicMax(&P.stats->max_rel_res_bits, (unsigned long long)__double_as_longlong(ctr.max_res));
#ifdef LRP_SECTION_TIMERS
  if (team == 0 && t.rank == 0 && t.tid == 0 && P.section_cycles) {
    for (int k = 0; k < 6; ++k) P.section_cycles[k] = s_sec[k];
    P.section_cycles[7] = (unsigned long long)(clock64() - k_t0);
  }
#endif
}

}  // namespace lrp
