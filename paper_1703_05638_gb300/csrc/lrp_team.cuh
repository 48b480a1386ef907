// Device building blocks of the persistent sweep kernel: the team (a
// thread-block cluster of C CTAs owning BV interleaved columns), its barrier
// and deterministic reductions, the finite-difference operator I + c L_l, and
// the multigrid transfer operators.
//
// Operator (Sec. 6 Eq. (pde), implicit Euler block row of Eq. (st_pde), M = I):
//   ((I + c L) v)_p = d_p v_p - (c/h^2) sum_faces kappa_f v_nbr(f),
//   d_p = 1 + (c/h^2) sum_faces kappa_f,  v = 0 outside the grid.
// Multigrid (preconditioner of PCG on I + c L): damped Jacobi smoothing,
// full-weighting restriction (1D stencil [1/4 1/2 1/4]), bi/trilinear
// prolongation (= 2^dim x restriction^T), rediscretised coarse operators,
// exact solve on the single-node coarsest level. With equal pre and post
// sweep counts the V-cycle is a fixed symmetric positive definite operator.
#pragma once

#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include "lrp_internal.h"

namespace cg = cooperative_groups;

namespace lrp {

// Optional section timers (build with -DLRP_SECTION_TIMERS): thread 0 of each
// CTA accumulates clock64() cycles per section into shared memory; CTA 0 of
// team 0 writes them to SweepParams::section_cycles at exit (slot 11: the
// whole kernel). Sections: 0 finest-level phases (band kernel: the band;
// generic kernel: level-0 smoothing and prolongation), 1 team barriers,
// 2 coarse level 1 (band) / global coarse levels (generic), 3 refinement,
// 4 reductions, 5 PCG vector phases (generic), 6 coarse levels >= 2 (band) /
// shared-memory levels (generic), 7 level-0 restriction (generic).
#ifdef LRP_SECTION_TIMERS
__shared__ unsigned long long s_sec[12];
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
enum {
  SEC_BAND = 0, SEC_SYNC = 1, SEC_COARSE = 2, SEC_REFINE = 3, SEC_REDUCE = 4, SEC_OTHER = 5, SEC_COARSE2 = 6,
  SEC_RESTRICT = 7
};

enum { SL_RR = 0, SL_BB = 1, SL_RZ = 2, SL_PQ = 3, SL_RRD = 4, SL_BBD = 5, NSLOT = 8 };

struct Team {
  int C, rank, NT, tid, g, S, BV, bvs, col;
  double* red;   // [2][NSLOT][LRP_MAXBV] CTA totals, two banks (shared memory)
  double* redw;  // [32][LRP_MAXBV] warp partials (shared memory)
  float* redf;   // the same for the FP32 reductions of the inner PCG (separate
  float* redwf;  //   arrays: no aliasing with FP64 totals other CTAs still read)
  // Team barriers passed so far (identical in every thread of the team).
  // A total is contributed before barrier k into bank k&1 and read after it;
  // its bank is next written before barrier k+2, which no CTA reaches before
  // every CTA has finished reading it (the reads precede barrier k+1).
  mutable unsigned phase;
};

__device__ __forceinline__ void team_sync(const Team& t) {
  if (t.C > 1) {
    cg::this_cluster().sync();  // barrier.cluster arrive(release) + wait(acquire)
  } else {
    __syncthreads();
  }
  ++t.phase;
}

// Sum v over the CTA per column (lanes with equal col), store the CTA total
// in slot. Deterministic order. Must be called by every thread of the CTA.
__device__ __forceinline__ void contribute(const Team& t, int slot, double v) {
  for (int off = 16; off >= t.BV; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int lane = t.tid & 31, w = t.tid >> 5;
  if (lane < t.BV) t.redw[w * LRP_MAXBV + lane] = v;
  __syncthreads();
  const int nw = t.NT >> 5;
  if (t.BV == 1) {
    // one column: warp 0 combines the warp partials with a shuffle tree
    if (w == 0) {
      double s = lane < nw ? t.redw[lane * LRP_MAXBV] : 0.0;
      for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
      if (lane == 0) t.red[((t.phase & 1) * NSLOT + slot) * LRP_MAXBV] = s;
    }
  } else if (t.tid < t.BV) {
    double s = 0.0;
    for (int i = 0; i < nw; ++i) s += t.redw[i * LRP_MAXBV + t.tid];
    t.red[((t.phase & 1) * NSLOT + slot) * LRP_MAXBV + t.tid] = s;
  }
  __syncthreads();
}

// FP32 version for the inner PCG's dot products (the FP64 pipe's ~64-cycle
// dependent adds made the FP64 trees a large part of a PCG iteration; the
// inner solve needs its dot products to FP32 accuracy only). Same
// deterministic order and bank protocol as the FP64 version.
__device__ __forceinline__ void contribute(const Team& t, int slot, float v) {
  for (int off = 16; off >= t.BV; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int lane = t.tid & 31, w = t.tid >> 5;
  if (lane < t.BV) t.redwf[w * LRP_MAXBV + lane] = v;
  __syncthreads();
  const int nw = t.NT >> 5;
  if (t.BV == 1) {
    if (w == 0) {
      float s = lane < nw ? t.redwf[lane * LRP_MAXBV] : 0.f;
      for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
      if (lane == 0) t.redf[((t.phase & 1) * NSLOT + slot) * LRP_MAXBV] = s;
    }
  } else if (t.tid < t.BV) {
    float s = 0.f;
    for (int i = 0; i < nw; ++i) s += t.redwf[i * LRP_MAXBV + t.tid];
    t.redf[((t.phase & 1) * NSLOT + slot) * LRP_MAXBV + t.tid] = s;
  }
  __syncthreads();
}

__device__ __forceinline__ double total_f(const Team& t, int slot) {
  const int idx = (((t.phase - 1) & 1) * NSLOT + slot) * LRP_MAXBV + t.col;
  if (t.C == 1) return (double)t.redf[idx];
  cg::cluster_group cl = cg::this_cluster();
  if (t.BV == 1) {
    const int lane = t.tid & 31;
    float s = lane < t.C ? *cl.map_shared_rank(t.redf + idx, lane) : 0.f;
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    return (double)s;
  }
  float s = 0.f;
  for (int r = 0; r < t.C; ++r) s += *cl.map_shared_rank(t.redf + idx, r);
  return (double)s;
}

// total of a slot contributed in the inner type T (float: total_f)
template <typename T>
__device__ __forceinline__ double total_t(const Team& t, int slot);

// Team-wide total of slot for this thread's column; valid after a team_sync
// that followed the contribute. Every CTA sums the ranks in the same order,
// so all CTAs obtain bit-identical totals (and take identical branches).
__device__ __forceinline__ double total(const Team& t, int slot) {
  const int idx = (((t.phase - 1) & 1) * NSLOT + slot) * LRP_MAXBV + t.col;
  if (t.C == 1) return t.red[idx];
  cg::cluster_group cl = cg::this_cluster();
  if (t.BV == 1) {
    // one column: lane r loads rank r's partial, a fixed shuffle tree sums
    // them (the same tree in every warp of every CTA: identical results)
    const int lane = t.tid & 31;
    double s = lane < t.C ? *cl.map_shared_rank(t.red + idx, lane) : 0.0;
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    return s;
  }
  double s = 0.0;
  for (int r = 0; r < t.C; ++r) s += *cl.map_shared_rank(t.red + idx, r);
  return s;
}

template <>
__device__ __forceinline__ double total_t<double>(const Team& t, int slot) {
  return total(t, slot);
}
template <>
__device__ __forceinline__ double total_t<float>(const Team& t, int slot) {
  return total_f(t, slot);
}

__device__ __forceinline__ uint32_t fdiv(uint32_t x, const FastDiv& f) {
  return (__umulhi(x, f.m) + x) >> f.s;
}

template <int DIM>
__device__ __forceinline__ void decomp(const OpLevel& lv, int p, int& i0, int& i1, int& i2) {
  const uint32_t q = fdiv((uint32_t)p, lv.dn);
  i0 = p - (int)q * lv.n;
  if (DIM == 3) {
    const uint32_t q2 = fdiv(q, lv.dn);
    i1 = (int)q - (int)q2 * lv.n;
    i2 = (int)q2;
  } else {
    i1 = (int)q;
    i2 = 0;
  }
}

template <typename T>
__device__ __forceinline__ const T* kap(const OpLevel& lv, int a);
template <>
__device__ __forceinline__ const double* kap<double>(const OpLevel& lv, int a) { return lv.kd[a]; }
template <>
__device__ __forceinline__ const float* kap<float>(const OpLevel& lv, int a) { return lv.kf[a]; }

// Conversions between the arithmetic type and a storage type (BF16
// storage of the multigrid vectors: round to nearest even on store).
template <typename T, typename S>
__device__ __forceinline__ T cvt(S x) {
  return (T)x;
}
template <>
__device__ __forceinline__ float cvt<float, __nv_bfloat16>(__nv_bfloat16 x) {
  return __bfloat162float(x);
}
template <typename S, typename T>
__device__ __forceinline__ S cst(T x) {
  return (S)x;
}
template <>
__device__ __forceinline__ __nv_bfloat16 cst<__nv_bfloat16, float>(float x) {
  return __float2bfloat16_rn(x);
}

// Loader of one interleaved column of a team vector stored as S, read as T.
template <typename S, typename T>
struct LdT {
  const S* v;
  int bvs, col;
  __device__ __forceinline__ T operator()(int q) const { return cvt<T>(v[(q << bvs) + col]); }
};

// Loader of one interleaved column of a team vector.
template <typename T>
struct Ld {
  const T* v;
  int bvs, col;
  __device__ __forceinline__ T operator()(int q) const { return v[(q << bvs) + col]; }
};

// Loader of (x + c * c_scale) for the refinement residual (x double, c the
// inner correction in the inner type, c_scale undoing its power-of-two scale).
template <typename TI>
struct LdSum {
  const double* x;  // may be NULL (zero)
  const TI* c;      // may be NULL (zero)
  int bvs, col;
  double c_scale;
  __device__ __forceinline__ double operator()(int q) const {
    const int i = (q << bvs) + col;
    double s = x ? x[i] : 0.0;
    if (c) s += (double)c[i] * c_scale;
    return s;
  }
};

// ((I + c L) v)_p and the diagonal d_p at node p = (i0,i1,i2).
template <typename T, int DIM, bool KAPPA, class LD>
__device__ __forceinline__ T op_at(const OpLevel& lv, const LD& ld, int p, int i0, int i1, int i2,
                                   T& diag) {
  const int n = lv.n;
  T s, kd;
  if (KAPPA) {
    const T* kx = kap<T>(lv, 0);
    const T* ky = kap<T>(lv, 1);
    const int fx = p + (DIM == 3 ? (i2 * n + i1) : i1);
    const T kw = kx[fx], ke = kx[fx + 1];
    const int fy = p + (DIM == 3 ? i2 * n : 0);
    const T ks = ky[fy], kn = ky[fy + n];
    kd = kw + ke + ks + kn;
    s = (i0 > 0 ? kw * ld(p - 1) : T(0)) + (i0 < n - 1 ? ke * ld(p + 1) : T(0)) +
        (i1 > 0 ? ks * ld(p - n) : T(0)) + (i1 < n - 1 ? kn * ld(p + n) : T(0));
    if (DIM == 3) {
      const T* kz = kap<T>(lv, 2);
      const int nn = n * n;
      const T kdn = kz[p], kup = kz[p + nn];
      kd += kdn + kup;
      s += (i2 > 0 ? kdn * ld(p - nn) : T(0)) + (i2 < n - 1 ? kup * ld(p + nn) : T(0));
    }
  } else {
    s = (i0 > 0 ? ld(p - 1) : T(0)) + (i0 < n - 1 ? ld(p + 1) : T(0)) +
        (i1 > 0 ? ld(p - n) : T(0)) + (i1 < n - 1 ? ld(p + n) : T(0));
    if (DIM == 3) {
      const int nn = n * n;
      s += (i2 > 0 ? ld(p - nn) : T(0)) + (i2 < n - 1 ? ld(p + nn) : T(0));
    }
    kd = T(2 * DIM);
  }
  const T ch2 = (T)lv.ch2;
  diag = T(1) + ch2 * kd;
  return diag * ld(p) - ch2 * s;
}

// 1 / diagonal of (I + c L) at node p (precomputed; no division in the kernel)
template <typename T, bool KAPPA>
__device__ __forceinline__ T dinv_at(const OpLevel& lv, int p);
template <>
__device__ __forceinline__ double dinv_at<double, true>(const OpLevel& lv, int p) { return lv.dinvd[p]; }
template <>
__device__ __forceinline__ float dinv_at<float, true>(const OpLevel& lv, int p) { return lv.dinvf[p]; }
template <>
__device__ __forceinline__ double dinv_at<double, false>(const OpLevel& lv, int) { return lv.dinv; }
template <>
__device__ __forceinline__ float dinv_at<float, false>(const OpLevel& lv, int) { return (float)lv.dinv; }

template <typename T, int DIM, bool KAPPA>
__device__ __forceinline__ T diag_at(const OpLevel& lv, int p, int i0, int i1, int i2) {
  const int n = lv.n;
  T kd;
  if (KAPPA) {
    const T* kx = kap<T>(lv, 0);
    const T* ky = kap<T>(lv, 1);
    const int fx = p + (DIM == 3 ? (i2 * n + i1) : i1);
    const int fy = p + (DIM == 3 ? i2 * n : 0);
    kd = kx[fx] + kx[fx + 1] + ky[fy] + ky[fy + n];
    if (DIM == 3) {
      const T* kz = kap<T>(lv, 2);
      kd += kz[p] + kz[p + n * n];
    }
  } else {
    kd = T(2 * DIM);
  }
  return T(1) + (T)lv.ch2 * kd;
}

// Grid-stride loop over items [start, items) that handles LRP_UNROLL items
// per group: compute(it) performs every load and the arithmetic of item it
// and returns its values, commit(it, v) performs the stores (and any
// accumulation, in item order). With more than one item per group, all loads
// of a group are issued before its first store (a store could alias later
// loads, so the compiler would not overlap them itself).
// Measured on GB300 (127^2 and 63^3 sweeps, 16 columns): 2 or 4 items per
// group spill registers and run 5-20% slower than 1, so 1 is the default.
#ifndef LRP_UNROLL
#define LRP_UNROLL 1
#endif
// The solver levels (V-cycle, PCG, refinement) are inlined into the one
// persistent kernel unless LRP_NOINLINE_SOLVER is defined (separate register
// allocations; slower when measured, kept for experiments with wider rounds).
#ifdef LRP_NOINLINE_SOLVER
#define LRP_SOLVER_FN __noinline__
#else
#define LRP_SOLVER_FN
#endif
template <class V, class Compute, class Commit>
__device__ __forceinline__ void batched_loop(int start, int items, int stride, Compute compute, Commit commit) {
  for (int it0 = start; it0 < items; it0 += LRP_UNROLL * stride) {
    V v[LRP_UNROLL];
#pragma unroll
    for (int u = 0; u < LRP_UNROLL; ++u) {
      const int it = it0 + u * stride;
      if (it < items) v[u] = compute(it);
    }
#pragma unroll
    for (int u = 0; u < LRP_UNROLL; ++u) {
      const int it = it0 + u * stride;
      if (it < items) commit(it, v[u]);
    }
  }
}

template <typename T>
struct V2 {
  T a, b;
};
template <typename T>
struct V3 {
  T a, b, c;
};

// ---------------------------------------------------------------------------
// Multigrid phases. Each works over items [start, N*BV) with the given
// stride; the caller ends the phase with a team barrier (global levels) or
// __syncthreads (shared-memory levels). The vectors are written by other
// phases of the same launch, so their pointers must not be declared
// __restrict__ read-only: that would allow the non-coherent read-only load
// path, which can return stale lines.

// One damped Jacobi sweep e_out = e_in + omega (f - A e_in) / d. If rz_r is
// non-NULL, accumulates rz_r * e_out into rz (used for r.z after the last
// post-smoothing sweep on the finest level).
// The item loop of a Jacobi sweep with the output marked __restrict__ (it
// is a different array from the inputs): the compiler may then issue the
// loads of the next SWEEP_UNROLL items before the stores of the earlier
// ones, which the ordinary loop (a store could alias a later load) forbids.
#ifndef LRP_SWEEP_UNROLL
#define LRP_SWEEP_UNROLL 1
#endif
// (eo, ei: the level's smoother iterates, f: its right-hand side, each in
// its storage type; arithmetic in T)
template <typename T, int DIM, bool KAPPA, typename EO, typename EI, typename FF>
__device__ __forceinline__ T mg_sweep_items(const OpLevel& lv, EO* __restrict__ eo, const EI* ei, const FF* f,
                                            int start, int stride, int bvs, int col, T omega, const T* rz_r) {
  const int items = lv.N << bvs;
  LdT<EI, T> ld{ei, bvs, col};
  T acc = T(0);  // per-thread partial in the inner type
  for (int it0 = start; it0 < items; it0 += LRP_SWEEP_UNROLL * stride) {
#pragma unroll
    for (int u = 0; u < LRP_SWEEP_UNROLL; ++u) {
      const int it = it0 + u * stride;
      if (it < items) {
        const int p = it >> bvs;
        int i0, i1, i2;
        decomp<DIM>(lv, p, i0, i1, i2);
        T d;
        const T ae = op_at<T, DIM, KAPPA>(lv, ld, p, i0, i1, i2, d);
        const T e = cvt<T>(ei[it]) + omega * (cvt<T>(f[it]) - ae) * dinv_at<T, KAPPA>(lv, p);
        eo[it] = cst<EO>(e);
        if (rz_r) acc += rz_r[it] * e;
      }
    }
  }
  return acc;
}

template <typename T, int DIM, bool KAPPA, typename EO, typename EI, typename FF>
__device__ __forceinline__ void mg_sweep(const OpLevel& lv, EO* eo,
                                         const EI* ei, const FF* f,
                                         int start, int stride, int bvs, int col, T omega,
                                         const T* rz_r, double& rz) {
  const T acc = mg_sweep_items<T, DIM, KAPPA>(lv, eo, ei, f, start, stride, bvs, col, omega, rz_r);
  if (rz_r) rz += (double)acc;
}

// Restrict the residual f - A e of level l (fine) to level l+1 (coarse) by
// full weighting, and start the coarse smoother: e_c = scale * f_c / d_c
// (scale = omega, or 1 on the single-node coarsest level: exact solve).
template <typename T, int DIM, bool KAPPA, typename EF, typename FF, typename FC, typename EC>
__device__ __forceinline__ void mg_restrict(const OpLevel& lf, const OpLevel& lc,
                                            const EF* ef, const FF* ff,
                                            FC* fc, EC* ec, int start,
                                            int stride, int bvs, int col, T scale) {
  const int items = lc.N << bvs;
  LdT<EF, T> ld{ef, bvs, col};
  const int nf = lf.n;
  batched_loop<V2<T>>(
      start, items, stride,
      [&](int it) {
        const int P = it >> bvs;
        int c0, c1, c2;
        decomp<DIM>(lc, P, c0, c1, c2);
        T acc = T(0);
        const int z0 = (DIM == 3) ? -1 : 0, z1 = (DIM == 3) ? 1 : 0;
        for (int dz = z0; dz <= z1; ++dz) {
          for (int dy = -1; dy <= 1; ++dy) {
            for (int dx = -1; dx <= 1; ++dx) {
              const int F0 = 2 * c0 + 1 + dx, F1 = 2 * c1 + 1 + dy;
              const int F2 = (DIM == 3) ? 2 * c2 + 1 + dz : 0;
              const int pf = F0 + nf * (F1 + nf * F2);
              T d;
              const T res = cvt<T>(ff[(pf << bvs) + col]) - op_at<T, DIM, KAPPA>(lf, ld, pf, F0, F1, F2, d);
              T w = (dx == 0 ? T(0.5) : T(0.25)) * (dy == 0 ? T(0.5) : T(0.25));
              if (DIM == 3) w *= (dz == 0 ? T(0.5) : T(0.25));
              acc += w * res;
            }
          }
        }
        V2<T> r;
        r.a = acc;
        r.b = scale * acc * dinv_at<T, KAPPA>(lc, P);
        return r;
      },
      [&](int it, const V2<T>& r) {
        fc[it] = cst<FC>(r.a);
        ec[it] = cst<EC>(r.b);
      });
}

// e_out = e_in + P e_c (bi/trilinear interpolation, zero boundary); e_out
// may equal e_in (in place).
template <typename T, int DIM, typename EF, typename EC>
__device__ __forceinline__ void mg_prolong(const OpLevel& lf, const OpLevel& lc, EF* ef,
                                           const EC* ec, int start, int stride, int bvs,
                                           int col, const EF* ein = nullptr) {
  const int items = lf.N << bvs;
  const int nc = lc.n;
  batched_loop<T>(start, items, stride, [&](int it) {
    const int p = it >> bvs;
    int F[3];
    decomp<DIM>(lf, p, F[0], F[1], F[2]);
    int ci[3][2], cnt[3];
    T cw[3][2];
    for (int a = 0; a < DIM; ++a) {
      if (F[a] & 1) {
        ci[a][0] = (F[a] - 1) >> 1;
        cw[a][0] = T(1);
        cnt[a] = 1;
      } else {
        cnt[a] = 0;
        const int lo = (F[a] >> 1) - 1, hi = F[a] >> 1;
        if (lo >= 0) { ci[a][cnt[a]] = lo; cw[a][cnt[a]] = T(0.5); ++cnt[a]; }
        if (hi < nc) { ci[a][cnt[a]] = hi; cw[a][cnt[a]] = T(0.5); ++cnt[a]; }
      }
    }
    T acc = T(0);
    const int n2 = (DIM == 3) ? cnt[2] : 1;
    for (int c = 0; c < n2; ++c) {
      const int z = (DIM == 3) ? ci[2][c] : 0;
      const T wz = (DIM == 3) ? cw[2][c] : T(1);
      for (int b = 0; b < cnt[1]; ++b) {
        for (int a = 0; a < cnt[0]; ++a) {
          const int P = ci[0][a] + nc * (ci[1][b] + nc * z);
          acc += wz * cw[1][b] * cw[0][a] * cvt<T>(ec[(P << bvs) + col]);
        }
      }
    }
    return cvt<T>(ein ? ein[it] : ef[it]) + acc;
  }, [&](int it, T v) { ef[it] = cst<EF>(v); });
}

}  // namespace lrp
