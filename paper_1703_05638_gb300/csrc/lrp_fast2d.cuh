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
//
// Addressing: every shared-memory array is an offset (in floats) into the
// kernel's dynamic shared memory, so local accesses are 32-bit shared-window
// accesses, and the neighbours' copies are 32-bit cluster-window addresses
// (mapa), which keeps address arithmetic in 32-bit registers. The hot loops
// can load the inputs of FAST_G column chunks before their first store.
#pragma once

#include "lrp_df64.cuh"
#include "lrp_sweep_kernel.cuh"

namespace lrp {

constexpr int FAST_HALO = 2;
constexpr int FAST_NJ = 4;  // column chunks per row a lane handles (col = lane + 32 j): n <= 128
// Chunks whose loads are issued together: 2 spills registers and measured
// 60% slower on GB300 than 1 (127^2, 16 columns), so 1 is the default.
#ifndef LRP_FAST_G
#define LRP_FAST_G 1
#endif
constexpr int FAST_G = LRP_FAST_G;
#ifndef LRP_FAST_THREADS
#define LRP_FAST_THREADS 512
#endif
constexpr int FAST_THREADS = LRP_FAST_THREADS;

extern __shared__ __align__(16) float s_fb[];  // the band kernel's dynamic shared memory

__device__ __forceinline__ unsigned smem_addr(int off) {
  return (unsigned)__cvta_generic_to_shared(s_fb + off);
}
// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ unsigned cluster_addr(unsigned local, int rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_cluster(unsigned addr, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}



struct Band {
  int n, r0, r1, pitch;  // grid size, own rows, row pitch (n + 1)
  int rank, C;
  int r0p, r0n;          // first row of the previous / next CTA's band
  int warp, lane, nwarp;
};

// Index of (row, col) in a band array whose band starts at row b0.
__device__ __forceinline__ int bidx(const Band& b, int b0, int row, int col) {
  return (row - b0 + FAST_HALO) * b.pitch + col;
}

// A band array (offset of its element 0) with the cluster addresses of the
// same array in the previous and next CTA of the team, for halo stores.
struct BArr {
  int a;
  unsigned prev, next;
};

__device__ __forceinline__ BArr barr(const Band& b, int A) {
  BArr r;
  r.a = A;
  const unsigned loc = smem_addr(A);
  r.prev = b.rank > 0 ? cluster_addr(loc, b.rank - 1) : 0u;
  r.next = b.rank < b.C - 1 ? cluster_addr(loc, b.rank + 1) : 0u;
  return r;
}

// Store v at (row, col) locally and, for boundary rows, into the halo of the
// neighbour that needs it.
__device__ __forceinline__ void bstore(const Band& b, const BArr& A, int row, int col, float v) {
  s_fb[A.a + bidx(b, b.r0, row, col)] = v;
  if (b.rank > 0 && row < b.r0 + FAST_HALO) st_cluster(A.prev + 4u * (unsigned)bidx(b, b.r0p, row, col), v);
  if (b.rank < b.C - 1 && row >= b.r1 - FAST_HALO)
    st_cluster(A.next + 4u * (unsigned)bidx(b, b.r0n, row, col), v);
}

// Sum of the four neighbours of index i of a band array.
__device__ __forceinline__ float bnb(const Band& b, int A, int i) {
  return s_fb[A + i - 1] + s_fb[A + i + 1] + s_fb[A + i - b.pitch] + s_fb[A + i + b.pitch];
}

struct FastVec {
  int E[2];
  int R, P, Q, X;
};

// Coarse levels: offsets of the two smoother buffers and the right-hand side.
struct CLv {
  int e[LRP_MAXLEV][2];
  int f[LRP_MAXLEV];
};

// One damped Jacobi sweep on the band: Eo = Ei + omega (R - A Ei) / d.
__device__ __forceinline__ void fast_sweep(const Band& b, const FastVec& v, int cur, float ch2, float d,
                                           float dinv, float omega, bool acc_rz, double& rz) {
  const int Ei = v.E[cur];
  const BArr Eo = barr(b, v.E[cur ^ 1]);
  float acc = 0.f;  // per-thread partial in FP32 (FP64 is a slow pipe here)
  for (int row = b.r0 + b.warp; row < b.r1; row += b.nwarp) {
    const int base = bidx(b, b.r0, row, 0);
#pragma unroll
    for (int j0 = 0; j0 < FAST_NJ; j0 += FAST_G) {
      float ec[FAST_G], nb[FAST_G], rv[FAST_G];
#pragma unroll
      for (int j = j0; j < j0 + FAST_G; ++j) {
        const int i = base + b.lane + 32 * j;
        if (b.lane + 32 * j < b.n) {
          ec[j - j0] = s_fb[Ei + i];
          nb[j - j0] = bnb(b, Ei, i);
          rv[j - j0] = s_fb[v.R + i];
        }
      }
#pragma unroll
      for (int j = j0; j < j0 + FAST_G; ++j) {
        const int col = b.lane + 32 * j;
        if (col < b.n) {
          const float e = ec[j - j0] + omega * (rv[j - j0] - (d * ec[j - j0] - ch2 * nb[j - j0])) * dinv;
          bstore(b, Eo, row, col, e);
          if (acc_rz) acc += rv[j - j0] * e;
        }
      }
    }
  }
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

__device__ __forceinline__ float cnb(int A, int n, int i) {
  return s_fb[A + i - 1] + s_fb[A + i + 1] + s_fb[A + i - (n + 1)] + s_fb[A + i + (n + 1)];
}

// Jacobi sweep on a coarse level: eo = ei + omega (f - A ei) / d
__device__ __forceinline__ void csweep(const Band& b, const OpLevel& lv, int eo, int ei, int f, float omega) {
  const int n = lv.n;
  const float ch2 = (float)lv.ch2, d = 1.f + 4.f * ch2, dinv = (float)lv.dinv;
  for (int row = b.warp; row < n; row += b.nwarp) {
    const int base = cidx(n, row, 0);
#pragma unroll
    for (int j0 = 0; j0 < FAST_NJ; j0 += FAST_G) {
      float ec[FAST_G], nb[FAST_G], fv[FAST_G];
#pragma unroll
      for (int j = j0; j < j0 + FAST_G; ++j) {
        const int i = base + b.lane + 32 * j;
        if (b.lane + 32 * j < n) {
          ec[j - j0] = s_fb[ei + i];
          nb[j - j0] = cnb(ei, n, i);
          fv[j - j0] = s_fb[f + i];
        }
      }
#pragma unroll
      for (int j = j0; j < j0 + FAST_G; ++j)
        if (b.lane + 32 * j < n)
          s_fb[eo + base + b.lane + 32 * j] =
              ec[j - j0] + omega * (fv[j - j0] - (d * ec[j - j0] - ch2 * nb[j - j0])) * dinv;
    }
  }
}

// Full-weighting restriction of f - A e from level lf to lc, and ec = sc fc / d
__device__ __forceinline__ void crestrict(const Band& b, const OpLevel& lf, const OpLevel& lc, int ef, int ff,
                                          int fc, int ec, float sc) {
  const int nf = lf.n, nc = lc.n;
  const float ch2 = (float)lf.ch2, d = 1.f + 4.f * ch2, dinvc = (float)lc.dinv;
  for_all(nc, b.warp, b.lane, b.nwarp, [&](int J, int I) {
    float acc = 0.f;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int i = cidx(nf, 2 * J + 1 + dy, 2 * I + 1 + dx);
        acc += (dx == 0 ? 0.5f : 0.25f) * (dy == 0 ? 0.5f : 0.25f) *
               (s_fb[ff + i] - (d * s_fb[ef + i] - ch2 * cnb(ef, nf, i)));
      }
    const int k = cidx(nc, J, I);
    s_fb[fc + k] = acc;
    s_fb[ec + k] = sc * acc * dinvc;
  });
}

// Bilinear value of the coarse field ec (level with nc nodes, padded) at fine
// node (row, col) of the level below it (pads give the zero boundary).
__device__ __forceinline__ float cinterp(int ec, int nc, int row, int col) {
  const int cy0 = (row - 1) >> 1, cx0 = (col - 1) >> 1;  // floor((row-1)/2): -1 for row 0
  const int base = ec + cidx(nc, cy0, cx0);
  if (row & 1) {
    if (col & 1) return s_fb[base];
    return 0.5f * (s_fb[base] + s_fb[base + 1]);
  }
  if (col & 1) return 0.5f * (s_fb[base] + s_fb[base + nc + 1]);
  return 0.25f * (s_fb[base] + s_fb[base + 1] + s_fb[base + nc + 1] + s_fb[base + nc + 2]);
}

// e += P ec on a coarse level (in place)
__device__ __forceinline__ void cprolong(const Band& b, const OpLevel& lf, const OpLevel& lc, int ef, int ec) {
  const int nf = lf.n, nc = lc.n;
  for (int row = b.warp; row < nf; row += b.nwarp) {
    const int base = cidx(nf, row, 0);
#pragma unroll
    for (int j0 = 0; j0 < FAST_NJ; j0 += FAST_G) {
      float cur[FAST_G], add[FAST_G];
#pragma unroll
      for (int j = j0; j < j0 + FAST_G; ++j)
        if (b.lane + 32 * j < nf) {
          cur[j - j0] = s_fb[ef + base + b.lane + 32 * j];
          add[j - j0] = cinterp(ec, nc, row, b.lane + 32 * j);
        }
#pragma unroll
      for (int j = j0; j < j0 + FAST_G; ++j)
        if (b.lane + 32 * j < nf) s_fb[ef + base + b.lane + 32 * j] = cur[j - j0] + add[j - j0];
    }
  }
}

// Coarse rows J whose fine centre row 2J+1 lies in this band: full-weighting
// restriction of the residual R - A E into every CTA's copy of f1 (padded
// coarse layout).
__device__ __forceinline__ void fast_restrict(const Band& b, const FastVec& v, int cur, float ch2, float d,
                                              int f1, int n1) {
  const int E = v.E[cur];
  const unsigned f1loc = smem_addr(f1);
  int J0 = b.r0 / 2;  // smallest J with 2J+1 >= r0
  if (2 * J0 + 1 < b.r0) ++J0;
  for (int J = J0 + b.warp; 2 * J + 1 < b.r1 && J < n1; J += b.nwarp) {
    for (int I = b.lane; I < n1; I += 32) {
      float acc = 0.f;
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy) {
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
          const int i = bidx(b, b.r0, 2 * J + 1 + dy, 2 * I + 1 + dx);
          const float res = s_fb[v.R + i] - (d * s_fb[E + i] - ch2 * bnb(b, E, i));
          acc += (dx == 0 ? 0.5f : 0.25f) * (dy == 0 ? 0.5f : 0.25f) * res;
        }
      }
      const int k = cidx(n1, J, I);
      for (int r = 0; r < b.C; ++r) {
        if (r == b.rank)
          s_fb[f1 + k] = acc;
        else
          st_cluster(cluster_addr(f1loc, r) + 4u * (unsigned)k, acc);
      }
    }
  }
}

// Eo = Ei + P e1 on the band (bilinear interpolation from the padded coarse copy).
__device__ __forceinline__ void fast_prolong(const Band& b, const FastVec& v, int cur, int e1, int n1) {
  const int Ei = v.E[cur];
  const BArr Eo = barr(b, v.E[cur ^ 1]);
  for (int row = b.r0 + b.warp; row < b.r1; row += b.nwarp) {
    const int base = bidx(b, b.r0, row, 0);
#pragma unroll
    for (int j0 = 0; j0 < FAST_NJ; j0 += FAST_G) {
      float cur_[FAST_G], add[FAST_G];
#pragma unroll
      for (int j = j0; j < j0 + FAST_G; ++j)
        if (b.lane + 32 * j < b.n) {
          cur_[j - j0] = s_fb[Ei + base + b.lane + 32 * j];
          add[j - j0] = cinterp(e1, n1, row, b.lane + 32 * j);
        }
#pragma unroll
      for (int j = j0; j < j0 + FAST_G; ++j)
        if (b.lane + 32 * j < b.n) bstore(b, Eo, row, b.lane + 32 * j, cur_[j - j0] + add[j - j0]);
    }
  }
}

// ---- level 1 split across the cluster (SweepParams::fast_split1): CTA k
// owns the level-1 rows J whose fine centre row 2J+1 lies in its band,
// J in [r0/2, r1/2), and keeps the full padded level-1 arrays with two halo
// rows on each side of its own rows, written by its neighbours (the same
// index in every CTA's copy). Every CTA owns at least two rows, so halos come
// from the immediate neighbours only.
struct CArr {
  int a;
  unsigned prev, next;
};

__device__ __forceinline__ CArr carr(const Band& b, int A) {
  CArr r;
  r.a = A;
  const unsigned loc = smem_addr(A);
  r.prev = b.rank > 0 ? cluster_addr(loc, b.rank - 1) : 0u;
  r.next = b.rank < b.C - 1 ? cluster_addr(loc, b.rank + 1) : 0u;
  return r;
}

// Store v at level-1 row J (owned rows [J0, J1)), and into the neighbours'
// halo copies for the first and last two owned rows.
__device__ __forceinline__ void cstore1(const Band& b, const CArr& A, int n1, int J0, int J1, int J, int col,
                                        float v) {
  const int i = cidx(n1, J, col);
  s_fb[A.a + i] = v;
  if (b.rank > 0 && J < J0 + 2) st_cluster(A.prev + 4u * (unsigned)i, v);
  if (b.rank < b.C - 1 && J >= J1 - 2) st_cluster(A.next + 4u * (unsigned)i, v);
}

// Restriction of the band residual into this CTA's level-1 rows of f1, and
// the first coarse smoother iterate e1 = sc f1 / d1, with halo copies.
__device__ __forceinline__ void fast_restrict_split(const Band& b, const FastVec& v, int cur, float ch2, float d,
                                                    int f1, int e1, int n1, float sc, float d1inv) {
  const int E = v.E[cur];
  const int J0 = b.r0 / 2, J1 = b.r1 / 2;
  const CArr F = carr(b, f1), Ec = carr(b, e1);
  for (int J = J0 + b.warp; J < J1; J += b.nwarp) {
    for (int I = b.lane; I < n1; I += 32) {
      float acc = 0.f;
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy) {
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
          const int i = bidx(b, b.r0, 2 * J + 1 + dy, 2 * I + 1 + dx);
          const float res = s_fb[v.R + i] - (d * s_fb[E + i] - ch2 * bnb(b, E, i));
          acc += (dx == 0 ? 0.5f : 0.25f) * (dy == 0 ? 0.5f : 0.25f) * res;
        }
      }
      cstore1(b, F, n1, J0, J1, J, I, acc);
      cstore1(b, Ec, n1, J0, J1, J, I, sc * acc * d1inv);
    }
  }
}

// Jacobi sweep on this CTA's level-1 rows (halo rows of ei read), eo with halo copies.
__device__ __forceinline__ void csweep_split(const Band& b, const OpLevel& lv, int eo, int ei, int f, float omega) {
  const int n = lv.n, J0 = b.r0 / 2, J1 = b.r1 / 2;
  const float ch2 = (float)lv.ch2, d = 1.f + 4.f * ch2, dinv = (float)lv.dinv;
  const CArr Eo = carr(b, eo);
  for (int J = J0 + b.warp; J < J1; J += b.nwarp) {
    const int base = cidx(n, J, 0);
    for (int col = b.lane; col < n; col += 32) {
      const int i = base + col;
      const float e = s_fb[ei + i] + omega * (s_fb[f + i] - (d * s_fb[ei + i] - ch2 * cnb(ei, n, i))) * dinv;
      cstore1(b, Eo, n, J0, J1, J, col, e);
    }
  }
}

// Restriction of level 1 (this CTA's rows, halos read) into the level-2 rows
// whose centre lies in them, all-gathered into every CTA's f2 and e2.
__device__ __forceinline__ void crestrict_split(const Band& b, const OpLevel& lf, const OpLevel& lc, int ef, int ff,
                                                int fc, int ec, float sc) {
  const int nf = lf.n, nc = lc.n;
  const int J0 = b.r0 / 2, J1 = b.r1 / 2;
  const int I0 = J0 / 2, I1 = J1 / 2;
  const float ch2 = (float)lf.ch2, d = 1.f + 4.f * ch2, dinvc = (float)lc.dinv;
  const unsigned fcl = smem_addr(fc), ecl = smem_addr(ec);
  for (int I = I0 + b.warp; I < I1; I += b.nwarp) {
    for (int K = b.lane; K < nc; K += 32) {
      float acc = 0.f;
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
          const int i = cidx(nf, 2 * I + 1 + dy, 2 * K + 1 + dx);
          acc += (dx == 0 ? 0.5f : 0.25f) * (dy == 0 ? 0.5f : 0.25f) *
                 (s_fb[ff + i] - (d * s_fb[ef + i] - ch2 * cnb(ef, nf, i)));
        }
      const int k = cidx(nc, I, K);
      const float ev = sc * acc * dinvc;
      for (int r = 0; r < b.C; ++r) {
        if (r == b.rank) {
          s_fb[fc + k] = acc;
          s_fb[ec + k] = ev;
        } else {
          st_cluster(cluster_addr(fcl, r) + 4u * (unsigned)k, acc);
          st_cluster(cluster_addr(ecl, r) + 4u * (unsigned)k, ev);
        }
      }
    }
  }
}

// e1 += P e2 on this CTA's level-1 rows (in place), with halo copies.
__device__ __forceinline__ void cprolong_split(const Band& b, const OpLevel& lf, const OpLevel& lc, int ef, int ec) {
  const int nf = lf.n, nc = lc.n, J0 = b.r0 / 2, J1 = b.r1 / 2;
  const CArr Ef = carr(b, ef);
  for (int J = J0 + b.warp; J < J1; J += b.nwarp)
    for (int col = b.lane; col < nf; col += 32)
      cstore1(b, Ef, nf, J0, J1, J, col, s_fb[ef + cidx(nf, J, col)] + cinterp(ec, nc, J, col));
}

// Multigrid V-cycle z = M R on the band. Entry: R and E[0] (first smoother
// sweep, pointwise) complete with halos. Exit: z in E[returned], r.z total in
// slot SL_RZ.
__device__ int fast_vcycle(const Team& t, const Band& b, const FastVec& v, const Op& op, const CLv& sm,
                           float omega, int nu, int nuc, bool split1) {
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
  // the coarsest level: one node is solved exactly (e = f / d); a hierarchy
  // cut above it smooths its coarsest level by 2 nuc damped Jacobi sweeps
  // from zero instead (a fixed symmetric polynomial)
  const bool exact = op.lv[L - 1].n == 1;
  if (split1 && L >= 3) {
    // level 1 split across the cluster, levels 2.. in every CTA
    unsigned ecur = 0;  // bit l: current smoother buffer of level l
    auto E = [&](int l) { return sm.e[l][(ecur >> l) & 1]; };
    auto Eo = [&](int l) { return sm.e[l][((ecur >> l) & 1) ^ 1]; };
    fast_restrict_split(b, v, cur, ch2, d, sm.f[1], sm.e[1][0], n1, omega, (float)op.lv[1].dinv);
    SEC_ADD(SEC_BAND);
    team_sync(t);
    SEC_ADD(SEC_SYNC);
    for (int s = 1; s < nuc; ++s) {
      csweep_split(b, op.lv[1], Eo(1), E(1), sm.f[1], omega);
      ecur ^= 2u;
      team_sync(t);
    }
    crestrict_split(b, op.lv[1], op.lv[2], E(1), sm.f[1], sm.f[2], sm.e[2][0], (L == 3 && exact) ? 1.f : omega);
    ecur &= ~4u;
    team_sync(t);
    SEC_ADD(SEC_COARSE);
    for (int c = 2; c < L - 1; ++c) {
      for (int s = 1; s < nuc; ++s) {
        csweep(b, op.lv[c], Eo(c), E(c), sm.f[c], omega);
        ecur ^= 1u << c;
        __syncthreads();
      }
      crestrict(b, op.lv[c], op.lv[c + 1], E(c), sm.f[c], sm.f[c + 1], sm.e[c + 1][0],
                (c + 1 == L - 1 && exact) ? 1.f : omega);
      ecur &= ~(1u << (c + 1));
      __syncthreads();
    }
    if (!exact) {
      for (int s = 1; s < 2 * nuc; ++s) {
        csweep(b, op.lv[L - 1], Eo(L - 1), E(L - 1), sm.f[L - 1], omega);
        ecur ^= 1u << (L - 1);
        __syncthreads();
      }
    }
    for (int c = L - 2; c >= 2; --c) {
      cprolong(b, op.lv[c], op.lv[c + 1], E(c), E(c + 1));
      __syncthreads();
      for (int s = 0; s < nuc; ++s) {
        csweep(b, op.lv[c], Eo(c), E(c), sm.f[c], omega);
        ecur ^= 1u << c;
        __syncthreads();
      }
    }
    SEC_ADD(SEC_COARSE2);
    cprolong_split(b, op.lv[1], op.lv[2], E(1), E(2));
    team_sync(t);
    for (int s = 0; s < nuc; ++s) {
      csweep_split(b, op.lv[1], Eo(1), E(1), sm.f[1], omega);
      ecur ^= 2u;
      team_sync(t);
    }
    SEC_ADD(SEC_COARSE);
    fast_prolong(b, v, cur, E(1), n1);
    cur ^= 1;
    SEC_ADD(SEC_BAND);
    team_sync(t);
    SEC_ADD(SEC_SYNC);
  } else {
  fast_restrict(b, v, cur, ch2, d, sm.f[1], n1);
  SEC_ADD(SEC_BAND);
  team_sync(t);
  SEC_ADD(SEC_SYNC);
  // every CTA: the coarse levels in its own shared memory
  {
    const OpLevel& l1 = op.lv[1];
    const float sc = (L == 2 && exact) ? 1.f : omega;
    const float d1inv = (float)l1.dinv;
    for_all(n1, b.warp, b.lane, b.nwarp, [&](int row, int col) {
      const int i = cidx(n1, row, col);
      s_fb[sm.e[1][0] + i] = sc * s_fb[sm.f[1] + i] * d1inv;
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
                (c + 1 == L - 1 && exact) ? 1.f : omega);
      ecur &= ~(1u << (c + 1));
      __syncthreads();
    }
    if (!exact) {
      for (int s = 1; s < 2 * nuc; ++s) {
        csweep(b, op.lv[L - 1], Eo(L - 1), E(L - 1), sm.f[L - 1], omega);
        ecur ^= 1u << (L - 1);
        __syncthreads();
      }
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
  }
  for (int s = 0; s < nu; ++s) {
    const bool last = (s == nu - 1);
    fast_sweep(b, v, cur, ch2, d, dinv, omega, last, rz);
    cur ^= 1;
    SEC_ADD(SEC_BAND);
    if (last) contribute(t, SL_RZ, (float)rz);
    SEC_ADD(SEC_REDUCE);
    team_sync(t);
    SEC_ADD(SEC_SYNC);
  }
  return cur;
}

// FP32 PCG on the band from a prepared state (R, E[0] set), updating X.
__device__ void fast_pcg(const Team& t, const Band& b, const FastVec& v, const Op& op, const CLv& sm, double tol2,
                         bool& done, const SolveCfg& cfg, Ctr& ctr, bool split1) {
  const OpLevel& l0 = op.lv[0];
  const float ch2 = (float)l0.ch2, d = 1.f + 4.f * ch2, dinv = (float)l0.dinv;
  const float omega = (float)cfg.omega;
  const float scale0 = (op.L == 1) ? 1.f : omega;
  int it_count = 0;
  double rz_old = 0.0;
  bool all = __syncthreads_and(done);
  while (!all) {
    const int zc = fast_vcycle(t, b, v, op, sm, omega, cfg.nu, cfg.nu_coarse, split1);
    SEC_T0();
    const int z = v.E[zc];
    const double rz = total_f(t, SL_RZ);
    SEC_ADD(SEC_REDUCE);
    const float beta = (float)((it_count == 0 || done || !(rz_old > 0.0)) ? 0.0 : rz / rz_old);
    float pqf = 0.f;
    const bool first = (it_count == 0);
    // phase A: p = z + beta p, q = A z + beta q (= A p), p.q
    for (int row = b.r0 + b.warp; row < b.r1; row += b.nwarp) {
      const int base = bidx(b, b.r0, row, 0);
#pragma unroll
      for (int j0 = 0; j0 < FAST_NJ; j0 += FAST_G) {
        float zc_[FAST_G], zn[FAST_G], pp[FAST_G], qq[FAST_G];
#pragma unroll
        for (int j = j0; j < j0 + FAST_G; ++j) {
          const int i = base + b.lane + 32 * j;
          if (b.lane + 32 * j < b.n) {
            zc_[j - j0] = s_fb[z + i];
            zn[j - j0] = bnb(b, z, i);
            if (!first) {
              pp[j - j0] = s_fb[v.P + i];
              qq[j - j0] = s_fb[v.Q + i];
            }
          }
        }
#pragma unroll
        for (int j = j0; j < j0 + FAST_G; ++j) {
          const int i = base + b.lane + 32 * j;
          if (b.lane + 32 * j < b.n) {
            const float az = d * zc_[j - j0] - ch2 * zn[j - j0];
            const float pv = first ? zc_[j - j0] : zc_[j - j0] + beta * pp[j - j0];
            const float qv = first ? az : az + beta * qq[j - j0];
            s_fb[v.P + i] = pv;
            s_fb[v.Q + i] = qv;
            pqf += pv * qv;
          }
        }
      }
    }
    SEC_ADD(SEC_BAND);
    contribute(t, SL_PQ, (float)pqf);
    SEC_ADD(SEC_REDUCE);
    team_sync(t);
    SEC_ADD(SEC_SYNC);
    const double pqt = total_f(t, SL_PQ);
    SEC_ADD(SEC_REDUCE);
    const float alpha = (float)((done || !(pqt > 0.0)) ? 0.0 : rz / pqt);
    float rrf = 0.f, rz1f = 0.f;
    // phase B: x += alpha p, r -= alpha q, first smoother sweep of the next
    // V-cycle. E[0] is written here; z may be E[0] but phase A has consumed it.
    {
      const BArr Xa = barr(b, v.X), Ra = barr(b, v.R), Ea = barr(b, v.E[0]);
      for (int row = b.r0 + b.warp; row < b.r1; row += b.nwarp) {
        const int base = bidx(b, b.r0, row, 0);
#pragma unroll
        for (int j0 = 0; j0 < FAST_NJ; j0 += FAST_G) {
          float xx[FAST_G], pp[FAST_G], rr_[FAST_G], qq[FAST_G];
#pragma unroll
          for (int j = j0; j < j0 + FAST_G; ++j) {
            const int i = base + b.lane + 32 * j;
            if (b.lane + 32 * j < b.n) {
              pp[j - j0] = s_fb[v.P + i];
              qq[j - j0] = s_fb[v.Q + i];
              rr_[j - j0] = s_fb[v.R + i];
              if (!first) xx[j - j0] = s_fb[v.X + i];
            }
          }
#pragma unroll
          for (int j = j0; j < j0 + FAST_G; ++j) {
            const int col = b.lane + 32 * j;
            if (col < b.n) {
              const float xv = first ? alpha * pp[j - j0] : xx[j - j0] + alpha * pp[j - j0];
              const float rv = rr_[j - j0] - alpha * qq[j - j0];
              bstore(b, Xa, row, col, xv);
              bstore(b, Ra, row, col, rv);
              rrf += rv * rv;
              const float e = scale0 * rv * dinv;
              bstore(b, Ea, row, col, e);
              if (op.L == 1) rz1f += rv * e;
            }
          }
        }
      }
    }
    SEC_ADD(SEC_BAND);
    contribute(t, SL_RR, (float)rrf);
    if (op.L == 1) contribute(t, SL_RZ, (float)rz1f);
    SEC_ADD(SEC_REDUCE);
    team_sync(t);
    SEC_ADD(SEC_SYNC);
    const double rrt = total_f(t, SL_RR);
    SEC_ADD(SEC_REDUCE);
    if (!isfinite(rrt)) {
      ctr.status |= STAT_NONFINITE;
      done = true;
    }
    done = done || (rrt <= tol2);
    ++it_count;
    rz_old = rz;
    const bool capped = it_count >= cfg.maxit;
    // an inner solve that stops at its cap is not a failure: the FP64
    // refinement around it decides convergence (and flags its own cap)
    all = __syncthreads_and(done) || capped;
  }
  ctr.iters += it_count;
  ctr.iters_max = max(ctr.iters_max, it_count);
}

// Right-hand side at node p: the previous state (double-float) plus the
// adjoint source B^T d (an FP64 sum over the sensors next to the node).
__device__ __forceinline__ df fast_rhs(const SweepParams& P, const float2* bsrc, const double* dsrc, int p) {
  df bv = bsrc ? df_load(bsrc + p) : df{0.f, 0.f};
  if (dsrc) {
    const int e0 = P.bt_ptr[p], e1 = P.bt_ptr[p + 1];
    if (e1 > e0) {
      double s = 0.0;
      for (int e = e0; e < e1; ++e) s += P.bt_w[e] * dsrc[P.bt_idx[e]];
      bv = df_add(bv, df_from_double(s));
    }
  }
  return bv;
}

// Solve (I + c L) x = b by iterative refinement around the band FP32
// MG-PCG; inner problems scaled by powers of two as in the generic kernel.
// The state x, the right-hand side b and the refinement residual
// r = b - (I + c L)(x + correction) are double-floats (about 48 bits: the
// residual of the outer tolerance 1e-10 is resolved with a wide margin);
// FP32 arithmetic runs at 64 times the FP64 rate here, and this pass was the
// FP64-bound fifth of the kernel. x and b live in global memory as float2
// (hi, lo) pairs.
__device__ float2* fast_solve(const Team& t, const Band& b, const SweepParams& P, const Op& op, float2* bd,
                              const FastVec& v, const CLv& sm, const float2* bsrc, const double* dsrc,
                              const float2* x0, float2* X1, float2* X2, Ctr& ctr) {
  const OpLevel& l0 = op.lv[0];
  const int n = b.n;
  const df ch2 = df_from_double(l0.ch2);
  const df dd = df_from_double(1.0 + 4.0 * l0.ch2);
  const float dinvf = (float)l0.dinv;
  const float omega = (float)P.cfg.omega;
  const float scale0 = (op.L == 1) ? 1.f : omega;
  const float2* xa = x0;
  float2* tgt = X1;
  float2* oth = X2;
  bool done = false;
  double bbt = 0.0;
  int ref = 0;
  const double inv_n = 1.0 / (double)l0.N;
  double sc = ctr.mix_scale;
  float isc_c = 1.f;  // 1 / scale of the current inner correction (a power of two)
  for (;; ++ref) {
    const bool first = (ref == 0);
    // sc is a power of two chosen so that the FP32 residual is O(1); the
    // scaled residual's squares are summed in FP32 and unscaled once
    const float scf = (float)sc;
    float rrs = 0.f;
    double bb = 0.0, rz1 = 0.0;
    SEC_T0();
    const BArr Ra = barr(b, v.R), Ea = barr(b, v.E[0]);
    const bool has_x = xa || !first;
    for (int row = b.r0 + b.warp; row < b.r1; row += b.nwarp) {
#pragma unroll
      for (int j0 = 0; j0 < FAST_NJ; ++j0) {
        const int col = b.lane + 32 * j0;
        if (col >= n) continue;
        const int p = row * n + col;
        df bp;
        if (first)
          bp = fast_rhs(P, bsrc, dsrc, p);
        else
          bp = dsrc ? df_load(bd + p) : (bsrc ? df_load(bsrc + p) : df{0.f, 0.f});
        df xcen = {0.f, 0.f}, ax = {0.f, 0.f};
        if (has_x) {
          // x + c / sc at the node and its four neighbours (c from the band
          // with halos; zero outside the grid)
          auto xc = [&](int rr_, int cc_) -> df {
            if (rr_ < 0 || rr_ >= n || cc_ < 0 || cc_ >= n) return df{0.f, 0.f};
            df s = xa ? df_load(xa + rr_ * n + cc_) : df{0.f, 0.f};
            if (!first) s = df_add_f(s, s_fb[v.X + bidx(b, b.r0, rr_, cc_)] * isc_c);
            return s;
          };
          xcen = xc(row, col);
          const df nb = df_add(df_add(xc(row, col - 1), xc(row, col + 1)), df_add(xc(row - 1, col), xc(row + 1, col)));
          ax = df_sub(df_mul(dd, xcen), df_mul(ch2, nb));
        }
        const df rd = df_sub(bp, ax);
        if (first) {
          if (dsrc) df_store(bd + p, bp);
          bb += (double)bp.hi * (double)bp.hi;
        }
        df_store(tgt + p, xcen);
        const float rf = rd.hi * scf;
        bstore(b, Ra, row, col, rf);
        const float e = scale0 * rf * dinvf;
        bstore(b, Ea, row, col, e);
        rrs = __fmaf_rn(rf, rf, rrs);
        if (op.L == 1) rz1 += (double)(rf * e);
      }
    }
    const double rr = (double)rrs / (sc * sc);
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
        for (int row = b.r0 + b.warp; row < b.r1; row += b.nwarp)
          for (int col = b.lane; col < n; col += 32) tgt[row * n + col] = make_float2(0.f, 0.f);
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
      // the refinement cap: the residual reached is reported with the status
      if (!done) ctr.max_res = fmax(ctr.max_res, bbt > 0.0 ? sqrt(rrt / bbt) : 0.0);
      ctr.status |= STAT_NOCONV;
      break;
    }
    bool idone = done;
    fast_pcg(t, b, v, op, sm, P.cfg.inner_rtol * P.cfg.inner_rtol * rrt * sc * sc, idone, P.cfg, ctr,
             P.fast_split1 != 0);
    xa = tgt;
    float2* tmp = tgt;
    tgt = oth;
    oth = tmp;
    isc_c = (float)(1.0 / sc);
    sc = pow2_inv(P.cfg.inner_rtol * sqrt(rrt * inv_n));
  }
  ctr.refines += ref;
  ctr.refine_max = max(ctr.refine_max, ref);
  ctr.solves += 1;
  return tgt;
}

__global__ void __launch_bounds__(FAST_THREADS, 1) fast2d_kernel(const SweepParams P) {
  __shared__ double s_red[2 * NSLOT * LRP_MAXBV];
  __shared__ double s_redw[32 * LRP_MAXBV];
  __shared__ float s_redf[2 * NSLOT * LRP_MAXBV];
  __shared__ float s_redwf[32 * LRP_MAXBV];
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
  t.redf = s_redf;
  t.redwf = s_redwf;
  t.phase = 0;
  const int team = blockIdx.x / P.C;
  const int n = P.step.lv[0].n;
#ifdef LRP_SECTION_TIMERS
  if (threadIdx.x < 12) s_sec[threadIdx.x] = 0;
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
  const int band_len = P.fast_band_len;
  v.E[0] = 0 * band_len + 1;
  v.E[1] = 1 * band_len + 1;
  v.R = 2 * band_len + 1;
  v.P = 3 * band_len + 1;
  v.Q = 4 * band_len + 1;
  v.X = 5 * band_len + 1;
  for (int i = t.tid; i < (int)(P.smem_bytes / sizeof(float)); i += t.NT) s_fb[i] = 0.f;
  CLv sm;
  for (int l = 0; l < LRP_MAXLEV; ++l) {
    sm.e[l][0] = (int)(P.smem_off[l][0] / sizeof(float));
    sm.e[l][1] = (int)(P.smem_off[l][1] / sizeof(float));
    sm.f[l] = (int)(P.smem_off[l][2] / sizeof(float));
  }
  // no neighbour may write into this CTA's halos before they are zeroed
  team_sync(t);
  char* base = P.ws + (size_t)team * P.team_bytes;
  // the implicit-Euler state buffers and the saved right-hand side hold
  // double-floats (hi, lo) in the space of the FP64 vectors
  float2* db[3];
  for (int k = 0; k < 3; ++k) db[k] = (float2*)(base + P.off_dbuf[k]);
  float2* bd = (float2*)(base + P.off_bd);
  double* obs = (double*)(base + P.off_obs);
  auto db_index = [&](const float2* x) { return x == db[0] ? 0 : (x == db[1] ? 1 : 2); };
  const int gcol = team;
  const bool valid = gcol < P.nvec;
  Ctr ctr;
  int cur = (P.stages & ST_LOAD_X) ? 0 : min(max(P.end_buf[team], 0), 2);
  auto for_own = [&](auto f) {
    for (int row = b.r0 + b.warp; row < b.r1; row += b.nwarp)
      for (int col = b.lane; col < n; col += 32) f(row, col);
  };
  // identity prior: Gamma_prior^{1/2} x = sqrt(gamma) x into the next buffer
  auto prior_scale = [&]() {
    const int nxt = (cur + 1) % 3;
    const df s = df_from_double(P.prior_scale);
    for_own([&](int row, int col) { df_store(db[nxt] + row * n + col, df_mul(s, df_load(db[cur] + row * n + col))); });
    team_sync(t);
    cur = nxt;
  };
  if (P.stages & ST_LOAD_X) {
    for_own([&](int row, int col) {
      const int p = row * n + col;
      df_store(db[0] + p, df_from_double(valid ? P.X[(size_t)gcol * P.ldx + p] : 0.0));
    });
    team_sync(t);
  }
  if (P.stages & ST_LOAD_D) {
    const int nd = P.n_obs * P.n_steps;
    for (int it = t.g; it < nd; it += t.S) obs[it] = valid ? P.Din[(size_t)gcol * P.lddin + it] : 0.0;
    team_sync(t);
  }
  if (P.stages & ST_PRIOR_IN) {
    if (P.prior_scale > 0.0) {
      prior_scale();
    } else {
      float2* res = fast_solve(t, b, P, P.prior, bd, v, sm, db[cur], nullptr, nullptr, db[(cur + 1) % 3],
                               db[(cur + 2) % 3], ctr);
      cur = db_index(res);
    }
  }
  if (P.stages & ST_FORWARD) {
    for (int step = P.t_begin + 1; step <= P.t_end; ++step) {
      float2* res = fast_solve(t, b, P, P.step, bd, v, sm, db[cur], nullptr, db[cur], db[(cur + 1) % 3],
                               db[(cur + 2) % 3], ctr);
      cur = db_index(res);
      if (P.n_steps > 0 && (step % P.obs_every) == 0 && step / P.obs_every <= P.n_steps) {
        const int k = step / P.obs_every - 1;
        for (int s = t.g; s < P.n_obs; s += t.S) {
          double y = 0.0;
          for (int c = 0; c < 8; ++c) {
            const int node = P.obs_node[s * 8 + c];
            if (node >= 0) y += P.obs_w[s * 8 + c] * df_to_double(df_load(res + node));
          }
          obs[(size_t)k * P.n_obs + s] = y * P.inv_sigma2;
          if ((P.stages & ST_STORE_D) && valid) P.Dout[(size_t)gcol * P.lddout + k * P.n_obs + s] = y;
        }
      }
      if ((P.stages & ST_TRAJ) && valid) {
        double* dst = P.traj + ((size_t)gcol * P.traj_cols + (step - P.t_begin - 1)) * P.traj_ld;
        for_own([&](int row, int col) { dst[row * n + col] = df_to_double(df_load(res + row * n + col)); });
      }
    }
    team_sync(t);
  }
  if (P.stages & ST_ADJOINT) {
    const float2* q = nullptr;
    for (int step = P.adj_begin; step >= 1; --step) {
      const bool is_obs = (step % P.obs_every) == 0 && step / P.obs_every <= P.n_steps;
      if (!q && !is_obs) continue;
      const double* dsrc = is_obs ? obs + (size_t)(step / P.obs_every - 1) * P.n_obs : nullptr;
      const int qi = q ? db_index(q) : cur;
      q = fast_solve(t, b, P, P.step, bd, v, sm, q, dsrc, q, db[(qi + 1) % 3], db[(qi + 2) % 3], ctr);
      if ((P.stages & ST_TRAJ_ADJ) && valid) {
        double* dst = P.traj + ((size_t)gcol * P.traj_cols + (step - 1)) * P.traj_ld;
        for_own([&](int row, int col) { dst[row * n + col] = df_to_double(df_load(q + row * n + col)); });
      }
    }
    if (q) {
      cur = db_index(q);
    } else {
      for_own([&](int row, int col) { db[cur][row * n + col] = make_float2(0.f, 0.f); });
      team_sync(t);
    }
  }
  if (P.stages & ST_PRIOR_OUT) {
    if (P.prior_scale > 0.0) {
      prior_scale();
    } else {
      float2* res = fast_solve(t, b, P, P.prior, bd, v, sm, db[cur], nullptr, nullptr, db[(cur + 1) % 3],
                               db[(cur + 2) % 3], ctr);
      cur = db_index(res);
    }
  }
  if ((P.stages & ST_STORE_Y) && valid) {
    for_own([&](int row, int col) {
      const int p = row * n + col;
      P.Y[(size_t)gcol * P.ldy + p] = df_to_double(df_load(db[cur] + p));
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
    for (int k = 0; k < 11; ++k) P.section_cycles[k] = s_sec[k];
    P.section_cycles[11] = (unsigned long long)(clock64() - k_t0);
  }
#endif
}

}  // namespace lrp
