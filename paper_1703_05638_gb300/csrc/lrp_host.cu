// Host side of the library: problem setup (grid, multigrid hierarchy,
// sensors), pointer staging, error handling and the sweep-based entry points
// (Hessian apply, forward map, adjoint, prior half-apply).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "lrp_dense.h"
#include "lrp_internal.h"

namespace lrp {

static thread_local std::string g_err = "no error";
static std::atomic<unsigned long long> g_launches{0};

void note_launch(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void set_error(const std::string& msg) { g_err = msg; }

lrp_status cuda_status(cudaError_t e, const char* where) {
  set_error(std::string(where) + ": " + cudaGetErrorString(e));
  cudaGetLastError();  // clear sticky non-fatal state
  return e == cudaErrorMemoryAllocation ? LRP_ENOMEM : LRP_ECUDA;
}

// Allocation-failure injection (lrp_debug_fail_alloc): when armed, the
// allocation after `fail_after` further successful ones returns
// cudaErrorMemoryAllocation once, as a full device would.
static std::atomic<long long> g_fail_after{-1};

cudaError_t dev_malloc_raw(void** p, size_t bytes) {
  long long n = g_fail_after.load();
  while (n >= 0) {
    if (g_fail_after.compare_exchange_weak(n, n - 1)) {
      if (n == 0) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
      }
      break;
    }
  }
  return cudaMalloc(p, bytes);
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device arrays must live on the problem's device: the kernels read them
// directly, and memory of another GPU without peer access would fault. NULL,
// host and managed memory pass; device memory of another device is
// LRP_EINVAL.
lrp_status check_on_device(int device, const void* p, const char* what) {
  if (!p) return LRP_OK;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return LRP_OK;
  }
  if (a.type == cudaMemoryTypeDevice && a.device != device) {
    set_error(std::string(what) + ": device array on device " + std::to_string(a.device) +
              ", the problem is on device " + std::to_string(device));
    return LRP_EINVAL;
  }
  return LRP_OK;
}

template <typename T>
static lrp_status dev_alloc(lrp_problem* P, T** out, size_t count) {
  void* p = nullptr;
  cudaError_t e = lrp::dev_malloc(&p, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) return cuda_status(e, "cudaMalloc");
  P->allocs.push_back(p);
  P->dev_bytes += std::max<size_t>(count, 1) * sizeof(T);
  *out = (T*)p;
  return LRP_OK;
}

template <typename T>
static lrp_status upload(lrp_problem* P, T** out, const std::vector<T>& v) {
  lrp_status s = dev_alloc(P, out, v.size());
  if (s != LRP_OK) return s;
  if (!v.empty()) {
    cudaError_t e = cudaMemcpy(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_status(e, "upload");
  }
  return LRP_OK;
}

lrp_status ensure_workspace(lrp_problem* P, size_t bytes) {
  if (bytes <= P->ws_bytes) return LRP_OK;
  if (P->ws) {
    cudaStreamSynchronize(P->stream);
    cudaFree(P->ws);
    P->ws = nullptr;
    P->ws_bytes = 0;
  }
  size_t want = bytes + bytes / 8;
  cudaError_t e = lrp::dev_malloc((void**)&P->ws, want);
  if (e != cudaSuccess) return cuda_status(e, "workspace cudaMalloc");
  P->ws_bytes = want;
  if (P->poison) cudaMemset(P->ws, P->poison & 0xFF, want);  // 0xFF bytes: NaN in FP32 and FP64
  return LRP_OK;
}

static uint64_t fnv1a(uint64_t h, const void* data, size_t n) {
  const unsigned char* c = (const unsigned char*)data;
  for (size_t i = 0; i < n; ++i) {
    h ^= c[i];
    h *= 1099511628211ull;
  }
  return h;
}

// Face array sizes of one level (faces normal to axis d): n+1 along d, n elsewhere.
static size_t face_count(int n, int dim) { return (size_t)(n + 1) * (size_t)std::pow(n, dim - 1); }

// Coarse face diffusivity: the coarse face between coarse nodes I-1 and I
// along axis d spans the two fine faces 2I and 2I+1 along d (transverse
// coarse index J -> fine index 2J+1); take their harmonic mean (series
// conduction through the two fine cells).
static std::vector<double> coarsen_faces(const std::vector<double>& kf, int nf, int dim, int d) {
  const int nc = (nf - 1) / 2;
  std::vector<double> kc(face_count(nc, dim));
  int ext_f[3], ext_c[3];
  for (int a = 0; a < 3; ++a) {
    ext_f[a] = (a < dim) ? (a == d ? nf + 1 : nf) : 1;
    ext_c[a] = (a < dim) ? (a == d ? nc + 1 : nc) : 1;
  }
  for (int c2 = 0; c2 < ext_c[2]; ++c2)
    for (int c1 = 0; c1 < ext_c[1]; ++c1)
      for (int c0 = 0; c0 < ext_c[0]; ++c0) {
        int cc[3] = {c0, c1, c2};
        int f[3];
        for (int a = 0; a < 3; ++a) f[a] = (a < dim) ? (a == d ? 2 * cc[a] : 2 * cc[a] + 1) : 0;
        const size_t i1 = (size_t)f[0] + (size_t)ext_f[0] * ((size_t)f[1] + (size_t)ext_f[1] * f[2]);
        f[d] += 1;
        const size_t i2 = (size_t)f[0] + (size_t)ext_f[0] * ((size_t)f[1] + (size_t)ext_f[1] * f[2]);
        const double a = kf[i1], b = kf[i2];
        kc[(size_t)c0 + (size_t)ext_c[0] * ((size_t)c1 + (size_t)ext_c[1] * c2)] = 2.0 * a * b / (a + b);
      }
  return kc;
}

static void default_tuning(lrp_problem* P) {
  const lrp_problem_desc& d = P->desc;
  P->nthreads = 512;
  P->team_cols = d.team_cols > 0 ? d.team_cols : 1;
  if (d.team_ctas > 0) {
    P->team_ctas = d.team_ctas;
  } else if (P->nx >= 16129) {
    P->team_ctas = 8;
  } else if (P->nx >= 3969) {
    P->team_ctas = 4;
  } else {
    P->team_ctas = 1;
  }
  P->coarse_items = d.coarse_items > 0 ? d.coarse_items : 1024;
  P->kernel_variant = d.kernel_variant;
  P->smem_cap = 160 * 1024;
}

}  // namespace lrp

using namespace lrp;

extern "C" {

const char* lrp_last_error(void) { return g_err.c_str(); }

const char* lrp_version(void) { return "lrpost-gb300 0.1"; }

unsigned long long lrp_kernel_launches(void) { return g_launches.load(); }

void lrp_debug_fail_alloc(long long after) { lrp::g_fail_after.store(after < 0 ? -1 : after); }

lrp_status lrp_setup_problem(const lrp_problem_desc* desc, void* cuda_stream, lrp_problem** out) {
  if (!desc || !out) {
    set_error("lrp_setup_problem: NULL argument");
    return LRP_EINVAL;
  }
  *out = nullptr;
  const lrp_problem_desc& d = *desc;
  if (d.dim != 2 && d.dim != 3) {
    set_error("dim must be 2 or 3");
    return LRP_EINVAL;
  }
  int L = 0;
  while ((1 << L) - 1 < d.n) ++L;
  if (d.n < 1 || (1 << L) - 1 != d.n || L > LRP_MAXLEV) {
    set_error("n must be 2^L - 1 with 1 <= L <= 10");
    return LRP_EINVAL;
  }
  const long long nx = (long long)std::pow((double)d.n, d.dim);
  if (nx * LRP_MAXBV >= (1ll << 31)) {
    set_error("grid too large for 32-bit item indexing");
    return LRP_EINVAL;
  }
  if (d.nt < 1 || !(d.T > 0) || !(d.sigma > 0) || !(d.prior_alpha >= 0) || d.n_obs < 1 ||
      !d.obs_xyz || d.obs_every < 1 || d.obs_every > d.nt) {
    set_error("invalid nt/T/sigma/alpha/sensors/obs_every");
    return LRP_EINVAL;
  }
  if (d.precision != LRP_FP64 && d.precision != LRP_MIXED) {
    set_error("precision must be LRP_FP64 or LRP_MIXED");
    return LRP_EINVAL;
  }
  if (d.pde != LRP_PDE_HEAT && d.pde != LRP_PDE_CONVDIFF) {
    set_error("pde must be LRP_PDE_HEAT or LRP_PDE_CONVDIFF");
    return LRP_EINVAL;
  }
  if (d.pde == LRP_PDE_CONVDIFF) {
    bool ok = d.precision == LRP_FP64 && !d.kappa_faces && d.conv_nu >= 0 && std::isfinite(d.conv_nu);
    for (int a = 0; a < d.dim; ++a) ok = ok && std::isfinite(d.wind[a]);
    if (!ok) {
      set_error("LRP_PDE_CONVDIFF needs LRP_FP64, no kappa field, a finite conv_nu >= 0 and a finite wind");
      return LRP_EINVAL;
    }
  }
  if (d.prior_kind != LRP_PRIOR_LAPLACE && d.prior_kind != LRP_PRIOR_IDENTITY) {
    set_error("prior_kind must be LRP_PRIOR_LAPLACE or LRP_PRIOR_IDENTITY");
    return LRP_EINVAL;
  }
  if (d.prior_kind == LRP_PRIOR_IDENTITY && !(d.prior_gamma > 0 && std::isfinite(d.prior_gamma))) {
    set_error("LRP_PRIOR_IDENTITY needs a finite prior_gamma > 0");
    return LRP_EINVAL;
  }
  if (d.team_cols != 0 && (d.team_cols < 1 || d.team_cols > LRP_MAXBV || (d.team_cols & (d.team_cols - 1)))) {
    set_error("team_cols must be a power of two <= 16");
    return LRP_EINVAL;
  }
  if (d.team_ctas < 0 || d.team_ctas > 16) {
    set_error("team_ctas must be in 0..16");
    return LRP_EINVAL;
  }
  for (int i = 0; i < d.n_obs * d.dim; ++i) {
    if (!std::isfinite(d.obs_xyz[i])) {
      set_error("non-finite sensor coordinate");
      return LRP_ENONFINITE;
    }
    if (!(d.obs_xyz[i] > 0.0 && d.obs_xyz[i] < 1.0)) {
      set_error("sensor coordinate outside (0,1)");
      return LRP_EINVAL;
    }
  }
  lrp_problem* P = new lrp_problem();
  P->desc = d;
  P->desc.kappa_faces = nullptr;
  P->desc.obs_xyz = nullptr;
  P->dim = d.dim;
  P->n = d.n;
  P->nx = (int)nx;
  P->nt = d.nt;
  P->L = L;
  P->n_obs = d.n_obs;
  P->n_steps = d.nt / d.obs_every;
  P->n_data = P->n_obs * P->n_steps;
  P->last_obs = P->n_steps * d.obs_every;
  P->tau = d.T / d.nt;
  P->h = 1.0 / (d.n + 1);
  P->stream = (cudaStream_t)cuda_stream;
  cudaGetDevice(&P->device);
  cudaDeviceGetAttribute(&P->sm_count, cudaDevAttrMultiProcessorCount, P->device);
  P->ws = nullptr;
  P->ws_bytes = 0;
  P->prof_on = 0;
  P->prof_ev[0] = P->prof_ev[1] = nullptr;
  {
    const char* pz = std::getenv("LRP_POISON");  // byte value to fill new workspace with (1 -> 0xFF)
    P->poison = pz ? (std::atoi(pz) == 1 ? 0xFF : (std::atoi(pz) | 0x100)) : 0;
  }
  P->ws_fixed = nullptr;
  P->ws_fixed_bytes = 0;
  auto fail = [&](lrp_status s) {
    lrp_problem_destroy(P);
    return s;
  };
  // ---- multigrid hierarchy of both operators
  const bool has_kappa = d.kappa_faces != nullptr;
  P->step.L = P->prior.L = L;
  P->step.has_kappa = has_kappa ? 1 : 0;
  P->prior.has_kappa = 0;
  P->step.conv = d.pde == LRP_PDE_CONVDIFF ? 1 : 0;
  P->prior.conv = 0;
  std::vector<std::vector<double>> kcur(d.dim);
  if (has_kappa) {
    size_t off = 0;
    for (int a = 0; a < d.dim; ++a) {
      const size_t cnt = face_count(d.n, d.dim);
      kcur[a].assign(d.kappa_faces + off, d.kappa_faces + off + cnt);
      off += cnt;
      for (double v : kcur[a])
        if (!std::isfinite(v) || !(v > 0.0)) {
          set_error("kappa must be finite and positive");
          return fail(std::isfinite(v) ? LRP_EINVAL : LRP_ENONFINITE);
        }
    }
  }
  uint64_t hash = 1469598103934665603ull;
  hash = fnv1a(hash, &d.dim, sizeof(int));
  hash = fnv1a(hash, &d.n, sizeof(int));
  hash = fnv1a(hash, &d.nt, sizeof(int));
  hash = fnv1a(hash, &d.T, sizeof(double));
  hash = fnv1a(hash, &d.prior_alpha, sizeof(double));
  hash = fnv1a(hash, &d.prior_kind, sizeof(int));
  if (d.prior_kind == LRP_PRIOR_IDENTITY) hash = fnv1a(hash, &d.prior_gamma, sizeof(double));
  hash = fnv1a(hash, &d.obs_every, sizeof(int));
  hash = fnv1a(hash, &d.pde, sizeof(int));
  if (d.pde == LRP_PDE_CONVDIFF) {
    hash = fnv1a(hash, &d.conv_nu, sizeof(double));
    hash = fnv1a(hash, d.wind, sizeof(double) * d.dim);
  }
  hash = fnv1a(hash, d.obs_xyz, sizeof(double) * d.n_obs * d.dim);
  for (int l = 0; l < L; ++l) {
    const int nl = ((d.n + 1) >> l) - 1;
    const double h2inv = (double)(nl + 1) * (double)(nl + 1);
    for (Op* op : {&P->step, &P->prior}) {
      OpLevel& lv = op->lv[l];
      lv.n = nl;
      lv.N = (int)std::pow((double)nl, d.dim);
      lv.dn = make_fastdiv((uint32_t)nl);
      for (int a = 0; a < 3; ++a) {
        lv.kd[a] = nullptr;
        lv.kf[a] = nullptr;
      }
    }
    P->step.lv[l].ch2 = P->tau * h2inv;
    P->prior.lv[l].ch2 = d.prior_alpha * h2inv;
    P->step.lv[l].dinv = 1.0 / (1.0 + P->step.lv[l].ch2 * 2 * d.dim);
    for (int a = 0; a < 3; ++a) P->step.lv[l].cw[a] = P->prior.lv[l].cw[a] = 0.0;
    if (d.pde == LRP_PDE_CONVDIFF) {
      // I + tau (nu (-Laplace) + w . grad): diffusion in ch2, upwind convection in cw
      P->step.lv[l].ch2 = P->tau * d.conv_nu * h2inv;
      double cs = 0.0;
      for (int a = 0; a < d.dim; ++a) {
        P->step.lv[l].cw[a] = P->tau * d.wind[a] * (double)(nl + 1);
        cs += std::fabs(P->step.lv[l].cw[a]);
      }
      P->step.lv[l].dinv = 1.0 / (1.0 + P->step.lv[l].ch2 * 2 * d.dim + cs);
    }
    P->prior.lv[l].dinv = 1.0 / (1.0 + P->prior.lv[l].ch2 * 2 * d.dim);
    P->step.lv[l].dinvd = P->prior.lv[l].dinvd = nullptr;
    P->step.lv[l].dinvf = P->prior.lv[l].dinvf = nullptr;
    if (has_kappa) {
      for (int a = 0; a < d.dim; ++a) {
        if (l > 0) kcur[a] = coarsen_faces(kcur[a], ((d.n + 1) >> (l - 1)) - 1, d.dim, a);
        if (l == 0) hash = fnv1a(hash, kcur[a].data(), kcur[a].size() * sizeof(double));
        double* kd = nullptr;
        float* kf = nullptr;
        lrp_status s = upload(P, &kd, kcur[a]);
        if (s != LRP_OK) return fail(s);
        std::vector<float> f32(kcur[a].begin(), kcur[a].end());
        s = upload(P, &kf, f32);
        if (s != LRP_OK) return fail(s);
        P->step.lv[l].kd[a] = kd;
        P->step.lv[l].kf[a] = kf;
      }
      // per-node inverse diagonal 1 / (1 + (tau/h^2) sum of the node's face kappas)
      const int nl = P->step.lv[l].n, Nl = P->step.lv[l].N;
      std::vector<double> dinv(Nl);
      for (int p = 0; p < Nl; ++p) {
        int ii[3] = {p % nl, (p / nl) % nl, p / (nl * nl)};
        double ks = 0.0;
        for (int a = 0; a < d.dim; ++a) {
          int ext[3];
          for (int b = 0; b < 3; ++b) ext[b] = (b < d.dim) ? (b == a ? nl + 1 : nl) : 1;
          int f[3] = {ii[0], ii[1], d.dim == 3 ? ii[2] : 0};
          const size_t lo = (size_t)f[0] + (size_t)ext[0] * ((size_t)f[1] + (size_t)ext[1] * f[2]);
          f[a] += 1;
          const size_t hi = (size_t)f[0] + (size_t)ext[0] * ((size_t)f[1] + (size_t)ext[1] * f[2]);
          ks += kcur[a][lo] + kcur[a][hi];
        }
        dinv[p] = 1.0 / (1.0 + P->step.lv[l].ch2 * ks);
      }
      double* dd = nullptr;
      float* df = nullptr;
      lrp_status s2 = upload(P, &dd, dinv);
      if (s2 != LRP_OK) return fail(s2);
      std::vector<float> dinv32(dinv.begin(), dinv.end());
      s2 = upload(P, &df, dinv32);
      if (s2 != LRP_OK) return fail(s2);
      P->step.lv[l].dinvd = dd;
      P->step.lv[l].dinvf = df;
    }
  }
  P->hash = hash;
  // ---- sensors: 2^dim interpolation corners each (node -1 = unused)
  const double h = P->h;
  std::vector<int> onode((size_t)d.n_obs * 8, -1);
  std::vector<double> ow((size_t)d.n_obs * 8, 0.0);
  std::vector<std::vector<std::pair<int, double>>> bt(P->nx);
  for (int s = 0; s < d.n_obs; ++s) {
    int base[3] = {0, 0, 0};
    double fr[3] = {0, 0, 0};
    for (int a = 0; a < d.dim; ++a) {
      const double t = d.obs_xyz[s * d.dim + a] / h;
      const double c = std::floor(t);
      base[a] = (int)c - 1;
      fr[a] = t - c;
    }
    int slot = 0;
    for (int corner = 0; corner < (1 << d.dim); ++corner) {
      double w = 1.0;
      int idx[3] = {0, 0, 0};
      bool inside = true;
      for (int a = 0; a < d.dim; ++a) {
        const int up = (corner >> a) & 1;
        w *= up ? fr[a] : (1.0 - fr[a]);
        idx[a] = base[a] + up;
        if (idx[a] < 0 || idx[a] > d.n - 1) inside = false;
      }
      if (w == 0.0 || !inside) continue;
      const int node = idx[0] + d.n * (idx[1] + d.n * idx[2]);
      onode[s * 8 + slot] = node;
      ow[s * 8 + slot] = w;
      ++slot;
      bt[node].push_back({s, w});
    }
  }
  std::vector<int> bptr(P->nx + 1, 0), bidx;
  std::vector<double> bw;
  for (int p = 0; p < P->nx; ++p) {
    std::sort(bt[p].begin(), bt[p].end());
    bptr[p + 1] = bptr[p] + (int)bt[p].size();
    for (auto& e : bt[p]) {
      bidx.push_back(e.first);
      bw.push_back(e.second);
    }
  }
  lrp_status s;
  if ((s = upload(P, &P->obs_node, onode)) != LRP_OK) return fail(s);
  if ((s = upload(P, &P->obs_w, ow)) != LRP_OK) return fail(s);
  if ((s = upload(P, &P->bt_ptr, bptr)) != LRP_OK) return fail(s);
  if ((s = upload(P, &P->bt_idx, bidx)) != LRP_OK) return fail(s);
  if ((s = upload(P, &P->bt_w, bw)) != LRP_OK) return fail(s);
  if ((s = dev_alloc(P, &P->stats, 1)) != LRP_OK) return fail(s);
  if ((s = dev_alloc(P, &P->end_buf, 65536)) != LRP_OK) return fail(s);
  {
    const cudaError_t e = cudaMemset(P->end_buf, 0, 65536 * sizeof(int));
    if (e != cudaSuccess) return fail(cuda_status(e, "end_buf"));
  }
  // ---- solver configuration
  SolveCfg& c = P->cfg;
  const bool mixed = d.precision == LRP_MIXED;
  c.rtol = d.solve_rtol > 0 ? d.solve_rtol : (mixed ? 1e-10 : 1e-13);
  c.inner_rtol = d.inner_rtol > 0 ? d.inner_rtol : 1e-4;
  c.maxit = d.pcg_maxit > 0 ? d.pcg_maxit : 200;
  c.maxref = 30;
  c.nu = d.mg_nu > 0 ? d.mg_nu : 2;
  c.nu_coarse = d.mg_nu_coarse > 0 ? d.mg_nu_coarse : c.nu;
  c.omega = d.dim == 2 ? 0.8 : 6.0 / 7.0;
  if (d.mg_levels != 0 && (d.mg_levels < 3 || d.mg_levels > L)) {
    set_error("mg_levels must be 0 or in 3..levels of the grid");
    return fail(LRP_EINVAL);
  }
  c.mg_levels = d.mg_levels;
  if (P->desc.time_chunk <= 0) P->desc.time_chunk = 16;
  if (P->desc.time_rank_max <= 0) P->desc.time_rank_max = 40;
  if (!(P->desc.time_trunc_tol > 0)) P->desc.time_trunc_tol = 1e-8;
  default_tuning(P);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(cuda_status(e, "setup"));
  *out = P;
  return LRP_OK;
}

lrp_status lrp_sweep_profile(lrp_problem* P, int mode, int kernel, double* ms, unsigned long long* launches,
                             double* algo_bytes) {
  if (!P || kernel < 0 || kernel > 4) {
    set_error("lrp_sweep_profile: NULL problem or kernel not in 0..4");
    return LRP_EINVAL;
  }
  if (ms) *ms = P->prof_ms[kernel];
  if (launches) *launches = P->prof_launches[kernel];
  if (algo_bytes) *algo_bytes = P->prof_bytes[kernel];
  if (mode >= 0) {
    if (mode == 1 && !P->prof_ev[0]) {
      cudaEventCreate(&P->prof_ev[0]);
      cudaEventCreate(&P->prof_ev[1]);
    }
    P->prof_on = (mode == 1) && P->prof_ev[0];
    for (int v = 0; v < 5; ++v) {
      P->prof_ms[v] = 0.0;
      P->prof_bytes[v] = 0.0;
      P->prof_launches[v] = 0;
    }
  }
  return LRP_OK;
}

lrp_status lrp_problem_tuning(const lrp_problem* P, lrp_tuning* out) {
  if (!P || !out) {
    set_error("lrp_problem_tuning: NULL argument");
    return LRP_EINVAL;
  }
  out->team_ctas = P->team_ctas;
  out->team_cols = P->team_cols;
  out->mg_nu = P->cfg.nu;
  out->mg_nu_coarse = P->cfg.nu_coarse;
  out->inner_rtol = P->cfg.inner_rtol;
  out->last_kernel = P->last_kernel;
  out->last_team_ctas = P->last_team_ctas;
  out->threads = P->nthreads;
  out->waves = P->allow_waves;
  out->team_ctas_narrow = P->team_ctas_narrow;
  out->mg_levels = P->cfg.mg_levels;
  return LRP_OK;
}

lrp_status lrp_set_tuning(lrp_problem* P, const lrp_tuning* t) {
  if (!P || !t) {
    set_error("lrp_set_tuning: NULL argument");
    return LRP_EINVAL;
  }
  if (t->team_ctas < 1 || t->team_ctas > 16 || t->team_cols < 1 || t->team_cols > LRP_MAXBV ||
      (t->team_cols & (t->team_cols - 1)) || t->mg_nu < 1 || t->mg_nu > 8 || t->mg_nu_coarse < 1 ||
      t->mg_nu_coarse > 8 || !(t->inner_rtol > 0 && t->inner_rtol < 1) || (t->threads != 256 && t->threads != 512) ||
      t->team_ctas_narrow < 0 || t->team_ctas_narrow > 16 ||
      (t->mg_levels != 0 && (t->mg_levels < 3 || t->mg_levels > P->L))) {
    set_error("lrp_set_tuning: value out of range");
    return LRP_EINVAL;
  }
  P->team_ctas = t->team_ctas;
  P->team_cols = t->team_cols;
  P->nthreads = t->threads;
  P->allow_waves = t->waves ? 1 : 0;
  P->team_ctas_narrow = t->team_ctas_narrow;
  P->cfg.nu = t->mg_nu;
  P->cfg.nu_coarse = t->mg_nu_coarse;
  P->cfg.inner_rtol = t->inner_rtol;
  P->cfg.mg_levels = t->mg_levels;
  return LRP_OK;
}

void lrp_problem_destroy(lrp_problem* P) {
  if (!P) return;
  if (P->stream) cudaStreamSynchronize(P->stream);
  if (P->prof_ev[0]) cudaEventDestroy(P->prof_ev[0]);
  if (P->prof_ev[1]) cudaEventDestroy(P->prof_ev[1]);
  for (void* p : P->allocs) cudaFree(p);
  if (P->ws) cudaFree(P->ws);
  delete P;
}

lrp_status lrp_problem_sizes(const lrp_problem* P, int* nx, int* n_obs, int* n_steps, int* n_data) {
  if (!P) {
    set_error("NULL problem");
    return LRP_EINVAL;
  }
  if (nx) *nx = P->nx;
  if (n_obs) *n_obs = P->n_obs;
  if (n_steps) *n_steps = P->n_steps;
  if (n_data) *n_data = P->n_data;
  return LRP_OK;
}

}  // extern "C"

namespace lrp {

// Stages a (rows x cols, leading dimension ld) column-major block to the device
// if it lives on the host. *dev receives a device pointer with leading
// dimension *dld; tmp owns any staging allocation.
struct Staged {
  void* tmp = nullptr;
  ~Staged() {
    if (tmp) cudaFree(tmp);
  }
};

static lrp_status stage_in(lrp_problem* P, const double* src, int rows, int cols, int ld,
                           const double** dev, int* dld, Staged& st) {
  if (is_device_ptr(src)) {
    *dev = src;
    *dld = ld;
    return LRP_OK;
  }
  cudaError_t e = lrp::dev_malloc(&st.tmp, (size_t)rows * cols * sizeof(double) + 8);
  if (e != cudaSuccess) return cuda_status(e, "staging cudaMalloc");
  e = cudaMemcpy2DAsync(st.tmp, (size_t)rows * sizeof(double), src, (size_t)ld * sizeof(double),
                        (size_t)rows * sizeof(double), cols, cudaMemcpyHostToDevice, P->stream);
  if (e != cudaSuccess) return cuda_status(e, "staging copy");
  *dev = (const double*)st.tmp;
  *dld = rows;
  return LRP_OK;
}

static lrp_status stage_out_alloc(lrp_problem* P, double* dst, int rows, int cols, int ld,
                                  double** dev, int* dld, Staged& st) {
  (void)P;
  if (is_device_ptr(dst)) {
    *dev = dst;
    *dld = ld;
    return LRP_OK;
  }
  cudaError_t e = lrp::dev_malloc(&st.tmp, (size_t)rows * cols * sizeof(double) + 8);
  if (e != cudaSuccess) return cuda_status(e, "staging cudaMalloc");
  *dev = (double*)st.tmp;
  *dld = rows;
  return LRP_OK;
}

static lrp_status stage_out_copy(lrp_problem* P, double* dst, int rows, int cols, int ld,
                                 const double* dev, int dld) {
  if (dev == dst) return LRP_OK;
  cudaError_t e = cudaMemcpy2DAsync(dst, (size_t)ld * sizeof(double), dev, (size_t)dld * sizeof(double),
                                    (size_t)rows * sizeof(double), cols, cudaMemcpyDeviceToHost, P->stream);
  if (e != cudaSuccess) return cuda_status(e, "staging copy back");
  e = cudaStreamSynchronize(P->stream);
  if (e != cudaSuccess) return cuda_status(e, "staging sync");
  return LRP_OK;
}

static lrp_status check_common(lrp_problem* P, int nvec, int ld_in, int rows_in, int ld_out, int rows_out,
                               const void* in, const void* out) {
  if (!P || !in || !out) {
    set_error("NULL argument");
    return LRP_EINVAL;
  }
  if (nvec < 0 || ld_in < rows_in || ld_out < rows_out) {
    set_error("invalid nvec or leading dimension");
    return LRP_EINVAL;
  }
  lrp_status s = check_on_device(P->device, in, "input");
  if (s == LRP_OK) s = check_on_device(P->device, out, "output");
  if (s != LRP_OK) return s;
  cudaSetDevice(P->device);
  return LRP_OK;
}

lrp_status sweep_call(lrp_problem* P, unsigned stages, int nvec, const double* in, int ldin, int rows_in,
                      double* out, int ldout, int rows_out, bool in_is_d, bool out_is_d,
                      lrp_apply_stats* st, bool misfit_only) {
  lrp_status s = check_common(P, nvec, ldin, rows_in, ldout, rows_out, in, out);
  if (s != LRP_OK) return s;
  if (nvec == 0) return LRP_OK;
  auto t0 = std::chrono::steady_clock::now();
  Staged sin, sout;
  const double* din;
  int dldin;
  double* dout;
  int dldout;
  if ((s = stage_in(P, in, rows_in, nvec, ldin, &din, &dldin, sin)) != LRP_OK) return s;
  if ((s = stage_out_alloc(P, out, rows_out, nvec, ldout, &dout, &dldout, sout)) != LRP_OK) return s;
  s = run_sweep(P, stages, nvec, in_is_d ? nullptr : din, dldin, out_is_d ? nullptr : dout, dldout,
                in_is_d ? din : nullptr, dldin, out_is_d ? dout : nullptr, dldout, st, misfit_only);
  if (s != LRP_OK && s != LRP_ENOCONV) return s;
  lrp_status s2 = stage_out_copy(P, out, rows_out, nvec, ldout, dout, dldout);
  if (s2 != LRP_OK) return s2;
  if (st) st->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return s;
}

// Hessian apply whose forward trajectory is carried in low-rank-in-time form
// (chunked forward sweep + streaming recompression, then the adjoint sweep).
static lrp_status hessian_with_factors(lrp_problem* P, int nvec, const double* X, int ldx, double* Y, int ldy,
                                       bool misfit, lrp_apply_stats* st) {
  lrp_status s = check_common(P, nvec, ldx, P->nx, ldy, P->nx, X, Y);
  if (s != LRP_OK) return s;
  if (nvec == 0) return LRP_OK;
  Staged sin, sout;
  const double* din;
  int dldin;
  double* dout;
  int dldout;
  if ((s = stage_in(P, X, P->nx, nvec, ldx, &din, &dldin, sin)) != LRP_OK) return s;
  if ((s = stage_out_alloc(P, Y, P->nx, nvec, ldy, &dout, &dldout, sout)) != LRP_OK) return s;
  if (misfit) {
    set_error("LRP_KEEP_TRAJ_FACTORS is supported with the prior-preconditioned Hessian only");
    return LRP_EINVAL;
  }
  s = trajectory_factors_impl(P, nvec, din, dldin, nullptr, nullptr, nullptr, st, true, dout, dldout);
  if (s != LRP_OK && s != LRP_ENOCONV) return s;
  lrp_status s2 = stage_out_copy(P, Y, P->nx, nvec, ldy, dout, dldout);
  return s2 != LRP_OK ? s2 : s;
}

// The truncated product of Algorithm 1 (LRP_LOWRANK_SOURCE), staged like
// the other calls.
static lrp_status hessian_lowrank_source(lrp_problem* P, int nvec, const double* X, int ldx, double* Y, int ldy,
                                         bool misfit, lrp_apply_stats* st) {
  lrp_status s = check_common(P, nvec, ldx, P->nx, ldy, P->nx, X, Y);
  if (s != LRP_OK) return s;
  if (nvec == 0) return LRP_OK;
  Staged sin, sout;
  const double* din;
  int dldin;
  double* dout;
  int dldout;
  if ((s = stage_in(P, X, P->nx, nvec, ldx, &din, &dldin, sin)) != LRP_OK) return s;
  if ((s = stage_out_alloc(P, Y, P->nx, nvec, ldy, &dout, &dldout, sout)) != LRP_OK) return s;
  s = lowrank_hessian_impl(P, nvec, din, dldin, dout, dldout, misfit, st);
  if (s != LRP_OK && s != LRP_ENOCONV) return s;
  lrp_status s2 = stage_out_copy(P, Y, P->nx, nvec, ldy, dout, dldout);
  return s2 != LRP_OK ? s2 : s;
}

// The product with both space-time solves by the alternating low-rank
// solver (LRP_ALS_SOLVES), staged like the other calls.
static lrp_status hessian_als(lrp_problem* P, int nvec, const double* X, int ldx, double* Y, int ldy, bool misfit,
                              lrp_apply_stats* st) {
  lrp_status s = check_common(P, nvec, ldx, P->nx, ldy, P->nx, X, Y);
  if (s != LRP_OK) return s;
  if (nvec == 0) return LRP_OK;
  Staged sin, sout;
  const double* din;
  int dldin;
  double* dout;
  int dldout;
  if ((s = stage_in(P, X, P->nx, nvec, ldx, &din, &dldin, sin)) != LRP_OK) return s;
  if ((s = stage_out_alloc(P, Y, P->nx, nvec, ldy, &dout, &dldout, sout)) != LRP_OK) return s;
  s = als_hessian_impl(P, nvec, din, dldin, dout, dldout, misfit, st);
  if (s != LRP_OK && s != LRP_ENOCONV) return s;
  lrp_status s2 = stage_out_copy(P, Y, P->nx, nvec, ldy, dout, dldout);
  return s2 != LRP_OK ? s2 : s;
}

}  // namespace lrp

extern "C" {

// Autotuner, on a pseudo-random block of nvec columns. Stage 1 (launch
// shape): every cluster size C, CTA size and columns per cluster times the
// prior solve and the first `steps` implicit-Euler steps of the forward sweep
// (the smooth start the Hessian apply sees) with the problem's multigrid
// settings. Stage 2 (solver): the two fastest shapes time the same with each
// smoothing-sweep count and (mixed path) inner tolerance. Stage 3: the five
// fastest of stage 2 time one whole Hessian apply each; the fastest is kept.
// Stage 4: the stage-1 screen for a single column at larger cluster sizes
// picks the size for narrow launches (team_ctas_narrow).
// Every candidate iterates to the same tolerances, so the choice changes the
// speed, not the result beyond rounding.
lrp_status lrp_autotune(lrp_problem* P, int nvec, int steps, double* best_ms) {
  if (!P || nvec < 1 || nvec > 4096) {
    set_error("lrp_autotune: invalid argument");
    return LRP_EINVAL;
  }
  cudaSetDevice(P->device);
  if (steps < 1) steps = 16;
  steps = std::min(steps, P->nt);
  double *X = nullptr, *Y = nullptr;
  cudaError_t e = lrp::dev_malloc(&X, (size_t)P->nx * nvec * sizeof(double));
  if (e == cudaSuccess) e = lrp::dev_malloc(&Y, (size_t)P->nx * nvec * sizeof(double));
  if (e == cudaSuccess) e = fill_random(P->stream, P->nx, nvec, X, P->nx, nullptr, 0xA070ull);
  if (e != cudaSuccess) {
    cudaFree(X);
    cudaFree(Y);
    return cuda_status(e, "autotune buffers");
  }
  struct Cand {
    int C, NT, BV, waves, nu, nuc;
    double inner, t1, t2;
    int levels;
  };
  const bool mixed = P->desc.precision == LRP_MIXED;
  const int save_C = P->team_ctas, save_BV = P->team_cols, save_NT = P->nthreads, save_W = P->allow_waves;
  const SolveCfg save_cfg = P->cfg;
  const int save_narrow = P->team_ctas_narrow;
  P->team_ctas_narrow = 0;  // stages 1-3 time nvec-column launches at the candidate's own size
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto apply_cand = [&](const Cand& c) {
    P->team_ctas = c.C;
    P->team_cols = c.BV;
    P->nthreads = c.NT;
    P->allow_waves = c.waves;
    P->cfg = save_cfg;
    P->cfg.nu = c.nu;
    P->cfg.nu_coarse = c.nuc;
    P->cfg.mg_levels = c.levels;
    if (mixed) P->cfg.inner_rtol = c.inner;
  };
  auto time_cols = [&](int ncols, unsigned stages, int t_end, double* out) {
    double best_t = 1e300;
    for (int rep = 0; rep < 2; ++rep) {
      cudaEventRecord(e0, P->stream);
      lrp_status st = run_sweep_ex(P, stages, ncols, X, P->nx, Y, P->nx, nullptr, 0, nullptr, 0, nullptr, 0, t_end,
                                   nullptr, 0);
      cudaEventRecord(e1, P->stream);
      cudaEventSynchronize(e1);
      if (st != LRP_OK) return;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      best_t = std::min(best_t, (double)ms);
    }
    *out = best_t;
  };
  auto time_it = [&](unsigned stages, int t_end, double* out) { time_cols(nvec, stages, t_end, out); };
  auto by_t1 = [](const Cand& a, const Cand& b) { return a.t1 < b.t1; };
  const unsigned screen = ST_LOAD_X | ST_PRIOR_IN | ST_FORWARD;
  // keep one screen near 20 ms: fewer steps for big problems
  {
    Cand c0{save_C,    save_NT, save_BV, save_W, save_cfg.nu, save_cfg.nu_coarse, save_cfg.inner_rtol,
            1e300,     1e300,   save_cfg.mg_levels};
    apply_cand(c0);
    double t = 1e300;
    time_it(screen, 1, &t);
    if (t < 1e300 && t > 0) steps = std::max(2, std::min(steps, (int)(20.0 / t)));
  }
  // stage 1: launch shape
  std::vector<Cand> shapes;
  for (int C : {1, 2, 3, 4, 5, 6, 7, 8, 12, 16})
    for (int NT : {512, 256})
      for (int BV : {1, 2})
        for (int waves : {0, 1}) {
          if (BV > 1 && nvec < 32) continue;  // one column per cluster wins for Lanczos-sized blocks
          if (C > 1 && (long long)P->nx / C < 256) continue;
          if (waves && C < 8) continue;  // more clusters than fit at once: only worth trying for big clusters
          shapes.push_back({C, NT, BV, waves, save_cfg.nu, save_cfg.nu_coarse, save_cfg.inner_rtol, 1e300, 1e300,
                            save_cfg.mg_levels});
        }
  for (Cand& c : shapes) {
    apply_cand(c);
    time_it(screen, steps, &c.t1);
  }
  std::sort(shapes.begin(), shapes.end(), by_t1);
  // stage 2: smoothing sweeps (finest level, coarse levels), inner
  // tolerance and depth of the time-step operator's hierarchy on the two
  // best shapes
  std::vector<int> depths{0};
  for (int lv = P->L - 1; lv >= std::max(3, P->L - 3); --lv) depths.push_back(lv);
  std::vector<Cand> cands;
  for (int i = 0; i < std::min<int>(2, (int)shapes.size()); ++i)
    for (int nu : {1, 2})
      for (int nuc : {1, 2})
        for (double inner : (mixed ? std::vector<double>{1e-4, 1e-5} : std::vector<double>{save_cfg.inner_rtol}))
          for (int levels : depths) {
            // only the band kernel smooths the coarse levels separately
            if (nuc != nu && P->last_kernel != 2) continue;
            Cand c = shapes[i];
            c.nu = nu;
            c.nuc = nuc;
            c.inner = inner;
            c.levels = levels;
            c.t1 = 1e300;
            apply_cand(c);
            time_it(screen, steps, &c.t1);
            cands.push_back(c);
          }
  std::sort(cands.begin(), cands.end(), by_t1);
  // stage 3: whole Hessian applies for the five best screens (the screen
  // ranks inner tolerances and smoothing counts only roughly), and for the
  // two best also their counterparts with the other inner tolerance: a
  // tighter inner tolerance screens faster (the screen's first steps start
  // from rough data) but can apply slower (measured on the 127^2 workload:
  // 1e-4 applied in 246 ms against 277 ms for 1e-5 with the same shape,
  // and was never among the five best screens)
  const unsigned hess = ST_LOAD_X | ST_PRIOR_IN | ST_FORWARD | ST_ADJOINT | ST_PRIOR_OUT | ST_STORE_Y;
  {
    const int top = std::min<int>(5, (int)cands.size());
    std::vector<Cand> sel(cands.begin(), cands.begin() + top);
    for (int i = 0; i < std::min(2, top) && mixed; ++i) {
      for (const Cand& o : cands) {
        const bool twin = o.C == sel[i].C && o.NT == sel[i].NT && o.BV == sel[i].BV && o.waves == sel[i].waves &&
                          o.nu == sel[i].nu && o.nuc == sel[i].nuc && o.levels == sel[i].levels &&
                          o.inner != sel[i].inner;
        if (!twin) continue;
        bool have = false;
        for (const Cand& q : sel)
          have = have || (q.C == o.C && q.NT == o.NT && q.BV == o.BV && q.waves == o.waves && q.nu == o.nu &&
                          q.nuc == o.nuc && q.levels == o.levels && q.inner == o.inner);
        if (!have) sel.push_back(o);
      }
    }
    cands = sel;
  }
  const int n2 = (int)cands.size();
  for (int i = 0; i < n2; ++i) {
    if (!(cands[i].t1 < 1e300)) continue;
    apply_cand(cands[i]);
    time_it(hess, -1, &cands[i].t2);
  }
  int bi = -1;
  for (int i = 0; i < n2; ++i)
    if (cands[i].t2 < 1e300 && (bi < 0 || cands[i].t2 < cands[bi].t2)) bi = i;
  if (bi < 0) {
    P->team_ctas = save_C;
    P->team_cols = save_BV;
    P->nthreads = save_NT;
    P->allow_waves = save_W;
    P->cfg = save_cfg;
    P->team_ctas_narrow = save_narrow;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(X);
    cudaFree(Y);
    set_error("lrp_autotune: no candidate ran");
    return LRP_ECUDA;
  }
  apply_cand(cands[bi]);
  if (best_ms) *best_ms = cands[bi].t2;
  // stage 4: cluster size for one-column launches (a single column leaves
  // most of the GPU idle; larger clusters shorten each step), kept only if
  // clearly faster than the winner's own size
  {
    double t_base = 1e300;
    time_cols(1, screen, steps, &t_base);
    int best_c = 0;
    double best_t = t_base;
    for (int Cn : {4, 8, 12, 16}) {
      if (Cn <= P->team_ctas || (long long)P->nx / Cn < 256) continue;
      P->team_ctas_narrow = Cn;
      double t = 1e300;
      time_cols(1, screen, steps, &t);
      if (t < 0.95 * best_t) {
        best_t = t;
        best_c = Cn;
      }
    }
    P->team_ctas_narrow = best_c;
    if (std::getenv("LRP_VERBOSE"))
      std::fprintf(stderr, "[lrp] autotune one column: %.2f ms at C=%d, %.2f ms at C=%d (kept %d)\n", t_base,
                   P->team_ctas, best_t, best_c ? best_c : P->team_ctas, best_c);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(X);
  cudaFree(Y);
  if (std::getenv("LRP_VERBOSE")) {
    for (int i = 0; i < std::min<int>(6, (int)shapes.size()); ++i)
      std::fprintf(stderr, "[lrp] autotune shape C=%d NT=%d BV=%d waves=%d: screen %.2f ms\n", shapes[i].C,
                   shapes[i].NT, shapes[i].BV, shapes[i].waves, shapes[i].t1);
    for (int i = 0; i < n2; ++i)
      std::fprintf(stderr,
                   "[lrp] autotune nvec=%d: C=%d NT=%d BV=%d waves=%d nu=%d/%d inner=%.0e levels=%d screen %.2f ms, "
                   "apply %.2f ms%s\n",
                   nvec, cands[i].C, cands[i].NT, cands[i].BV, cands[i].waves, cands[i].nu, cands[i].nuc, cands[i].inner,
                   cands[i].levels, cands[i].t1, cands[i].t2, i == bi ? " <- kept" : "");
  }
  return LRP_OK;
}

lrp_status lrp_hessian_apply(lrp_problem* P, int nvec, const double* X, int ldx, double* Y, int ldy,
                             unsigned flags, lrp_apply_stats* st) {
  if (!P) {
    set_error("NULL problem");
    return LRP_EINVAL;
  }
  const bool misfit = (flags & LRP_MISFIT_ONLY) != 0;
  if ((flags & LRP_KEEP_TRAJ_FACTORS) && (flags & LRP_LOWRANK_SOURCE)) {
    set_error("LRP_KEEP_TRAJ_FACTORS and LRP_LOWRANK_SOURCE are exclusive");
    return LRP_EINVAL;
  }
  if ((flags & LRP_ALS_SOLVES) && (flags & (LRP_KEEP_TRAJ_FACTORS | LRP_LOWRANK_SOURCE))) {
    set_error("LRP_ALS_SOLVES excludes LRP_KEEP_TRAJ_FACTORS and LRP_LOWRANK_SOURCE");
    return LRP_EINVAL;
  }
  if (flags & LRP_ALS_SOLVES) return hessian_als(P, nvec, X, ldx, Y, ldy, misfit, st);
  if (flags & LRP_LOWRANK_SOURCE) return hessian_lowrank_source(P, nvec, X, ldx, Y, ldy, misfit, st);
  if (flags & LRP_KEEP_TRAJ_FACTORS) return hessian_with_factors(P, nvec, X, ldx, Y, ldy, misfit, st);
  unsigned stages = ST_LOAD_X | ST_FORWARD | ST_ADJOINT | ST_STORE_Y;
  if (!misfit) stages |= ST_PRIOR_IN | ST_PRIOR_OUT;
  return sweep_call(P, stages, nvec, X, ldx, P->nx, Y, ldy, P->nx, false, false, st, misfit);
}

lrp_status lrp_forward_observe(lrp_problem* P, int nvec, const double* U, int ldu, double* D, int ldd,
                               lrp_apply_stats* st) {
  if (!P) {
    set_error("NULL problem");
    return LRP_EINVAL;
  }
  return sweep_call(P, ST_LOAD_X | ST_FORWARD | ST_STORE_D, nvec, U, ldu, P->nx, D, ldd, P->n_data, false,
                    true, st, false);
}

lrp_status lrp_adjoint(lrp_problem* P, int nvec, const double* D, int ldd, double* U, int ldu,
                       lrp_apply_stats* st) {
  if (!P) {
    set_error("NULL problem");
    return LRP_EINVAL;
  }
  return sweep_call(P, ST_LOAD_D | ST_ADJOINT | ST_STORE_Y, nvec, D, ldd, P->n_data, U, ldu, P->nx, true,
                    false, st, false);
}

lrp_status lrp_prior_half(lrp_problem* P, int nvec, const double* X, int ldx, double* Y, int ldy,
                          lrp_apply_stats* st) {
  if (!P) {
    set_error("NULL problem");
    return LRP_EINVAL;
  }
  return sweep_call(P, ST_LOAD_X | ST_PRIOR_IN | ST_STORE_Y, nvec, X, ldx, P->nx, Y, ldy, P->nx, false,
                    false, st, false);
}

}  // extern "C"
