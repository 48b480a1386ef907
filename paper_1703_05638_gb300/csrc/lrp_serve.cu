// Posterior-query server: continuous batching of queries over several
// problems ("models": a problem and its rank-k posterior factors) on one GPU.
//
// What a query computes is the low-rank posterior of Sec. 2 (the SMW form of
// the posterior covariance, its mean and samples), with the noise level of
// each request applied to the stored eigenvalues (they scale with 1/sigma^2).
//
// Scheduling. `slots` worker threads each own a CUDA stream. A free worker
// takes the model whose oldest pending request is the oldest overall, admits
// it (its factors on the device, a problem handle of its own for that model),
// and serves up to max_batch of that model's pending requests in one batch:
// one adjoint sweep over all the batch's data columns, one prior sweep over
// all its mean and sample columns, and the dense FP64 steps in between.
// Requests that arrive while batches are on the GPU wait for the next free
// worker, so batches of different models (and of the same model) overlap on
// the device. Every column of a sweep is an independent solve, so a
// request's result does not depend on the batch it was served in beyond the
// solver tolerance.
//
// Pointwise variance uses the prior diagonal at every node, computed once
// per model from the sine-transform closed form of (I + alpha L0)^-2 and
// kept with the factors.
//
// Memory. The server accounts every device byte it holds (factors, problem
// handles with their workspaces, batch scratch) against hbm_budget. A model
// whose factors are not resident is admitted by evicting the least recently
// used idle models (their factors stay in pinned host memory and come back
// by one copy); a batch waits while the memory it needs is held by batches
// in flight, and fails with LRP_EBUDGET only if the model cannot fit even
// with every other model evicted.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "lrp_dense.h"
#include "lrp_internal.h"

namespace lrp {

namespace {

// C[:, c] *= s[c]
__global__ void k_scale_cols(int n, int ncols, double* X, int ld, const double* s) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)n * ncols) return;
  const int c = (int)(e / n);
  X[(size_t)c * ld + (e - (size_t)c * n)] *= s[c];
}

// Per-column low-rank weights with lambda_j scaled by s[c] = sigma0^2/sigma_c^2:
// mode 0: d = l/(l+1) (posterior mean); mode 1: 1/sqrt(1+l) - 1 (samples).
__global__ void k_lowrank_scale(int k, int ncols, const double* lam, const double* s, int mode, double* C,
                                int ldc) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= k * ncols) return;
  const int i = e % k, c = e / k;
  const double l = lam[i] * s[c];
  C[(size_t)c * ldc + i] *= (mode == 0) ? l / (l + 1.0) : 1.0 / sqrt(1.0 + l) - 1.0;
}

// S[:, j] += M[:, owner[j]]
__global__ void k_add_owner_cols(int nx, int ncols, const double* M, int ldm, const int* owner, double* S,
                                 int lds) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)nx * ncols) return;
  const int j = (int)(e / nx);
  const size_t p = e - (size_t)j * nx;
  S[(size_t)j * lds + p] += M[(size_t)owner[j] * ldm + p];
}

// var[i] = prior_diag[node_i] - sum_j d_j(s_req(i)) G[node_i, j]^2
__global__ void k_variance_batch(int np, const int* nodes, const int* req, const double* s, const double* pdiag,
                                 int k, const double* lam, const double* G, int ldg, double* var) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const int node = nodes[i];
  const double sc = s[req[i]];
  double acc = 0.0;
  for (int j = 0; j < k; ++j) {
    const double l = lam[j] * sc;
    const double g = G[(size_t)j * ldg + node];
    acc += (l / (l + 1.0)) * g * g;
  }
  var[i] = pdiag[node] - acc;
}

unsigned nblk(size_t n) { return (unsigned)((n + 255) / 256); }

double now_ms(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

struct Request {
  unsigned long long ticket = 0;
  int model = 0;
  unsigned kind = 0;
  double sigma = 0.0;
  std::vector<double> y, xi;
  std::vector<int> pts;
  int ns = 0;
  // results
  std::vector<double> mean, var, samples;
  lrp_status status = LRP_OK;
  std::string err;
  lrp_request_stats st{};
  bool done = false;
};

struct Model;

// A worker's handle and scratch for one model.
struct SlotModel {
  lrp_problem* P = nullptr;
  size_t bytes = 0;  // device bytes accounted (problem + workspace + scratch)
  int B = 0, NS = 0, NP = 0, CH = 0, nx = 0, nd = 0, k = 0;
  double *y = nullptr, *zx = nullptr, *out = nullptr, *coef = nullptr, *part = nullptr, *scal = nullptr,
         *var = nullptr;
  size_t part_cap = 0;
  int *nodes = nullptr, *req = nullptr, *owner = nullptr;
  // pinned host staging
  double *h_y = nullptr, *h_xi = nullptr, *h_mean = nullptr, *h_samp = nullptr, *h_var = nullptr,
         *h_scal = nullptr;
  int *h_nodes = nullptr, *h_req = nullptr, *h_owner = nullptr;
  std::vector<void*> dev, host;

  ~SlotModel() {
    if (P) lrp_problem_destroy(P);
    for (void* p : dev) cudaFree(p);
    for (void* p : host) cudaFreeHost(p);
  }
  template <typename T>
  cudaError_t dalloc(T** p, size_t n) {
    cudaError_t e = lrp::dev_malloc((void**)p, std::max<size_t>(n, 1) * sizeof(T));
    if (e == cudaSuccess) {
      dev.push_back(*p);
      bytes += std::max<size_t>(n, 1) * sizeof(T);
    }
    return e;
  }
  template <typename T>
  cudaError_t halloc(T** p, size_t n) {
    cudaError_t e = cudaMallocHost((void**)p, std::max<size_t>(n, 1) * sizeof(T));
    if (e == cudaSuccess) host.push_back(*p);
    return e;
  }
};

struct Model {
  int id = 0;
  lrp_problem_desc desc{};
  std::vector<double> obs_xyz, kappa;
  int nx = 0, n_data = 0, k = 0;
  double sigma0 = 0.0;
  // pinned host copies of the factors (always kept)
  double *h_lam = nullptr, *h_V = nullptr, *h_G = nullptr, *h_diag = nullptr;
  // device copies while resident (d_diag: prior variance at every node)
  double *d_lam = nullptr, *d_V = nullptr, *d_G = nullptr, *d_diag = nullptr;
  size_t factor_bytes = 0;
  size_t handle_bytes = 0;  // measured bytes of one worker handle for this model
  // launch shape and multigrid settings every worker handle uses (autotuned)
  bool tuned = false;
  int team_ctas = 0, team_cols = 0, nthreads = 0, allow_waves = 0, team_ctas_narrow = 0;
  SolveCfg cfg{};
  int in_use = 0;
  double last_used = 0.0;
  std::deque<Request*> pending;
  long long admissions = 0, evictions = 0;
  bool resident() const { return d_V != nullptr; }
};

}  // namespace

}  // namespace lrp

struct lrp_server {
  lrp_server_config cfg{};
  int device = 0;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  std::vector<std::unique_ptr<lrp::Model>> models;
  std::map<unsigned long long, std::unique_ptr<lrp::Request>> reqs;
  unsigned long long next_ticket = 1;
  size_t used = 0;  // device bytes accounted
  long long batches = 0, served = 0;
  int in_flight = 0;
  // per worker: stream and per-model handles
  std::vector<cudaStream_t> streams;
  std::vector<std::map<int, std::unique_ptr<lrp::SlotModel>>> handles;
  std::vector<std::thread> workers;
};

namespace lrp {
namespace {

lrp_status slot_model_create(lrp_server* S, cudaStream_t s, Model& m, std::unique_ptr<SlotModel>& out) {
  auto h = std::make_unique<SlotModel>();
  lrp_problem_desc d = m.desc;
  d.obs_xyz = m.obs_xyz.data();
  d.kappa_faces = m.kappa.empty() ? nullptr : m.kappa.data();
  lrp_status st = lrp_setup_problem(&d, (void*)s, &h->P);
  if (st != LRP_OK) return st;
  lrp_problem* P = h->P;
  if (m.tuned) {
    P->team_ctas = m.team_ctas;
    P->team_cols = m.team_cols;
    P->nthreads = m.nthreads;
    P->allow_waves = m.allow_waves;
    P->team_ctas_narrow = m.team_ctas_narrow;
    P->cfg = m.cfg;
  }
  h->nx = m.nx;
  h->nd = m.n_data;
  h->k = m.k;
  h->B = S->cfg.max_batch;
  h->NS = S->cfg.max_samples;
  h->NP = S->cfg.max_points;
  const int cols = h->B * (1 + h->NS);
  h->CH = cols;
  h->part_cap = (size_t)std::max(m.k, 16) * 16 * 128;
#define SA(x)                                               \
  do {                                                      \
    cudaError_t e_ = (x);                                   \
    if (e_ != cudaSuccess) return cuda_status(e_, #x);      \
  } while (0)
  SA(h->dalloc(&h->y, (size_t)m.n_data * h->B));
  SA(h->dalloc(&h->zx, (size_t)m.nx * cols));
  SA(h->dalloc(&h->out, (size_t)m.nx * cols));
  SA(h->dalloc(&h->coef, (size_t)std::max(m.k, 1) * cols));
  SA(h->dalloc(&h->part, h->part_cap));
  SA(h->dalloc(&h->scal, (size_t)h->B + cols));
  SA(h->dalloc(&h->var, (size_t)h->B * h->NP));
  SA(h->dalloc(&h->nodes, (size_t)h->B * h->NP));
  SA(h->dalloc(&h->req, (size_t)h->B * h->NP));
  SA(h->dalloc(&h->owner, (size_t)cols));
  SA(h->halloc(&h->h_y, (size_t)m.n_data * h->B));
  SA(h->halloc(&h->h_xi, (size_t)m.nx * h->B * h->NS));
  SA(h->halloc(&h->h_mean, (size_t)m.nx * h->B));
  SA(h->halloc(&h->h_samp, (size_t)m.nx * h->B * h->NS));
  SA(h->halloc(&h->h_var, (size_t)h->B * h->NP));
  SA(h->halloc(&h->h_scal, (size_t)h->B + cols));
  SA(h->halloc(&h->h_nodes, (size_t)h->B * h->NP));
  SA(h->halloc(&h->h_req, (size_t)h->B * h->NP));
  SA(h->halloc(&h->h_owner, (size_t)cols));
  // grow the sweep workspace to the widest batch now: a zero block solves
  // at once, and later batches never reallocate it
  SA(cudaMemsetAsync(h->zx, 0, (size_t)m.nx * cols * sizeof(double), s));
  st = run_sweep(P, ST_LOAD_X | ST_PRIOR_IN | ST_STORE_Y, cols, h->zx, m.nx, h->out, m.nx, nullptr, 0, nullptr, 0,
                 nullptr, false);
  if (st != LRP_OK) return st;
  SA(cudaMemsetAsync(h->y, 0, (size_t)m.n_data * h->B * sizeof(double), s));
  st = run_sweep(P, ST_LOAD_D | ST_ADJOINT | ST_PRIOR_OUT | ST_STORE_Y, h->B, nullptr, 0, h->zx, m.nx, h->y,
                 m.n_data, nullptr, 0, nullptr, false);
  if (st != LRP_OK) return st;
  h->bytes += P->dev_bytes + P->ws_bytes;
#undef SA
  out = std::move(h);
  return LRP_OK;
}

void factors_free(lrp_server* S, Model& m) {
  if (m.d_V) cudaFree(m.d_V);
  if (m.d_G) cudaFree(m.d_G);
  if (m.d_lam) cudaFree(m.d_lam);
  if (m.d_diag) cudaFree(m.d_diag);
  m.d_V = m.d_G = m.d_lam = m.d_diag = nullptr;
  S->used -= m.factor_bytes;
}

// Under S->mu: evict least recently used idle models until `need` more bytes
// fit the budget. Returns false if that is impossible right now.
bool make_room(lrp_server* S, size_t need, const Model* keep) {
  while (S->used + need > S->cfg.hbm_budget) {
    Model* victim = nullptr;
    for (auto& mp : S->models) {
      Model* m = mp.get();
      if (m == keep || m->in_use > 0) continue;
      bool holds = m->d_V != nullptr;
      for (auto& hw : S->handles)
        if (hw.count(m->id)) holds = true;
      if (!holds) continue;
      if (!victim || m->last_used < victim->last_used) victim = m;
    }
    if (!victim) return false;
    if (victim->d_V) factors_free(S, *victim);
    for (auto& hw : S->handles) {
      auto it = hw.find(victim->id);
      if (it != hw.end()) {
        S->used -= it->second->bytes;
        hw.erase(it);
      }
    }
    victim->evictions++;
  }
  return true;
}

// The batch computation (no lock held). Fills each request's results.
// Pinned staging regions are each written once per batch before their copy
// is queued, and read back only after the final stream synchronisation.
// h_scal / scal layout: [0, B) data weights 1/sigma_r^2; [B, B + R + NSt)
// eigenvalue scalings sigma0^2/sigma^2 of the mean columns, then of the
// sample columns.
lrp_status serve_batch(lrp_server* S, int w, Model& m, SlotModel& h, std::vector<Request*>& batch) {
  cudaStream_t s = S->streams[w];
  const int R = (int)batch.size(), nx = m.nx, nd = m.n_data, k = m.k, B = h.B;
  lrp_problem* P = h.P;
#define SK(x)                                                 \
  do {                                                        \
    cudaError_t e_ = (x);                                     \
    if (e_ != cudaSuccess) return cuda_status(e_, #x);        \
  } while (0)
  // a sweep whose solves miss their tolerance still fills its output: the
  // batch completes and every request of it reports LRP_ENOCONV
  bool noconv = false;
#define SS(x)                                                 \
  do {                                                        \
    lrp_status s_ = (x);                                      \
    if (s_ != LRP_OK && s_ != LRP_ENOCONV) return s_;         \
    if (s_ == LRP_ENOCONV) noconv = true;                     \
  } while (0)
  // column layout of zx/out: [0, R) mean columns, [R, R+NSt) sample columns
  int NSt = 0;
  bool any_mean = false;
  double* hw = h.h_scal;      // data weights
  double* he = h.h_scal + B;  // eigenvalue scalings per column
  for (int r = 0; r < R; ++r) {
    const Request* q = batch[r];
    const bool wm = (q->kind & (LRP_Q_MEAN | LRP_Q_SAMPLES)) != 0;
    any_mean |= wm;
    if (wm)
      std::memcpy(h.h_y + (size_t)r * nd, q->y.data(), nd * sizeof(double));
    else
      std::memset(h.h_y + (size_t)r * nd, 0, nd * sizeof(double));
    const double sig = q->sigma > 0 ? q->sigma : m.sigma0;
    hw[r] = 1.0 / (sig * sig);
    he[r] = (m.sigma0 * m.sigma0) / (sig * sig);
  }
  for (int r = 0; r < R; ++r) {
    const Request* q = batch[r];
    if (!(q->kind & LRP_Q_SAMPLES)) continue;
    std::memcpy(h.h_xi + (size_t)NSt * nx, q->xi.data(), (size_t)q->ns * nx * sizeof(double));
    for (int j = 0; j < q->ns; ++j) {
      h.h_owner[NSt + j] = r;
      he[R + NSt + j] = he[r];
    }
    NSt += q->ns;
  }
  const int ncol = R + NSt;
  SK(cudaMemcpyAsync(h.scal, h.h_scal, (size_t)(B + ncol) * sizeof(double), cudaMemcpyHostToDevice, s));
  if (any_mean) {
    SK(cudaMemcpyAsync(h.y, h.h_y, (size_t)nd * R * sizeof(double), cudaMemcpyHostToDevice, s));
    note_launch();
    k_scale_cols<<<nblk((size_t)nd * R), 256, 0, s>>>(nd, R, h.y, nd, h.scal);
    SK(cudaGetLastError());
    // z = R^{-1} F^T Gamma_noise^{-1} y   (adjoint sweep + prior solve, all R columns)
    SS(run_sweep(P, ST_LOAD_D | ST_ADJOINT | ST_PRIOR_OUT | ST_STORE_Y, R, nullptr, 0, h.zx, nx, h.y, nd, nullptr,
                 0, nullptr, false));
    if (NSt > 0) {
      SK(cudaMemcpyAsync(h.zx + (size_t)R * nx, h.h_xi, (size_t)NSt * nx * sizeof(double), cudaMemcpyHostToDevice,
                         s));
      SK(cudaMemcpyAsync(h.owner, h.h_owner, NSt * sizeof(int), cudaMemcpyHostToDevice, s));
    }
    if (k > 0) {
      // z <- z - V diag(d) V^T z ; xi <- xi + V diag((1+l)^{-1/2} - 1) V^T xi
      SK(gemm_tn(s, nx, k, ncol, m.d_V, nx, h.zx, nx, h.coef, k, 1.0, 0.0, h.part, h.part_cap));
      note_launch();
      k_lowrank_scale<<<nblk((size_t)k * R), 256, 0, s>>>(k, R, m.d_lam, h.scal + B, 0, h.coef, k);
      if (NSt > 0) {
        note_launch();
        k_lowrank_scale<<<nblk((size_t)k * NSt), 256, 0, s>>>(k, NSt, m.d_lam, h.scal + B + R, 1,
                                                              h.coef + (size_t)R * k, k);
      }
      SK(cudaGetLastError());
      SK(gemm_nn(s, nx, k, R, -1.0, m.d_V, nx, h.coef, k, 1.0, h.zx, nx));
      if (NSt > 0)
        SK(gemm_nn(s, nx, k, NSt, 1.0, m.d_V, nx, h.coef + (size_t)R * k, k, 1.0, h.zx + (size_t)R * nx, nx));
    }
    // [mean | samples - mean] = R^{-1} [z | xi]   (one prior sweep over all columns)
    SS(run_sweep(P, ST_LOAD_X | ST_PRIOR_IN | ST_STORE_Y, ncol, h.zx, nx, h.out, nx, nullptr, 0, nullptr, 0,
                 nullptr, false));
    if (NSt > 0) {
      note_launch();
      k_add_owner_cols<<<nblk((size_t)nx * NSt), 256, 0, s>>>(nx, NSt, h.out, nx, h.owner, h.out + (size_t)R * nx,
                                                              nx);
      SK(cudaGetLastError());
    }
    SK(cudaMemcpyAsync(h.h_mean, h.out, (size_t)R * nx * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (NSt > 0)
      SK(cudaMemcpyAsync(h.h_samp, h.out + (size_t)R * nx, (size_t)NSt * nx * sizeof(double),
                         cudaMemcpyDeviceToHost, s));
  }
  // pointwise variance: prior diagonal minus the low-rank correction
  int NPt = 0;
  for (int r = 0; r < R; ++r) {
    const Request* q = batch[r];
    if (!(q->kind & LRP_Q_VARIANCE)) continue;
    for (int v : q->pts) {
      h.h_nodes[NPt] = v;
      h.h_req[NPt] = r;
      ++NPt;
    }
  }
  if (NPt > 0) {
    SK(cudaMemcpyAsync(h.nodes, h.h_nodes, NPt * sizeof(int), cudaMemcpyHostToDevice, s));
    SK(cudaMemcpyAsync(h.req, h.h_req, NPt * sizeof(int), cudaMemcpyHostToDevice, s));
    note_launch();
    k_variance_batch<<<nblk(NPt), 256, 0, s>>>(NPt, h.nodes, h.req, h.scal + B, m.d_diag, k, m.d_lam, m.d_G, nx,
                                                h.var);
    SK(cudaGetLastError());
    SK(cudaMemcpyAsync(h.h_var, h.var, NPt * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  SK(cudaStreamSynchronize(s));
  // hand the results to the requests
  int sc = 0, pc = 0;
  for (int r = 0; r < R; ++r) {
    Request* q = batch[r];
    if (q->kind & (LRP_Q_MEAN | LRP_Q_SAMPLES))
      q->mean.assign(h.h_mean + (size_t)r * nx, h.h_mean + (size_t)(r + 1) * nx);
    if (q->kind & LRP_Q_SAMPLES) {
      q->samples.assign(h.h_samp + (size_t)sc * nx, h.h_samp + (size_t)(sc + q->ns) * nx);
      sc += q->ns;
    }
    if (q->kind & LRP_Q_VARIANCE) {
      q->var.assign(h.h_var + pc, h.h_var + pc + q->pts.size());
      pc += (int)q->pts.size();
    }
  }
#undef SK
#undef SS
  if (noconv) {
    set_error("a solve of this batch missed its tolerance within pcg_maxit");
    return LRP_ENOCONV;
  }
  return LRP_OK;
}

void worker_main(lrp_server* S, int w) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (true) {
    Model* m = nullptr;
    bool blocked = false;
    // the model with the oldest pending request that can be admitted now
    std::vector<Model*> order;
    for (auto& mp : S->models)
      if (!mp->pending.empty()) order.push_back(mp.get());
    std::sort(order.begin(), order.end(),
              [](const Model* a, const Model* b) { return a->pending.front()->ticket < b->pending.front()->ticket; });
    for (Model* c : order) {
      size_t need = (c->resident() ? 0 : c->factor_bytes) +
                    (S->handles[w].count(c->id) ? 0 : std::max(c->handle_bytes, (size_t)1));
      if (make_room(S, need, c)) {
        m = c;
        break;
      }
      blocked = true;
      // nothing in flight can free memory for this model: it never fits
      if (S->in_flight == 0) {
        while (!c->pending.empty()) {
          Request* q = c->pending.front();
          c->pending.pop_front();
          q->status = LRP_EBUDGET;
          q->err = "the model does not fit the server's memory budget";
          q->done = true;
        }
        S->cv_done.notify_all();
      }
    }
    if (!m) {
      if (S->stop && order.empty()) break;
      (void)blocked;
      S->cv_work.wait(lk);
      continue;
    }
    // admit: factors to the device, this worker's handle
    std::vector<Request*> batch;
    while (!m->pending.empty() && (int)batch.size() < S->cfg.max_batch) {
      batch.push_back(m->pending.front());
      m->pending.pop_front();
    }
    m->in_use++;
    S->in_flight++;
    const double t_start = now_ms(S->t0);
    int admitted = 0;
    lrp_status st = LRP_OK;
    std::string err;
    if (!m->resident()) {
      admitted = 1;
      const size_t vk = (size_t)m->nx * m->k * sizeof(double);
      double *dV = nullptr, *dG = nullptr, *dl = nullptr, *dd = nullptr;
      cudaError_t e = lrp::dev_malloc(&dV, std::max<size_t>(vk, 8));
      if (e == cudaSuccess) e = lrp::dev_malloc(&dG, std::max<size_t>(vk, 8));
      if (e == cudaSuccess) e = lrp::dev_malloc(&dl, std::max(m->k, 1) * sizeof(double));
      if (e == cudaSuccess) e = lrp::dev_malloc(&dd, (size_t)m->nx * sizeof(double));
      if (e == cudaSuccess) e = cudaMemcpyAsync(dV, m->h_V, vk, cudaMemcpyHostToDevice, S->streams[w]);
      if (e == cudaSuccess) e = cudaMemcpyAsync(dG, m->h_G, vk, cudaMemcpyHostToDevice, S->streams[w]);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(dl, m->h_lam, m->k * sizeof(double), cudaMemcpyHostToDevice, S->streams[w]);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(dd, m->h_diag, (size_t)m->nx * sizeof(double), cudaMemcpyHostToDevice, S->streams[w]);
      if (e == cudaSuccess) e = cudaStreamSynchronize(S->streams[w]);
      if (e == cudaSuccess) {
        m->d_V = dV;
        m->d_G = dG;
        m->d_lam = dl;
        m->d_diag = dd;
        S->used += m->factor_bytes;
        m->admissions++;
      } else {
        st = cuda_status(e, "factor admission");
        err = lrp_last_error();
        cudaStreamSynchronize(S->streams[w]);
        if (dV) cudaFree(dV);
        if (dG) cudaFree(dG);
        if (dl) cudaFree(dl);
        if (dd) cudaFree(dd);
      }
    }
    SlotModel* h = nullptr;
    if (st == LRP_OK) {
      auto it = S->handles[w].find(m->id);
      if (it == S->handles[w].end()) {
        // reserve the measured footprint while the lock is released
        const size_t reserve = m->handle_bytes;
        S->used += reserve;
        std::unique_ptr<SlotModel> hp;
        lk.unlock();
        st = slot_model_create(S, S->streams[w], *m, hp);
        if (st != LRP_OK) err = lrp_last_error();
        lk.lock();
        S->used -= reserve;
        if (st == LRP_OK) {
          if (m->handle_bytes < hp->bytes) m->handle_bytes = hp->bytes;
          S->used += hp->bytes;
          h = hp.get();
          S->handles[w][m->id] = std::move(hp);
        }
      } else {
        h = it->second.get();
      }
    }
    lk.unlock();
    if (st == LRP_OK) {
      st = serve_batch(S, w, *m, *h, batch);
      if (st != LRP_OK) err = lrp_last_error();
    }
    lk.lock();
    const double t_done = now_ms(S->t0);
    for (Request* q : batch) {
      q->status = st;
      q->err = err;
      q->st.t_start_ms = t_start;
      q->st.t_done_ms = t_done;
      q->st.batch = (int)batch.size();
      q->st.slot = w;
      q->st.admitted = admitted;
      q->done = true;
    }
    m->in_use--;
    m->last_used = t_done;
    S->in_flight--;
    S->batches++;
    S->served += (long long)batch.size();
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
}

}  // namespace
}  // namespace lrp

using namespace lrp;

lrp_status lrp_server_create(const lrp_server_config* cfg, lrp_server** out) {
  if (!out) {
    set_error("lrp_server_create: NULL out");
    return LRP_EINVAL;
  }
  *out = nullptr;
  auto S = std::make_unique<lrp_server>();
  if (cfg) S->cfg = *cfg;
  if (S->cfg.hbm_budget == 0) S->cfg.hbm_budget = (size_t)16 << 30;
  if (S->cfg.slots <= 0) S->cfg.slots = 4;
  if (S->cfg.max_batch <= 0) S->cfg.max_batch = 16;
  if (S->cfg.max_samples <= 0) S->cfg.max_samples = 8;
  if (S->cfg.max_points <= 0) S->cfg.max_points = 1024;
  if (S->cfg.slots > 64 || S->cfg.max_batch > 256 || S->cfg.max_samples > 64) {
    set_error("lrp_server_create: slots <= 64, max_batch <= 256, max_samples <= 64");
    return LRP_EINVAL;
  }
  cudaError_t e = cudaGetDevice(&S->device);
  if (e != cudaSuccess) return cuda_status(e, "cudaGetDevice");
  S->t0 = std::chrono::steady_clock::now();
  S->streams.resize(S->cfg.slots);
  S->handles.resize(S->cfg.slots);
  for (auto& s : S->streams) {
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_status(e, "cudaStreamCreate");
  }
  lrp_server* raw = S.release();
  for (int w = 0; w < raw->cfg.slots; ++w) raw->workers.emplace_back(worker_main, raw, w);
  *out = raw;
  return LRP_OK;
}

lrp_status lrp_server_add_model(lrp_server* S, const lrp_problem_desc* d, int k, int block, double eig_tol,
                                const char* factors_path, int* model, lrp_lanczos_stats* st) {
  if (!S || !d || !model || k < 1) {
    set_error("lrp_server_add_model: invalid argument");
    return LRP_EINVAL;
  }
  cudaSetDevice(S->device);
  auto m = std::make_unique<Model>();
  m->desc = *d;
  const int dim = d->dim;
  if (d->obs_xyz && d->n_obs > 0) m->obs_xyz.assign(d->obs_xyz, d->obs_xyz + (size_t)d->n_obs * dim);
  lrp_problem* P = nullptr;
  cudaStream_t s = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_status(e, "cudaStreamCreate");
  lrp_status r = lrp_setup_problem(d, (void*)s, &P);
  if (r != LRP_OK) {
    cudaStreamDestroy(s);
    return r;
  }
  if (d->kappa_faces) {
    const size_t nf = (size_t)(d->n + 1) * (size_t)std::pow((double)d->n, dim - 1) * dim;
    m->kappa.assign(d->kappa_faces, d->kappa_faces + nf);
  }
  m->desc.obs_xyz = nullptr;
  m->desc.kappa_faces = nullptr;
  m->nx = P->nx;
  m->n_data = P->n_data;
  m->sigma0 = d->sigma;
  lrp_posterior* post = nullptr;
  bool loaded = false;
  if (factors_path) {
    FILE* f = std::fopen(factors_path, "rb");
    if (f) {
      std::fclose(f);
      r = lrp_posterior_load(P, factors_path, &post);
      if (r != LRP_OK) {
        lrp_problem_destroy(P);
        cudaStreamDestroy(s);
        return r;
      }
      loaded = true;
      if (st) std::memset(st, 0, sizeof(*st));
    }
  }
  if (!post) {
    r = lrp_lowrank_posterior(P, k, block, eig_tol, 0.0, 0, nullptr, &post, st);
    if (r != LRP_OK && r != LRP_ENOCONV) {
      lrp_problem_destroy(P);
      cudaStreamDestroy(s);
      return r;
    }
    if (factors_path && !loaded) lrp_posterior_save(post, factors_path);
  }
  m->k = post->k;
  const size_t vk = (size_t)m->nx * m->k * sizeof(double);
  m->factor_bytes = 2 * std::max<size_t>(vk, 8) + std::max(m->k, 1) * sizeof(double) + (size_t)m->nx * sizeof(double);
  e = cudaMallocHost(&m->h_V, std::max<size_t>(vk, 8));
  if (e == cudaSuccess) e = cudaMallocHost(&m->h_G, std::max<size_t>(vk, 8));
  if (e == cudaSuccess) e = cudaMallocHost(&m->h_lam, std::max<size_t>(m->k, 1) * sizeof(double));
  if (e == cudaSuccess && m->k) e = cudaMemcpy(m->h_V, post->V, vk, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && m->k) e = cudaMemcpy(m->h_G, post->G, vk, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && m->k) e = cudaMemcpy(m->h_lam, post->lambda, m->k * sizeof(double), cudaMemcpyDeviceToHost);
  // prior variance at every node (sine-transform closed form)
  if (e == cudaSuccess) e = cudaMallocHost(&m->h_diag, (size_t)m->nx * sizeof(double));
  if (e == cudaSuccess) {
    double* dwork = nullptr;
    const size_t nwork = (size_t)d->n * d->n + 3 * (size_t)m->nx;
    e = lrp::dev_malloc(&dwork, nwork * sizeof(double));
    if (e == cudaSuccess) e = prior_diag(s, *d, dwork + nwork - m->nx, dwork);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(m->h_diag, dwork + nwork - m->nx, (size_t)m->nx * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (dwork) cudaFree(dwork);
  }
  lrp_posterior_destroy(post);
  if (e == cudaSuccess && S->cfg.autotune) {
    r = lrp_autotune(P, S->cfg.max_batch, 0, nullptr);
    if (r == LRP_OK) {
      m->tuned = true;
      m->team_ctas = P->team_ctas;
      m->team_cols = P->team_cols;
      m->nthreads = P->nthreads;
      m->allow_waves = P->allow_waves;
      m->team_ctas_narrow = P->team_ctas_narrow;
      m->cfg = P->cfg;
    }
  }
  lrp_problem_destroy(P);
  if (e != cudaSuccess) {
    cudaStreamDestroy(s);
    return cuda_status(e, "factor copy");
  }
  // footprint of one worker handle for this model (problem, workspace grown
  // to the widest batch, scratch), measured once so admission can plan it
  {
    std::unique_ptr<SlotModel> probe;
    r = slot_model_create(S, s, *m, probe);
    if (r != LRP_OK) {
      cudaStreamDestroy(s);
      return r;
    }
    m->handle_bytes = probe->bytes;
  }
  cudaStreamDestroy(s);
  std::lock_guard<std::mutex> lk(S->mu);
  m->id = (int)S->models.size();
  *model = m->id;
  S->models.push_back(std::move(m));
  return LRP_OK;
}

lrp_status lrp_server_submit(lrp_server* S, int model, const lrp_query* q, unsigned long long* ticket) {
  if (!S || !q || !ticket) {
    set_error("lrp_server_submit: NULL argument");
    return LRP_EINVAL;
  }
  auto rq = std::make_unique<Request>();
  std::unique_lock<std::mutex> lk(S->mu);
  if (model < 0 || model >= (int)S->models.size()) {
    set_error("lrp_server_submit: unknown model");
    return LRP_EINVAL;
  }
  Model& m = *S->models[model];
  lk.unlock();
  rq->model = model;
  rq->kind = q->kind;
  rq->sigma = q->sigma;
  if (!(q->sigma >= 0) || !std::isfinite(q->sigma)) {
    set_error("lrp_server_submit: sigma must be finite and >= 0");
    return LRP_EINVAL;
  }
  if (q->kind & (LRP_Q_MEAN | LRP_Q_SAMPLES)) {
    if (!q->y_obs) {
      set_error("lrp_server_submit: y_obs required for MEAN/SAMPLES");
      return LRP_EINVAL;
    }
    rq->y.resize(m.n_data);
    if (is_device_ptr(q->y_obs)) {
      cudaError_t e = cudaMemcpy(rq->y.data(), q->y_obs, m.n_data * sizeof(double), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_status(e, "submit y_obs");
    } else {
      std::memcpy(rq->y.data(), q->y_obs, m.n_data * sizeof(double));
    }
  }
  if (q->kind & LRP_Q_VARIANCE) {
    if (q->n_points < 1 || q->n_points > S->cfg.max_points || !q->points) {
      set_error("lrp_server_submit: VARIANCE needs 1 <= n_points <= max_points and points");
      return LRP_EINVAL;
    }
    rq->pts.resize(q->n_points);
    if (is_device_ptr(q->points)) {
      cudaError_t e = cudaMemcpy(rq->pts.data(), q->points, q->n_points * sizeof(int), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_status(e, "submit points");
    } else {
      std::memcpy(rq->pts.data(), q->points, q->n_points * sizeof(int));
    }
    for (int v : rq->pts)
      if (v < 0 || v >= m.nx) {
        set_error("lrp_server_submit: node index out of range");
        return LRP_EINVAL;
      }
  }
  if (q->kind & LRP_Q_SAMPLES) {
    if (q->n_samples < 1 || q->n_samples > S->cfg.max_samples || !q->xi) {
      set_error("lrp_server_submit: SAMPLES needs 1 <= n_samples <= max_samples and xi");
      return LRP_EINVAL;
    }
    rq->ns = q->n_samples;
    rq->xi.resize((size_t)m.nx * rq->ns);
    if (is_device_ptr(q->xi)) {
      cudaError_t e = cudaMemcpy(rq->xi.data(), q->xi, rq->xi.size() * sizeof(double), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_status(e, "submit xi");
    } else {
      std::memcpy(rq->xi.data(), q->xi, rq->xi.size() * sizeof(double));
    }
  }
  lk.lock();
  rq->ticket = S->next_ticket++;
  rq->st.t_submit_ms = now_ms(S->t0);
  *ticket = rq->ticket;
  m.pending.push_back(rq.get());
  S->reqs[rq->ticket] = std::move(rq);
  S->cv_work.notify_one();
  return LRP_OK;
}

lrp_status lrp_server_wait(lrp_server* S, unsigned long long ticket, double timeout_s, lrp_query_result* res,
                           lrp_request_stats* st) {
  if (!S) {
    set_error("lrp_server_wait: NULL server");
    return LRP_EINVAL;
  }
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) {
    set_error("lrp_server_wait: unknown ticket");
    return LRP_EINVAL;
  }
  Request* q = it->second.get();
  auto pred = [&] { return q->done; };
  if (timeout_s > 0) {
    if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred)) {
      set_error("lrp_server_wait: timed out");
      return LRP_ETIMEOUT;
    }
  } else {
    S->cv_done.wait(lk, pred);
  }
  std::unique_ptr<Request> own = std::move(it->second);
  S->reqs.erase(it);
  lk.unlock();
  if (st) *st = own->st;
  if (own->status != LRP_OK && own->status != LRP_ENOCONV) {
    set_error(own->err);
    return own->status;
  }
  // LRP_ENOCONV: the results are filled (a solve of the request's batch
  // missed its tolerance); they are copied out and the status returned
  if (own->status == LRP_ENOCONV) set_error(own->err);
  if (res) {
    if (res->mean && !own->mean.empty()) std::memcpy(res->mean, own->mean.data(), own->mean.size() * sizeof(double));
    if (res->variance && !own->var.empty())
      std::memcpy(res->variance, own->var.data(), own->var.size() * sizeof(double));
    if (res->samples && !own->samples.empty())
      std::memcpy(res->samples, own->samples.data(), own->samples.size() * sizeof(double));
    res->ms = own->st.t_done_ms - own->st.t_submit_ms;
  }
  return own->status;
}

lrp_status lrp_server_info(lrp_server* S, lrp_server_stats* out) {
  if (!S || !out) {
    set_error("lrp_server_info: NULL argument");
    return LRP_EINVAL;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  std::memset(out, 0, sizeof(*out));
  out->device_bytes = S->used;
  out->batches = S->batches;
  out->served = S->served;
  for (auto& m : S->models) {
    out->models++;
    if (m->d_V) out->resident++;
    out->admissions += m->admissions;
    out->evictions += m->evictions;
    out->pending += (long long)m->pending.size();
  }
  return LRP_OK;
}

void lrp_server_destroy(lrp_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  for (auto& hw : S->handles) hw.clear();
  for (auto& m : S->models) {
    if (m->d_V) factors_free(S, *m);
    if (m->h_V) cudaFreeHost(m->h_V);
    if (m->h_G) cudaFreeHost(m->h_G);
    if (m->h_lam) cudaFreeHost(m->h_lam);
    if (m->h_diag) cudaFreeHost(m->h_diag);
  }
  for (auto& s : S->streams) cudaStreamDestroy(s);
  delete S;
}
