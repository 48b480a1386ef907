// Low-rank posterior: block Lanczos with full re-orthogonalisation on the
// prior-preconditioned misfit Hessian (Sec. 4 Algorithm 1 in its symmetric
// form), Ritz pairs, the Sherman-Morrison-Woodbury factors (Sec. 2), and the
// posterior queries (mean, pointwise variance, samples). Host code drives
// the iteration; every arithmetic step runs in the library's kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <string>
#include <new>
#include <vector>

#include "lrp_dense.h"
#include "lrp_internal.h"

namespace lrp {

lrp_status sweep_call(lrp_problem* P, unsigned stages, int nvec, const double* in, int ldin, int rows_in,
                      double* out, int ldout, int rows_out, bool in_is_d, bool out_is_d,
                      lrp_apply_stats* st, bool misfit_only);

template <typename T>
struct DArr {
  T* p = nullptr;
  size_t n = 0;
  DArr() = default;
  DArr(const DArr&) = delete;
  DArr& operator=(const DArr&) = delete;
  ~DArr() {
    if (p) cudaFree(p);
  }
  cudaError_t alloc(size_t count) {
    if (p) cudaFree(p);
    p = nullptr;
    n = count;
    return lrp::dev_malloc((void**)&p, std::max<size_t>(count, 1) * sizeof(T));
  }
  T* release() {
    T* r = p;
    p = nullptr;
    return r;
  }
};

#define CK(call)                                             \
  do {                                                       \
    cudaError_t _e = (call);                                 \
    if (_e != cudaSuccess) return cuda_status(_e, #call);    \
  } while (0)

static const unsigned HESS_STAGES = ST_LOAD_X | ST_PRIOR_IN | ST_FORWARD | ST_ADJOINT | ST_PRIOR_OUT | ST_STORE_Y;

// Scratch of one Lanczos run.
struct LanczosWS {
  DArr<double> part, R, C1, C2, ref, gs;
  size_t part_cap = 0;
};

// Orthonormalise the nb columns of Wn (nx x nb, ld nx) against Q[:, :nprev]
// (already orthonormal) by block CGS2 when nprev > 0 (coefficients added to
// Cacc), then within the block by rank-revealing CGS2: Wn = Qn R with R upper
// triangular in ws.R. A column numerically inside the span of the others
// becomes zero with a zero diagonal in R (block-Lanczos deflation).
static lrp_status block_orth(lrp_problem* P, int nx, int nb, double* Wn, const double* Q, int nprev,
                             LanczosWS& ws, double* Cacc, double drop_tol) {
  cudaStream_t s = P->stream;
  // norms before the projection: a column whose remainder is rounding noise
  // relative to them is dependent (deflated), even if the remainder is large
  // relative to itself
  if (nprev > 0) CK(col_norm2(s, nx, nb, Wn, nx, ws.ref.p));
  for (int pass = 0; pass < 2 && nprev > 0; ++pass) {
    CK(gemm_tn(s, nx, nprev, nb, Q, nx, Wn, nx, ws.C1.p, nprev, 1.0, 0.0, ws.part.p, ws.part_cap));
    CK(gemm_nn(s, nx, nprev, nb, -1.0, Q, nx, ws.C1.p, nprev, 1.0, Wn, nx));
    if (Cacc) CK(axpby(s, (size_t)nprev * nb, 1.0, ws.C1.p, 1.0, Cacc));
  }
  CK(block_gs(s, 1, nx, nb, Wn, 0, nx, ws.R.p, 0, drop_tol, nullptr, nprev > 0 ? ws.ref.p : nullptr, ws.gs.p));
  return LRP_OK;
}

// One block-Lanczos run on one problem, split so that its block steps can be
// enqueued without host synchronisation (and captured into a CUDA graph
// together with other problems' steps): enqueue_step() queues the Hessian
// apply of block j, the full re-orthogonalisation, the update of the block
// tridiagonal T and, once the basis has k columns, the eigensolve of T and
// the Ritz residuals with their copy to pinned host memory; after_step()
// reads them once the stream has been synchronised.
struct LanczosRun {
  lrp_problem* P = nullptr;
  int k = 0, nb = 0, nx = 0, mmax = 0;
  bool apply_noconv = false;  // a solve of some Hessian apply missed its tolerance
  double eig_tol = 1e-6, eig_threshold = 0.0;
  DArr<double> Q, W, T, Tw, Z, theta, work, resid;
  DArr<int> estat;
  LanczosWS ws;
  double* h_theta = nullptr;  // pinned
  double* h_res = nullptr;    // pinned
  Stats* h_stats = nullptr;   // pinned
  cudaEvent_t ev[2] = {nullptr, nullptr};
  SweepLaunch info;
  int j = 0, cols = 0, kk = 0, n_iter = 0, n_matvec = 0;
  bool check = false, last = false, converged = false, done = false;
  double max_res = 0.0, ms_apply = 0.0, drop_tol = 1e-13;
  std::chrono::steady_clock::time_point t0;

  ~LanczosRun() {
    if (h_theta) cudaFreeHost(h_theta);
    if (h_res) cudaFreeHost(h_res);
    if (h_stats) cudaFreeHost(h_stats);
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
  }

  lrp_status init(lrp_problem* P_, int k_, int block, double eig_tol_, double eig_threshold_, int max_basis,
                  const double* start) {
    P = P_;
    nx = P->nx;
    if (block < 1 || block > 64 || k_ < 1 || k_ > nx) {
      set_error("need 1 <= block <= 64 and 1 <= k <= nx");
      return LRP_EINVAL;
    }
    cudaSetDevice(P->device);
    t0 = std::chrono::steady_clock::now();
    k = k_;
    nb = block;
    eig_tol = eig_tol_ > 0 ? eig_tol_ : 1e-6;
    eig_threshold = eig_threshold_;
    mmax = max_basis > 0 ? max_basis : std::min(nx, 3 * k + 4 * nb);
    mmax = std::min(mmax, nx);
    mmax = std::min(mmax, 1024);
    mmax = std::max(nb, mmax / nb * nb);
    cudaStream_t s = P->stream;
    CK(Q.alloc((size_t)nx * (mmax + nb)));
    CK(W.alloc((size_t)nx * nb));
    CK(T.alloc((size_t)(mmax + nb) * (mmax + nb)));
    CK(Tw.alloc((size_t)mmax * mmax));
    CK(Z.alloc((size_t)mmax * mmax));
    CK(theta.alloc(mmax));
    CK(work.alloc(6 * (size_t)mmax + 8));
    CK(resid.alloc(mmax));
    CK(estat.alloc(1));
    ws.part_cap = (size_t)std::max(mmax + nb, 16) * 16 * 128;
    CK(ws.part.alloc(ws.part_cap));
    CK(ws.R.alloc(nb * nb));
    CK(ws.C1.alloc((size_t)(mmax + nb) * nb));
    CK(ws.C2.alloc((size_t)(mmax + nb) * nb));
    CK(ws.ref.alloc(nb));
    CK(ws.gs.alloc(block_gs_scratch_doubles()));
    CK(cudaMallocHost(&h_theta, mmax * sizeof(double)));
    CK(cudaMallocHost(&h_res, mmax * sizeof(double)));
    CK(cudaMallocHost(&h_stats, sizeof(Stats)));
    CK(cudaEventCreate(&ev[0]));
    CK(cudaEventCreate(&ev[1]));
    CK(cudaMemsetAsync(T.p, 0, T.n * sizeof(double), s));
    // start block
    if (start) {
      if (is_device_ptr(start)) {
        CK(copy_cols(s, nx, nb, start, nx, Q.p, nx));
      } else {
        CK(cudaMemcpyAsync(Q.p, start, (size_t)nx * nb * sizeof(double), cudaMemcpyHostToDevice, s));
      }
    } else {
      CK(fill_random(s, nx, nb, Q.p, nx, nullptr, 0x5EEDull));
    }
    // a direction whose remainder after re-orthogonalisation is below what the
    // apply resolves is noise of the inexact Hessian apply (2 nt + 2 solves,
    // each to the relative tolerance rtol), not a new Krylov direction: it is
    // deflated. Its effect on the Ritz values would be quadratic in it.
    drop_tol = std::max(1e-9, 1000.0 * P->cfg.rtol);
    lrp_status st = block_orth(P, nx, nb, Q.p, Q.p, 0, ws, nullptr, drop_tol);
    if (st != LRP_OK) return st;
    // grow the sweep workspace for nb columns now (an empty launch), so the
    // block steps never reallocate it
    st = sweep_enqueue(P, 0u, nb, nullptr, 0, nullptr, 0, nullptr, 0, nullptr, 0, 0, 0, nullptr, 0, nullptr, nullptr);
    if (st != LRP_OK) return st;
    CK(cudaStreamSynchronize(s));
    return LRP_OK;
  }

  // timing event: an event-record node when the stream is being captured
  static cudaError_t mark(cudaEvent_t e, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t err = cudaStreamIsCapturing(s, &cs);
    if (err != cudaSuccess) return err;
    return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal)
                                               : cudaEventRecord(e, s);
  }

  lrp_status enqueue_step() {
    cudaStream_t s = P->stream;
    const int c0 = j * nb;
    cols = c0 + nb;
    CK(mark(ev[0], s));
    lrp_status st = sweep_enqueue(P, HESS_STAGES, nb, Q.p + (size_t)c0 * nx, nx, W.p, nx, nullptr, 0, nullptr, 0, 0,
                                  -1, nullptr, 0, h_stats, &info);
    if (st != LRP_OK) return st;
    CK(mark(ev[1], s));
    // full re-orthogonalisation (CGS2 against the whole basis), the
    // coefficients of block j give A_j; block CGS2 of the remainder gives B_j
    CK(cudaMemsetAsync(ws.C2.p, 0, (size_t)cols * nb * sizeof(double), s));
    st = block_orth(P, nx, nb, W.p, Q.p, cols, ws, ws.C2.p, drop_tol);
    if (st != LRP_OK) return st;
    // T = Q^T Htilde Q as measured: the diagonal block A_j (symmetrised), the
    // coupling of block j to every earlier block (the re-orthogonalisation
    // coefficients; ~0 in exact arithmetic, kept so that T stays the exact
    // projection when the apply is inexact), and B_j below the diagonal
    CK(set_block(s, T.p, mmax + nb, c0, c0, nb, ws.C2.p + c0, cols, true, false));
    if (c0 > 0) CK(set_rect(s, T.p, mmax + nb, 0, c0, c0, nb, ws.C2.p, cols, true));
    CK(set_block(s, T.p, mmax + nb, cols, c0, nb, ws.R.p, nb, false, true));
    if (cols < mmax) CK(copy_cols(s, nx, nb, W.p, nx, Q.p + (size_t)cols * nx, nx));
    last = cols + nb > mmax;
    // with a threshold the number of pairs is not known in advance: every
    // block step (every 8 columns for narrower blocks) checks whether the
    // Ritz values have crossed it
    check = cols >= std::min(k, mmax) || last || (eig_threshold > 0 && cols % std::max(nb, 8) == 0);
    if (check) {
      kk = std::min(k, cols);
      // eigenpairs of T_j (copied: the solver destroys its input)
      CK(cudaMemcpy2DAsync(Tw.p, (size_t)cols * sizeof(double), T.p, (size_t)(mmax + nb) * sizeof(double),
                           (size_t)cols * sizeof(double), cols, cudaMemcpyDeviceToDevice, s));
      CK(eig_sym(s, cols, Tw.p, cols, Z.p, cols, theta.p, work.p, estat.p));
      CK(ritz_resid(s, kk, nb, ws.R.p, Z.p, cols, c0, resid.p));
      CK(cudaMemcpyAsync(h_theta, theta.p, kk * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(h_res, resid.p, kk * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    return LRP_OK;
  }

  // after the stream (or the graph holding the step) has completed
  lrp_status after_step() {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ev[0], ev[1]) == cudaSuccess) {
      ms_apply += ms;
      ledger_add(P, *h_stats, info, ms);
    } else {
      cudaGetLastError();  // no timing for this step; do not leave the error for later checks
    }
    n_matvec += nb;
    ++n_iter;
    lrp_status st = sweep_status(*h_stats, info, nullptr, 0.0);
    if (st != LRP_OK && st != LRP_ENOCONV) return st;
    if (st == LRP_ENOCONV) apply_noconv = true;
    if (check) {
      const double th0 = std::max(h_theta[0], 1e-300);
      if (std::getenv("LRP_VERBOSE")) {
        double mr = 0.0;
        for (int i = 0; i < kk; ++i) mr = std::max(mr, h_res[i] / th0);
        std::fprintf(stderr, "[lrp] lanczos j=%d cols=%d theta1=%.6e max_resid=%.3e apply_ms=%.1f total_ms=%.1f\n", j,
                     cols, h_theta[0], mr, ms_apply,
                     std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count());
      }
      bool ok = kk == k || cols >= nx;
      if (eig_threshold > 0) {
        // done once some Ritz value lies below the threshold (the kept ones
        // still have to meet the residual test below)
        for (int i = 0; i < kk; ++i)
          if (h_theta[i] < eig_threshold) ok = true;
      }
      max_res = 0.0;
      for (int i = 0; i < kk; ++i) {
        if (eig_threshold > 0 && h_theta[i] < eig_threshold) continue;
        max_res = std::max(max_res, h_res[i] / th0);
        if (h_res[i] > eig_tol * th0) ok = false;
      }
      if (ok) {
        converged = true;
        done = true;
      } else if (last) {
        done = true;
      }
    }
    ++j;
    return LRP_OK;
  }

  // Ritz vectors V_k = Q_m S_k, eigenvalues theta_k, G = R^-1 V_k
  lrp_status finish(lrp_posterior** out, lrp_lanczos_stats* stats) {
    cudaStream_t s = P->stream;
    int kout = kk;
    if (eig_threshold > 0) {
      kout = 0;
      for (int i = 0; i < kk; ++i)
        if (h_theta[i] >= eig_threshold) ++kout;
    }
    lrp_posterior* post = new lrp_posterior();
    post->prob = P;
    post->k = kout;
    post->nx = nx;
    post->sigma0 = P->desc.sigma;
    post->diag = nullptr;
    post->diag_cap = 0;
    post->lambda_host.assign(h_theta, h_theta + kout);
    DArr<double> V, G, lam;
    CK(V.alloc((size_t)nx * std::max(kout, 1)));
    CK(G.alloc((size_t)nx * std::max(kout, 1)));
    CK(lam.alloc(std::max(kout, 1)));
    if (kout > 0) {
      CK(gemm_nn(s, nx, cols, kout, 1.0, Q.p, nx, Z.p, cols, 0.0, V.p, nx));
      CK(cudaMemcpyAsync(lam.p, theta.p, kout * sizeof(double), cudaMemcpyDeviceToDevice, s));
      CK(cudaStreamSynchronize(s));
      lrp_apply_stats ast;
      lrp_status st = run_sweep(P, ST_LOAD_X | ST_PRIOR_IN | ST_STORE_Y, kout, V.p, nx, G.p, nx, nullptr, 0, nullptr,
                                0, &ast, false);
      if (st != LRP_OK && st != LRP_ENOCONV) {
        delete post;
        return st;
      }
    }
    CK(cudaStreamSynchronize(s));
    post->V = V.release();
    post->G = G.release();
    post->lambda = lam.release();
    *out = post;
    if (stats) {
      stats->n_iter = n_iter;
      stats->n_matvec = n_matvec;
      stats->k_converged = converged ? kout : 0;
      stats->max_ritz_resid = max_res;
      stats->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      stats->ms_apply = ms_apply;
    }
    if (!converged) {
      set_error("Lanczos reached its basis cap before all Ritz pairs converged");
      return LRP_ENOCONV;
    }
    if (apply_noconv) {
      set_error("a solve of a Hessian apply missed its tolerance within pcg_maxit");
      return LRP_ENOCONV;
    }
    return LRP_OK;
  }
};

}  // namespace lrp

using namespace lrp;

extern "C" {

lrp_status lrp_lowrank_posterior(lrp_problem* P, int k, int block, double eig_tol, double eig_threshold,
                                 int max_basis, const double* start, lrp_posterior** out,
                                 lrp_lanczos_stats* stats) {
  if (!P || !out) {
    set_error("NULL argument");
    return LRP_EINVAL;
  }
  *out = nullptr;
  lrp_status st = check_on_device(P->device, start, "lrp_lowrank_posterior start");
  if (st != LRP_OK) return st;
  LanczosRun run;
  st = run.init(P, k, block, eig_tol, eig_threshold, max_basis, start);
  if (st != LRP_OK) return st;
  while (!run.done) {
    st = run.enqueue_step();
    if (st != LRP_OK) return st;
    CK(cudaStreamSynchronize(P->stream));
    st = run.after_step();
    if (st != LRP_OK) return st;
  }
  return run.finish(out, stats);
}

lrp_status lrp_batch_lowrank_posterior(lrp_problem* const* probs, int count, int k, int block, double eig_tol,
                                       int use_graph, int max_steps, lrp_posterior** outs,
                                       lrp_lanczos_stats* stats, lrp_batch_stats* bst) {
  if (!probs || !outs || count < 1) {
    set_error("lrp_batch_lowrank_posterior: invalid argument");
    return LRP_EINVAL;
  }
  for (int i = 0; i < count; ++i) {
    outs[i] = nullptr;
    if (!probs[i]) {
      set_error("lrp_batch_lowrank_posterior: NULL problem");
      return LRP_EINVAL;
    }
    if (probs[i]->device != probs[0]->device) {
      set_error("lrp_batch_lowrank_posterior: problems on different devices");
      return LRP_EINVAL;
    }
    for (int j = 0; j < i; ++j)
      if (probs[j] == probs[i]) {
        set_error("lrp_batch_lowrank_posterior: a problem appears twice");
        return LRP_EINVAL;
      }
  }
  cudaSetDevice(probs[0]->device);
  // every problem works on a private stream for the duration of the call
  // (its own stream is drained first and restored at the end)
  struct StreamSwap {
    std::vector<lrp_problem*> probs;
    std::vector<cudaStream_t> saved, own;
    ~StreamSwap() {
      for (size_t i = 0; i < own.size(); ++i) {
        cudaStreamSynchronize(own[i]);
        probs[i]->stream = saved[i];
        cudaStreamDestroy(own[i]);
      }
    }
  } swap;
  for (int i = 0; i < count; ++i) {
    cudaStream_t ps = nullptr;
    CK(cudaStreamSynchronize(probs[i]->stream));
    CK(cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking));
    swap.probs.push_back(probs[i]);
    swap.saved.push_back(probs[i]->stream);
    swap.own.push_back(ps);
    probs[i]->stream = ps;
  }
  auto t0 = std::chrono::steady_clock::now();
  std::vector<std::unique_ptr<LanczosRun>> runs(count);
  for (int i = 0; i < count; ++i) {
    runs[i].reset(new LanczosRun());
    lrp_status st = runs[i]->init(probs[i], k, block, eig_tol, 0.0, 0, nullptr);
    if (st != LRP_OK) return st;
  }
  cudaStream_t origin = nullptr;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join(count, nullptr);
  CK(cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
  for (auto& e : join) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  auto cleanup = [&]() {
    for (auto& e : join)
      if (e) cudaEventDestroy(e);
    if (fork) cudaEventDestroy(fork);
    if (origin) cudaStreamDestroy(origin);
  };
  long long steps = 0, graph_nodes = 0;
  double ms_steps = 0.0;
  lrp_status result = LRP_OK;
  while (true) {
    std::vector<int> active;
    for (int i = 0; i < count; ++i)
      if (!runs[i]->done) active.push_back(i);
    if (active.empty() || (max_steps > 0 && steps >= max_steps)) break;
    auto ts = std::chrono::steady_clock::now();
    lrp_status st = LRP_OK;
    if (use_graph) {
      // one CUDA graph per step: every active problem's block step on its own
      // stream, forked from and joined back into the origin stream
      cudaGraph_t graph = nullptr;
      cudaGraphExec_t exec = nullptr;
      cudaError_t e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeRelaxed);
      if (e == cudaSuccess) e = cudaEventRecord(fork, origin);
      for (int i : active) {
        if (e != cudaSuccess) break;
        e = cudaStreamWaitEvent(probs[i]->stream, fork, 0);
        if (e != cudaSuccess) break;
        st = runs[i]->enqueue_step();
        if (st != LRP_OK) break;
        e = cudaEventRecord(join[i], probs[i]->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(origin, join[i], 0);
      }
      cudaError_t e2 = cudaStreamEndCapture(origin, &graph);
      if (st != LRP_OK || e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cleanup();
        if (st != LRP_OK) return st;
        return cuda_status(e != cudaSuccess ? e : e2, "batched step capture");
      }
      size_t nn = 0;
      cudaGraphGetNodes(graph, nullptr, &nn);
      graph_nodes += (long long)nn;
      e = cudaGraphInstantiate(&exec, graph, 0);
      if (e == cudaSuccess) e = cudaGraphLaunch(exec, origin);
      if (e == cudaSuccess) e = cudaStreamSynchronize(origin);
      if (exec) cudaGraphExecDestroy(exec);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        cleanup();
        return cuda_status(e, "batched step graph");
      }
    } else {
      for (int i : active) {
        st = runs[i]->enqueue_step();
        if (st != LRP_OK) {
          cleanup();
          return st;
        }
      }
      for (int i : active) {
        cudaError_t e = cudaStreamSynchronize(probs[i]->stream);
        if (e != cudaSuccess) {
          cleanup();
          return cuda_status(e, "batched step");
        }
      }
    }
    ms_steps += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - ts).count();
    ++steps;
    for (int i : active) {
      st = runs[i]->after_step();
      if (st != LRP_OK) {
        cleanup();
        return st;
      }
    }
  }
  cleanup();
  for (int i = 0; i < count; ++i) {
    if (!runs[i]->check) runs[i]->kk = 0;  // stopped before T had k columns: no Ritz pairs yet
    lrp_status st = runs[i]->finish(&outs[i], stats ? &stats[i] : nullptr);
    if (st != LRP_OK && st != LRP_ENOCONV) return st;
    if (st == LRP_ENOCONV) result = LRP_ENOCONV;
  }
  if (bst) {
    bst->steps = (int)steps;
    bst->graph_nodes = graph_nodes;
    bst->ms_steps = ms_steps;
    bst->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    long long mv = 0;
    for (auto& r : runs) mv += r->n_matvec;
    bst->n_matvec = mv;
  }
  return result;
}

void lrp_posterior_destroy(lrp_posterior* post) {
  if (!post) return;
  if (post->V) cudaFree(post->V);
  if (post->G) cudaFree(post->G);
  if (post->lambda) cudaFree(post->lambda);
  if (post->diag) cudaFree(post->diag);
  delete post;
}

lrp_status lrp_posterior_eigs(const lrp_posterior* post, int* r, double* lambda, double* V, int ldv) {
  if (!post || !r) {
    set_error("NULL argument");
    return LRP_EINVAL;
  }
  {
    lrp_status sd = check_on_device(post->prob->device, V, "lrp_posterior_eigs V");
    if (sd != LRP_OK) return sd;
  }
  *r = post->k;
  if (lambda) std::memcpy(lambda, post->lambda_host.data(), post->k * sizeof(double));
  if (V && post->k > 0) {
    if (ldv < post->nx) {
      set_error("ldv < nx");
      return LRP_EINVAL;
    }
    const cudaMemcpyKind kind = is_device_ptr(V) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaError_t e = cudaMemcpy2D(V, (size_t)ldv * sizeof(double), post->V, (size_t)post->nx * sizeof(double),
                                 (size_t)post->nx * sizeof(double), post->k, kind);
    if (e != cudaSuccess) return cuda_status(e, "posterior_eigs copy");
  }
  return LRP_OK;
}

lrp_status lrp_posterior_query(lrp_posterior* post, const lrp_query* q, lrp_query_result* r) {
  if (!post || !q || !r) {
    set_error("NULL argument");
    return LRP_EINVAL;
  }
  lrp_problem* P = post->prob;
  for (const void* a : {(const void*)q->y_obs, (const void*)q->points, (const void*)q->xi, (const void*)r->mean,
                        (const void*)r->variance, (const void*)r->samples}) {
    lrp_status sd = check_on_device(P->device, a, "lrp_posterior_query");
    if (sd != LRP_OK) return sd;
  }
  cudaSetDevice(P->device);
  cudaStream_t s = P->stream;
  auto t0 = std::chrono::steady_clock::now();
  const int nx = P->nx, k = post->k;
  const double sigma = q->sigma > 0 ? q->sigma : P->desc.sigma;
  const double lam_scale = (post->sigma0 * post->sigma0) / (sigma * sigma);
  const bool want_mean = (q->kind & (LRP_Q_MEAN | LRP_Q_SAMPLES)) != 0;
  lrp_status st;
  // a sweep whose solves miss their tolerance still fills its output: the
  // query completes and reports LRP_ENOCONV at the end
  lrp_status result = LRP_OK;
  DArr<double> mean, tmp, coef;
  if (want_mean) {
    if (!q->y_obs) {
      set_error("query: y_obs required for MEAN/SAMPLES");
      return LRP_EINVAL;
    }
    // g = F^T y / sigma^2 ; z = R^{-1} g (one adjoint sweep + prior solve)
    DArr<double> y;
    CK(y.alloc(P->n_data));
    const cudaMemcpyKind kind = is_device_ptr(q->y_obs) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(y.p, q->y_obs, P->n_data * sizeof(double), kind, s));
    CK(axpby(s, P->n_data, 1.0 / (sigma * sigma), y.p, 0.0, y.p));
    CK(mean.alloc(nx));
    CK(tmp.alloc(nx));
    st = run_sweep(P, ST_LOAD_D | ST_ADJOINT | ST_PRIOR_OUT | ST_STORE_Y, 1, nullptr, 0, tmp.p, nx, y.p,
                   P->n_data, nullptr, 0, nullptr, false);
    if (st != LRP_OK && st != LRP_ENOCONV) return st;
    if (st == LRP_ENOCONV) result = LRP_ENOCONV;
    // z <- z - V (d .* V^T z)
    if (k > 0) {
      CK(coef.alloc(k));
      DArr<double> part;
      CK(part.alloc((size_t)k * 16 * 128));
      CK(gemm_tn(s, nx, k, 1, post->V, nx, tmp.p, nx, coef.p, k, 1.0, 0.0, part.p, part.n));
      CK(diag_scale(s, k, 1, post->lambda, lam_scale, 0, coef.p, k));
      CK(gemm_nn(s, nx, k, 1, -1.0, post->V, nx, coef.p, k, 1.0, tmp.p, nx));
    }
    st = run_sweep(P, ST_LOAD_X | ST_PRIOR_IN | ST_STORE_Y, 1, tmp.p, nx, mean.p, nx, nullptr, 0, nullptr, 0,
                   nullptr, false);
    if (st != LRP_OK && st != LRP_ENOCONV) return st;
    if (st == LRP_ENOCONV) result = LRP_ENOCONV;
    if (r->mean) {
      const cudaMemcpyKind k2 = is_device_ptr(r->mean) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
      CK(cudaMemcpyAsync(r->mean, mean.p, nx * sizeof(double), k2, s));
    }
  }
  if (q->kind & LRP_Q_VARIANCE) {
    const int np = q->n_points;
    if (np < 1 || !q->points || !r->variance) {
      set_error("query: VARIANCE needs points and a variance buffer");
      return LRP_EINVAL;
    }
    std::vector<int> nodes(np);
    if (is_device_ptr(q->points)) {
      CK(cudaMemcpy(nodes.data(), q->points, np * sizeof(int), cudaMemcpyDeviceToHost));
    } else {
      std::memcpy(nodes.data(), q->points, np * sizeof(int));
    }
    for (int v : nodes)
      if (v < 0 || v >= nx) {
        set_error("query: node index out of range");
        return LRP_EINVAL;
      }
    DArr<int> dnodes;
    CK(dnodes.alloc(np));
    CK(cudaMemcpyAsync(dnodes.p, nodes.data(), np * sizeof(int), cudaMemcpyHostToDevice, s));
    if (!post->diag || post->diag_cap != nx) {
      // prior variance at every node: (R^-2)_ii with R = I + alpha L0 (constant
      // coefficients on the box) by the sine-transform closed form, or gamma
      // for the identity prior; computed once per posterior
      if (post->diag) cudaFree(post->diag);
      post->diag = nullptr;
      CK(lrp::dev_malloc(&post->diag, (size_t)nx * sizeof(double)));
      post->diag_cap = nx;
      DArr<double> dwork;
      CK(dwork.alloc((size_t)P->n * P->n + 2 * (size_t)nx));
      CK(prior_diag(s, P->desc, post->diag, dwork.p));
      CK(cudaStreamSynchronize(s));
    }
    // gather the diagonal at the query nodes
    DArr<double> pdiag;
    CK(pdiag.alloc(np));
    CK(gather(s, np, dnodes.p, post->diag, pdiag.p));
    DArr<double> var;
    CK(var.alloc(np));
    CK(variance(s, np, dnodes.p, pdiag.p, k, post->lambda, lam_scale, post->G, nx, var.p));
    const cudaMemcpyKind k2 = is_device_ptr(r->variance) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CK(cudaMemcpyAsync(r->variance, var.p, np * sizeof(double), k2, s));
  }
  if (q->kind & LRP_Q_SAMPLES) {
    const int ns = q->n_samples;
    if (ns < 1 || !q->xi || !r->samples) {
      set_error("query: SAMPLES needs xi and a samples buffer");
      return LRP_EINVAL;
    }
    DArr<double> Xi, Sm;
    CK(Xi.alloc((size_t)nx * ns));
    CK(Sm.alloc((size_t)nx * ns));
    const cudaMemcpyKind kind = is_device_ptr(q->xi) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(Xi.p, q->xi, (size_t)nx * ns * sizeof(double), kind, s));
    if (k > 0) {
      DArr<double> Cc, part;
      CK(Cc.alloc((size_t)k * ns));
      CK(part.alloc((size_t)k * 16 * 128));
      CK(gemm_tn(s, nx, k, ns, post->V, nx, Xi.p, nx, Cc.p, k, 1.0, 0.0, part.p, part.n));
      CK(diag_scale(s, k, ns, post->lambda, lam_scale, 1, Cc.p, k));
      CK(gemm_nn(s, nx, k, ns, 1.0, post->V, nx, Cc.p, k, 1.0, Xi.p, nx));
    }
    st = run_sweep(P, ST_LOAD_X | ST_PRIOR_IN | ST_STORE_Y, ns, Xi.p, nx, Sm.p, nx, nullptr, 0, nullptr, 0,
                   nullptr, false);
    if (st != LRP_OK && st != LRP_ENOCONV) return st;
    if (st == LRP_ENOCONV) result = LRP_ENOCONV;
    CK(add_vec_cols(s, nx, ns, mean.p, Sm.p, nx));
    const cudaMemcpyKind k2 = is_device_ptr(r->samples) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CK(cudaMemcpyAsync(r->samples, Sm.p, (size_t)nx * ns * sizeof(double), k2, s));
  }
  CK(cudaStreamSynchronize(s));
  r->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (result == LRP_ENOCONV) set_error("query: a solve missed its tolerance within pcg_maxit");
  return result;
}

lrp_status lrp_posterior_save(const lrp_posterior* post, const char* path) {
  if (!post || !path) {
    set_error("NULL argument");
    return LRP_EINVAL;
  }
  const size_t nx = post->nx, k = post->k;
  std::vector<double> V, G;
  try {
    V.resize(nx * k);
    G.resize(nx * k);
  } catch (const std::bad_alloc&) {
    set_error("posterior_save: host allocation failed");
    return LRP_ENOMEM;
  }
  if (k) {
    cudaError_t e = cudaMemcpy(V.data(), post->V, V.size() * sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(G.data(), post->G, G.size() * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e, "posterior_save");
  }
  // written to a temporary name and renamed at the end: a failed save leaves
  // no partial checkpoint under `path`
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) {
    set_error(std::string("cannot open ") + tmp);
    return LRP_EINVAL;
  }
  const char magic[8] = {'L', 'R', 'P', 'O', 'S', 'T', '0', '1'};
  const uint64_t hdr[3] = {post->prob->hash, (uint64_t)nx, (uint64_t)k};
  bool ok = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(hdr, sizeof(uint64_t), 3, f) == 3 &&
            std::fwrite(&post->sigma0, sizeof(double), 1, f) == 1 &&
            std::fwrite(post->lambda_host.data(), sizeof(double), k, f) == k &&
            std::fwrite(V.data(), sizeof(double), V.size(), f) == V.size() &&
            std::fwrite(G.data(), sizeof(double), G.size(), f) == G.size();
  ok = (std::fclose(f) == 0) && ok;
  if (!ok || std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    set_error("write failed");
    return LRP_EINVAL;
  }
  return LRP_OK;
}

lrp_status lrp_posterior_load(lrp_problem* P, const char* path, lrp_posterior** out) {
  if (!P || !path || !out) {
    set_error("NULL argument");
    return LRP_EINVAL;
  }
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) {
    set_error(std::string("cannot open ") + path);
    return LRP_EINVAL;
  }
  char magic[8];
  uint64_t hdr[3];
  double sigma0;
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "LRPOST01", 8) == 0 &&
            std::fread(hdr, sizeof(uint64_t), 3, f) == 3 && std::fread(&sigma0, sizeof(double), 1, f) == 1;
  if (!ok || hdr[0] != P->hash || hdr[1] != (uint64_t)P->nx) {
    std::fclose(f);
    set_error("checkpoint does not match this problem");
    return LRP_EINVAL;
  }
  // the rank can be at most nx: a larger value is a corrupt header, rejected
  // before anything is sized from it
  if (hdr[2] > hdr[1]) {
    std::fclose(f);
    set_error("corrupt checkpoint header (rank > nx)");
    return LRP_EINVAL;
  }
  const size_t nx = hdr[1], k = hdr[2];
  std::vector<double> lam, V, G;
  try {
    lam.resize(k);
    V.resize(nx * k);
    G.resize(nx * k);
  } catch (const std::bad_alloc&) {
    std::fclose(f);
    set_error("posterior_load: host allocation failed");
    return LRP_ENOMEM;
  }
  ok = std::fread(lam.data(), sizeof(double), k, f) == k && std::fread(V.data(), sizeof(double), V.size(), f) == V.size() &&
       std::fread(G.data(), sizeof(double), G.size(), f) == G.size();
  std::fclose(f);
  if (!ok) {
    set_error("truncated checkpoint");
    return LRP_EINVAL;
  }
  cudaSetDevice(P->device);
  lrp_posterior* post = new lrp_posterior();
  post->prob = P;
  post->k = (int)k;
  post->nx = (int)nx;
  post->sigma0 = sigma0;
  post->lambda_host = lam;
  post->diag = nullptr;
  post->diag_cap = 0;
  post->V = post->G = post->lambda = nullptr;
  cudaError_t e = lrp::dev_malloc(&post->V, std::max<size_t>(1, V.size()) * sizeof(double));
  if (e == cudaSuccess) e = lrp::dev_malloc(&post->G, std::max<size_t>(1, G.size()) * sizeof(double));
  if (e == cudaSuccess) e = lrp::dev_malloc(&post->lambda, std::max<size_t>(1, k) * sizeof(double));
  if (e == cudaSuccess && k) {
    e = cudaMemcpy(post->V, V.data(), V.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(post->G, G.data(), G.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(post->lambda, lam.data(), k * sizeof(double), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    lrp_posterior_destroy(post);
    return cuda_status(e, "posterior_load");
  }
  *out = post;
  return LRP_OK;
}

}  // extern "C"
