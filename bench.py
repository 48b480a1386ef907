"""Benchmark: low-rank posterior covariance hot path on the 2D heat workload
(127x127 interior, nx = 16129, nt = 500, 400 uniform sensors observed at
every step, sigma = 1e-3, prior (I + 0.05 L)^-2, rank k = 100).

One step = one pass of the whole hot path over one batch of synthetic input:
block Lanczos (block 32, full re-orthogonalisation) on the prior-
preconditioned misfit Hessian until the k = 100 Ritz pairs meet
||Htilde v - theta v|| <= 1e-6 theta_1 — every Hessian apply being a prior
solve, a 500-step forward and a 500-step adjoint implicit-Euler sweep of
multigrid-preconditioned CG solves — then the posterior factors, then one
posterior query (mean, pointwise variance at 1024 nodes, 8 samples).

value = Hessian matvecs (Htilde applied to one vector) per second over the
whole step; s_to_rank_k is the Lanczos part alone. Inputs are resident in
HBM; L2 is flushed (256 MB write) before every timed step. e2e repeats the
step through the C ABI with host buffers (copies inside the timed region).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank runs an independent replica of the workload on its
own GPU (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "Hessian matvecs/s (s to rank-k Gamma_post at 1e-6 rel. Ritz residual reported beside)"
UNIT = "matvec/s"


def workload_name(name: str, nt: int) -> str:
    """The workload description both arms report."""
    if name == "heat3d_63":
        return (f"heat3d_63: 3D heat eq 63^3 interior (nx=250047), kappa=exp(g) field, nt={nt}, 400 uniform "
                "sensors every 10th step, sigma=1e-3, prior (I-0.05 Lap)^-2")
    return (f"heat2d_127: 2D heat eq 127x127 interior (nx=16129), nt={nt}, 400 uniform sensors at every step, "
            "sigma=1e-3, prior (I-0.05 Lap)^-2")


# rank and Lanczos block per workload (the benchmark configurations)
WORKLOAD_DEFAULTS = {"heat2d_127": (100, 32), "heat3d_63": (200, 16)}
# The two sweep kernels, the sources their device code comes from, and the
# committed ncu summary (DRAM traffic per launch) for this workload.
KERNELS = {
    1: ("sweep_kernel", "persistent cluster-team MG-PCG forward/adjoint sweeps",
        ["lrp_sweep_kernel.cuh", "lrp_team.cuh"]),
    2: ("fast2d_kernel", "2D band kernel: shared-memory MG-PCG forward/adjoint sweeps",
        ["lrp_fast2d.cuh", "lrp_sweep_kernel.cuh", "lrp_team.cuh", "lrp_sweep_fast.cu"]),
}


def profile_summary(name: str, workload: str = "heat2d_127") -> str:
    return os.path.join(ROOT, "profiles", f"{name}_{workload}.json")


def kernel_hash(sources) -> str:
    """Hash of the kernel's sources with comments and whitespace removed (so
    that only a code change invalidates a committed profile)."""
    import re
    h = hashlib.sha256()
    for f in sources:
        with open(os.path.join(ROOT, "paper_1703_05638_gb300", "csrc", f)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        h.update("".join(text.split()).encode())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- the oracle on the host cores
# One process per host core, each holding its own oracle problem (sparse LU
# factors for 2D, CG solves for the 3D grid whose LU fill-in is prohibitive),
# applying Htilde to its own columns: a block of `cores` columns per round.
# On the 3D workload a full apply (2 nt + 2 solves) takes tens of minutes per
# column, so each worker times `sample_steps` forward and adjoint steps plus
# the two prior solves and scales the steps to nt (labelled as extrapolated).
_ORACLE = None


def _oracle_init(workload: str, nt: int):
    global _ORACLE
    from oracle.problem import Problem as OProblem
    spec = synth.workload(workload)
    if nt:
        spec.T, spec.nt = spec.T * nt / spec.nt, nt
    _ORACLE = OProblem(spec, solver="cg" if spec.dim == 3 else "lu")


def _oracle_apply_time(arg):
    """Seconds of one Htilde apply to one column on this worker (sampled and
    extrapolated when sample_steps > 0)."""
    seed, sample_steps = arg
    P = _ORACLE
    x = synth.normal_block(P.nx, 1, seed)[:, 0]
    if not sample_steps:
        t0 = time.perf_counter()
        P.hessian_apply(x)
        return time.perf_counter() - t0
    t0 = time.perf_counter()
    z = P.prior_half(x)
    t_prior = time.perf_counter() - t0
    t0 = time.perf_counter()
    y = z
    for _ in range(sample_steps):
        y = P.step(y)
    for _ in range(sample_steps):
        y = P.step_adjoint(y)
    t_steps = time.perf_counter() - t0
    return 2 * t_prior + t_steps * P.nt / sample_steps


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OraclePool:
    """The oracle on all host cores (spawned processes: safe after CUDA is
    initialised in the parent)."""

    def __init__(self, workload: str, nt: int = 0):
        import multiprocessing as mp
        self.cores = host_cores()
        self.workload = workload
        self.dim = 3 if workload.startswith("heat3d") else 2
        self.sample_steps = 10 if self.dim == 3 else 0
        env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in env:
            os.environ[k] = "1"  # one thread per worker process: cores = processes
        try:
            self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_oracle_init, initargs=(workload, nt))
        finally:
            for k, v in env.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        self.seed = 770

    def block(self):
        """Apply Htilde to one block of `cores` columns (one per process).
        Returns (wall seconds, columns), extrapolated on the 3D workload."""
        args = [(self.seed + j, self.sample_steps) for j in range(self.cores)]
        self.seed += self.cores
        t0 = time.perf_counter()
        per = self.pool.map(_oracle_apply_time, args, chunksize=1)
        wall = time.perf_counter() - t0
        if self.sample_steps:
            # the block's time is that of its slowest column at full length
            return max(per), len(per)
        return wall, len(per)

    def sample_text(self, blocks: int, seconds: float) -> str:
        if self.sample_steps:
            return (f"{blocks} blocks of {self.cores} single-column Htilde applies (one per core) on {self.workload}, "
                    f"each timed over 2 prior solves + {self.sample_steps} forward + {self.sample_steps} adjoint "
                    f"steps and extrapolated to nt steps; {seconds:.1f} s of sampled work")
        return (f"{blocks} blocks of {self.cores} single-column Htilde applies (one per core, sparse LU solves) "
                f"on {self.workload} in {seconds:.1f} s")

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline(workload: str, nt: int, n_matvec_to_k: int, seconds: float = 20.0):
    """The FP64 oracle on this host's cores: matvec/s over blocks of one
    column per core, and the time to rank k extrapolated from it with the
    GPU run's matvec count (the oracle's own eigensolver is not run)."""
    pool = OraclePool(workload, nt)
    try:
        pool.block()  # warm-up (factorisations, page-in)
        t_tot, cols, blocks = 0.0, 0, 0
        t0 = time.perf_counter()
        while True:
            dt, c = pool.block()
            t_tot += dt
            cols += c
            blocks += 1
            if time.perf_counter() - t0 >= seconds:
                break
        value = cols / t_tot
        out = {"value": value, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
               "sample": pool.sample_text(blocks, time.perf_counter() - t0)}
        if n_matvec_to_k:
            out["s_to_rank_k_extrapolated"] = n_matvec_to_k / value
            out["s_to_rank_k_basis"] = (f"{n_matvec_to_k} matvecs (the GPU Lanczos run's count) at the oracle's "
                                        "matvec rate; extrapolated, not run")
        return out
    finally:
        pool.close()


def serve_bench(lrp, count: int, rate_hz: float, budget_gib: float, slots: int, max_batch: int):
    """The serving workload: Poisson arrivals of posterior queries (mean,
    variance at 1024 nodes, 8 samples) over a 2D 127^2 and two 3D problems,
    through the library's server (continuous batching, factors resident,
    admission by memory budget). Factors (k=50) are computed before the
    stream starts and reported separately. Latency = result on the host
    minus the scheduled arrival."""
    import torch
    reqs = synth.serving_requests(count=count, rate_hz=rate_hz)
    sizes = sorted({r["size"] for r in reqs})
    srv = lrp.Server(hbm_budget=int(budget_gib * (1 << 30)), slots=slots, max_batch=max_batch, max_samples=8,
                     max_points=1024, autotune=True)
    t0 = time.perf_counter()
    mids, pools, setup = {}, {}, {}
    for size in sizes:
        spec = synth.serving_model_spec(size)
        ts = time.perf_counter()
        mid, lst = srv.add_model(spec, k=50, precision=lrp.LRP_MIXED, block=16, eig_tol=1e-6)
        mids[size] = mid
        setup[f"{size[0]}_{size[1]}"] = {"s": time.perf_counter() - ts, "n_matvec": lst["n_matvec"],
                                         "k_converged": lst["k_converged"]}
        # noise-free data of 8 seeded prior draws, and 2 blocks of sample draws
        G = lrp.lrp_setup_problem(spec, precision=lrp.LRP_MIXED)
        u = lrp.lrp_prior_half(G, torch.from_numpy(synth.normal_block(G.nx, 8, spec.seed + 11)).cuda())[0]
        d = lrp.lrp_forward_observe(G, u)[0].cpu().numpy()
        pools[size] = (d, [synth.normal_block(G.nx, 8, spec.seed + 13 + j) for j in range(2)], G.nx, G.n_data)
        G.close()
    warm_s = time.perf_counter() - t0
    kind = lrp.LRP_Q_MEAN | lrp.LRP_Q_VARIANCE | lrp.LRP_Q_SAMPLES
    # inputs of every request prepared before the clock starts
    prepared = []
    for r in reqs:
        d, xis, nx, nd = pools[r["size"]]
        g = synth.rng(r["seed"])
        y = d[:, r["index"] % d.shape[1]] + r["sigma"] * g.standard_normal(nd)
        prepared.append((mids[r["size"]], y, r["sigma"], synth.query_nodes(nx, r["n_query"], r["seed"]),
                         xis[r["index"] % 2]))
    tickets = [None] * len(reqs)
    lag = [0.0] * len(reqs)
    start = time.perf_counter() + 0.05

    def submitter():
        for i, r in enumerate(reqs):
            due = start + r["arrival_s"]
            while True:
                now = time.perf_counter()
                if now >= due:
                    break
                time.sleep(min(due - now, 0.002))
            mid, y, sig, pts, xi = prepared[i]
            tickets[i] = srv.submit(mid, kind, y_obs=y, sigma=sig, points=pts, xi=xi)
            lag[i] = (time.perf_counter() - due) * 1e3

    th = threading.Thread(target=submitter)
    th.start()
    lat, batch = [], []
    for i in range(len(reqs)):
        while tickets[i] is None:
            time.sleep(0.0005)
        out = srv.wait(tickets[i], timeout=600.0)
        lat.append(out["latency_ms"] + lag[i])
        batch.append(out["stats"]["batch"])
    th.join()
    t_end = time.perf_counter()
    info = srv.info()
    srv.close()
    lat_a = np.asarray(lat)
    by_size = {}
    for size in sizes:
        sel = [j for j, r in enumerate(reqs) if r["size"] == size]
        by_size[f"{size[0]}_{size[1]}"] = {"n": len(sel), "p50_ms": float(np.percentile(lat_a[sel], 50)),
                                           "p99_ms": float(np.percentile(lat_a[sel], 99))}
    return {"p50_ms": float(np.percentile(lat_a, 50)), "p99_ms": float(np.percentile(lat_a, 99)),
            "requests": len(reqs), "rate_hz": rate_hz,
            "throughput_rps": len(reqs) / (t_end - start), "mean_batch": float(np.mean(batch)),
            "batches": info["batches"], "admissions": info["admissions"], "evictions": info["evictions"],
            "device_gib_held": info["device_bytes"] / (1 << 30), "budget_gib": budget_gib, "slots": slots,
            "max_batch": max_batch, "by_size": by_size, "factor_setup": setup, "warmup_s": warm_s,
            "query": "mean + variance@1024 + 8 samples, sigma log-uniform [1e-4, 1e-2], k=50"}


def batched_bench(lrp, count: int, block: int, steps: int, use_graph: bool = True):
    """The batched workload: `count` independent 2D instances (grids 63^2,
    127^2 or 255^2, nt 200-2000, 50-1000 sensors, sigma log-uniform) each on
    its own stream, block Lanczos for k=50 advanced together, one CUDA graph
    per block step. A bounded sample: `steps` block steps of every instance
    (the whole run to k=50 takes minutes). One autotune per grid size."""
    import torch
    insts = synth.batched_instances(count=count)
    probs = [lrp.lrp_setup_problem(sp, precision=lrp.LRP_MIXED) for sp in insts]
    t0 = time.perf_counter()
    tuned = {}
    for sp, G in zip(insts, probs):
        if sp.n not in tuned:
            lrp.lrp_autotune(G, block)
            tuned[sp.n] = lrp.lrp_problem_tuning(G)
        else:
            lrp.lrp_set_tuning(G, tuned[sp.n])
    tune_s = time.perf_counter() - t0
    res, _ = lrp.lrp_batch_lowrank_posterior(probs, k=50, block=block, eig_tol=1e-6, use_graph=use_graph,
                                             max_steps=1)
    for post, _ in res:
        post.close()
    torch.cuda.synchronize()
    res, bst = lrp.lrp_batch_lowrank_posterior(probs, k=50, block=block, eig_tol=1e-6, use_graph=use_graph,
                                               max_steps=steps)
    for post, _ in res:
        post.close()
    sizes = {}
    for sp in insts:
        sizes[str(sp.n)] = sizes.get(str(sp.n), 0) + 1
    out = {"instances": count, "block": block, "steps": bst["steps"], "n_matvec": bst["n_matvec"],
           "graph_nodes": bst["graph_nodes"], "use_graph": use_graph, "s_steps": bst["ms_steps"] / 1e3,
           "s_call": bst["ms"] / 1e3, "matvec_per_s": bst["n_matvec"] / (bst["ms_steps"] / 1e3),
           "grids": sizes, "nt_range": [min(sp.nt for sp in insts), max(sp.nt for sp in insts)],
           "tuning_by_grid": tuned, "autotune_s": tune_s}
    for G in probs:
        G.close()
    return out


# Arnoldi iteration counts printed by the paper for its Q1 finite-element
# version of this experiment (MATLAB, one CPU core): context, not a target
PAPER_ARNOLDI_ITERATIONS = {(1e6, 1.0): 72, (1e6, 0.1): 163, (1e8, 1.0): 347, (1e8, 0.1): 470}
# the same for its convection-diffusion experiment, by (nu, epsilon)
PAPER_CD_ARNOLDI_ITERATIONS = {(1e-2, 10.0): 17, (1e-2, 1.0): 121, (1e-3, 10.0): 52, (1e-3, 1.0): 131}


def arnoldi_leg(lrp, G, eps, lam_lanczos):
    """Algorithm 1 as the paper runs it: Arnoldi with the truncated product
    (state and adjoint trajectories truncated to 1e-8, the paper's threshold
    for the low-rank approximation), stopped by the threshold rule at Ritz
    residual 1e-6 theta_1. Steps, Ritz values kept, the largest trajectory
    ranks, how far H is from symmetric, and the largest difference of the
    kept Ritz values from the Lanczos eigenvalues (relative to lambda_1)."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = lrp.lrp_arnoldi(G, min(1000, G.nx), eig_tol=1e-6, eig_threshold=eps, flags=lrp.LRP_LOWRANK_SOURCE)
    dt = time.perf_counter() - t0
    st = res["stats"]
    th = res["theta"]
    kept = np.sort(th.real[(th.real >= eps) & (th.imag == 0)])[::-1]
    n = min(len(kept), len(lam_lanczos))
    diff = float(np.max(np.abs(kept[:n] - lam_lanczos[:n])) / lam_lanczos[0]) if n else None
    return {"arnoldi_steps": st["n_steps"], "kept": int(len(kept)), "s": dt, "status": st["status"],
            "max_rank_state": st["time_rank_max"], "max_rank_adjoint": st["adj_rank_max"],
            "hess_asym": st["hess_asym"], "n_complex": st["n_complex"], "max_imag_rel": st["max_imag"],
            "max_rel_diff_vs_lanczos": diff, "ms_apply": st["ms_apply"]}


def spacetime_leg(lrp, spec, precision, eps, max_steps=300):
    """Algorithm 1 on low-rank space-time vectors (the parameter a source
    u(x, t), Sec. 4): steps to resolve the eigenvalues above epsilon, the
    largest ranks of the Krylov vectors and of the products, time."""
    import torch
    G = lrp.lrp_setup_problem(spec, precision=precision)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = lrp.lrp_st_arnoldi(G, max_steps, eig_tol=1e-6, eig_threshold=eps)
    dt = time.perf_counter() - t0
    st = res["stats"]
    th = res["theta"]
    G.close()
    return {"epsilon": eps, "steps": st["n_steps"], "kept": int(np.sum((th.real >= eps) & (th.imag == 0))),
            "lambda_1": float(th.real[0]) if len(th) else None, "max_rank_krylov_vector": st["time_rank_max"],
            "max_rank_product": st["adj_rank_max"], "hess_asym": st["hess_asym"], "n_complex": st["n_complex"],
            "s": dt, "ms_apply": st["ms_apply"], "status": st["status"], "nx_nt": G.nx * spec.nt}


def als_bench(lrp, spec, precision, ranks=(12, 16, 20), sweeps=3, ncols=4, prec=((0.0, 2), (0.0, 1), (1e-4, 0))):
    """The Hessian product with both space-time systems solved by the
    alternating low-rank solver (Sec. 6.1, Eq. (amen_1)-(pre_1);
    LRP_ALS_SOLVES) beside the time-stepping product on the same columns:
    wall time per column (one column at a time, the ALS form's unit; and the
    time-stepping block of ncols columns in one launch), the relative
    difference to the time-stepping result, and the solver's own counts for
    one forward solve of the initial condition (GMRES iterations, time in
    the space and the time steps). prec: (als_prec_rtol, als_prec_its)
    pairs of the preconditioner (the first for every rank, the others at the
    second rank)."""
    import torch
    G = lrp.lrp_setup_problem(spec, precision=precision)
    X = synth.normal_block(G.nx, ncols, 1000 + 17)
    Xd = torch.from_numpy(X).cuda()
    ref, _ = lrp.lrp_hessian_apply(G, Xd)          # warm-up and reference
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ref, st_ts = lrp.lrp_hessian_apply(G, Xd)
    torch.cuda.synchronize()
    ms_block = (time.perf_counter() - t0) * 1e3
    t0 = time.perf_counter()
    one, _ = lrp.lrp_hessian_apply(G, Xd[:, :1])
    torch.cuda.synchronize()
    ms_one = (time.perf_counter() - t0) * 1e3
    refn = ref.cpu().numpy()
    out = {"workload": f"{spec.dim}D n={spec.n} nt={spec.nt}", "precision": int(precision),
           "time_stepping": {"ms_per_column_alone": ms_one, "ms_block": ms_block, "block": ncols,
                             "solves_per_column": st_ts["n_solves"]},
           "als": []}
    for r, (prt, pits) in [(r, prec[0]) for r in ranks] + [(ranks[min(1, len(ranks) - 1)], p) for p in prec[1:]]:
        G.close()
        G = lrp.lrp_setup_problem(spec, precision=precision, als_rank=r, als_sweeps=sweeps, als_prec_rtol=prt,
                                  als_prec_its=pits)
        lrp.lrp_hessian_apply(G, Xd[:, :1], flags=lrp.LRP_ALS_SOLVES)   # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Y, st = lrp.lrp_hessian_apply(G, Xd, flags=lrp.LRP_ALS_SOLVES)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3
        Yn = Y.cpu().numpy()
        rel = float(np.max(np.linalg.norm(Yn - refn, axis=0) / np.linalg.norm(refn, axis=0)))
        e1 = np.zeros((G.nt, 1))
        e1[0, 0] = 1.0
        W, V, res, ast = lrp.lrp_als_solve(G, X[:, :1], e1, np.eye(G.nt)[:, :r], sweeps)
        out["als"].append({"rank": r, "sweeps": sweeps, "prec_rtol": prt, "prec_its": pits, "ms_per_column": ms / ncols,
                           "status": st["status"],
                           "max_rel_diff_vs_time_stepping": rel, "residual_forward": st["time_trunc_err"],
                           "residual_adjoint": st["adj_trunc_err"],
                           "precond_solves_per_column": st["n_solves"],
                           "forward_solve": {"gmres_iters": ast["gmres_iters"], "ms": ast["ms"],
                                             "ms_space": ast["ms_space"], "ms_time": ast["ms_time"],
                                             "residuals": [float(v) for v in res]}})
    G.close()
    return out


def als_arnoldi_leg(lrp, spec, precision, eps, lam_lanczos, rank=16, sweeps=3):
    """Algorithm 1 in the paper's arrangement: Arnoldi outside, the forward
    and adjoint space-time systems of every product solved by the
    alternating low-rank solver (LRP_ALS_SOLVES) inside; steps, Ritz values
    kept and their largest difference from the Lanczos eigenvalues."""
    import torch
    G = lrp.lrp_setup_problem(spec, precision=precision, als_rank=rank, als_sweeps=sweeps)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = lrp.lrp_arnoldi(G, min(1000, G.nx), eig_tol=1e-6, eig_threshold=eps, flags=lrp.LRP_ALS_SOLVES)
    dt = time.perf_counter() - t0
    G.close()
    st = res["stats"]
    th = res["theta"]
    kept = np.sort(th.real[(th.real >= eps) & (th.imag == 0)])[::-1]
    n = min(len(kept), len(lam_lanczos))
    diff = float(np.max(np.abs(kept[:n] - lam_lanczos[:n])) / lam_lanczos[0]) if n else None
    return {"rank": rank, "sweeps": sweeps, "arnoldi_steps": st["n_steps"], "kept": int(len(kept)), "s": dt,
            "status": st["status"], "hess_asym": st["hess_asym"], "n_complex": st["n_complex"],
            "max_rel_diff_vs_lanczos": diff, "ms_apply": st["ms_apply"]}


def paper_bench(lrp, precision):
    """The heat experiment of the paper's numerical section on finite
    differences (63^2 nodes, nt = 30, 9 sensor patches, Gamma_prior = 10 I)
    for beta_noise / beta_prior in {1e4, 1e6, 1e8} and thresholds epsilon in
    {1, 0.1}: single-vector Lanczos until every eigenvalue above epsilon is
    resolved (Ritz residual 1e-6 theta_1); Lanczos steps, eigenvalues kept,
    time, and the posterior variance over the grid (min / mean / max); then
    Algorithm 1 itself (Arnoldi on the truncated product, ``arnoldi_leg``).
    The same for the convection-diffusion experiment (31^2 nodes, nt = 90)."""
    import torch
    out = []
    for ratio in (1e4, 1e6, 1e8):
        spec = synth.paper_heat_spec(ratio)
        G = lrp.lrp_setup_problem(spec, precision=precision)
        nodes = np.arange(G.nx, dtype=np.int32)
        for eps in (1.0, 0.1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            post, st = lrp.lrp_lowrank_posterior(G, k=1000, block=1, eig_tol=1e-6, eig_threshold=eps)
            dt = time.perf_counter() - t0
            lam = post.eigs()
            var = lrp.lrp_posterior_query(post, lrp.LRP_Q_VARIANCE, points=nodes)["variance"]
            out.append({"ratio": ratio, "epsilon": eps, "lanczos_steps": st["n_matvec"], "kept": int(len(lam)),
                        "lambda_1": float(lam[0]) if len(lam) else None, "s": dt, "status": st["status"],
                        "variance_min_mean_max": [float(var.min()), float(var.mean()), float(var.max())],
                        "paper_arnoldi_iterations": PAPER_ARNOLDI_ITERATIONS.get((ratio, eps)),
                        "arnoldi": arnoldi_leg(lrp, G, eps, lam)})
            if ratio == 1e6:
                out[-1]["arnoldi_als"] = als_arnoldi_leg(lrp, spec, precision, eps, lam)
            post.close()
        G.close()
    # the space-time parameter on the heat experiment's setting
    out.append({"spacetime": spacetime_leg(lrp, synth.paper_heat_spec(1e4), precision, 1.0)})
    # the convection-diffusion experiment (FP64 path: the nonsymmetric steps
    # are solved by BiCGStab)
    for nu in (1e-2, 1e-3):
        spec = synth.paper_convdiff_spec(nu)
        G = lrp.lrp_setup_problem(spec, precision=lrp.LRP_FP64)
        nodes = np.arange(G.nx, dtype=np.int32)
        for eps in (10.0, 1.0):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            post, st = lrp.lrp_lowrank_posterior(G, k=min(1000, G.nx), block=1, eig_tol=1e-6, eig_threshold=eps)
            dt = time.perf_counter() - t0
            lam = post.eigs()
            var = lrp.lrp_posterior_query(post, lrp.LRP_Q_VARIANCE, points=nodes)["variance"]
            out.append({"pde": "convdiff", "nu": nu, "ratio": 1e4, "epsilon": eps, "lanczos_steps": st["n_matvec"],
                        "kept": int(len(lam)), "lambda_1": float(lam[0]) if len(lam) else None, "s": dt,
                        "status": st["status"],
                        "variance_min_mean_max": [float(var.min()), float(var.mean()), float(var.max())],
                        "paper_arnoldi_iterations": PAPER_CD_ARNOLDI_ITERATIONS.get((nu, eps)),
                        "arnoldi": arnoldi_leg(lrp, G, eps, lam)})
            post.close()
        G.close()
    return out


def aggregate_replicas(dist, total_ms: float, matvecs: int, device: str):
    """Whole-job throughput of independent replicas: the matvecs of all ranks
    over the slowest rank's time (max over ranks). dist is torch.distributed
    or None (one process). Returns (value, total_ms, matvecs)."""
    if dist is not None:
        import torch
        t = torch.tensor([total_ms], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        m = torch.tensor([float(matvecs)], device=device, dtype=torch.float64)
        dist.all_reduce(m, op=dist.ReduceOp.SUM)
        matvecs = int(m.item())
    return matvecs / (total_ms / 1e3), total_ms, matvecs


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def roofline_object(kdom, workload, ledger, unit, peaks, peak_kind, dev, block):
    """Roofline figures of the dominant sweep kernel, per launch of the
    Lanczos block apply (`block` columns, a whole Hessian apply): algorithmic
    bytes (the sweep ledger: passes over the solver's fine-level vectors
    implied by the iteration counts) / CUDA-event time, against the bound
    that applies. The band kernel keeps those vectors in shared memory, so
    its bound is shared-memory bandwidth (measured live by the library's own
    kernel) and its DRAM traffic is a side figure; the generic kernel moves
    its vectors through L2/HBM and is set against the HBM copy bandwidth."""
    kname, kdesc, ksources = KERNELS[kdom]
    ms, launches, algo = unit
    achieved = (algo / launches) / (ms / launches / 1e3) / 1e9 if ms > 0 else 0.0
    prof = {}
    try:
        with open(profile_summary(kname, workload)) as f:
            prof = json.load(f)
        if prof.get("kernel_hash") != kernel_hash(ksources):
            prof = {"stale": True}
    except (OSError, ValueError):
        prof = {}
    traffic = prof.get("dram_bytes_per_launch_full")
    hbm = peaks["hbm_gbs"]
    if kdom == 2:
        obj = {"bound": "smem", "achieved": achieved, "peak": dev["smem_gbs"], "unit": "GB/s",
               "frac": achieved / dev["smem_gbs"], "traffic": traffic,
               "peak_kind": "shared-memory bandwidth measured live by lrp_measure_device_peaks (own kernel)"}
        if traffic:
            dram = traffic / (ms / launches / 1e3) / 1e9
            obj["hbm_side_note"] = {"dram_gbs": dram, "frac_of_hbm": dram / hbm,
                                    "hbm_peak_gbs": hbm, "hbm_peak_kind": f"{peak_kind} copy bandwidth"}
    else:
        obj = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
               "traffic": traffic, "peak_kind": f"{peak_kind} copy bandwidth"}
    obj.update({"kernel": f"{kname} ({kdesc})", "kernel_hash": kernel_hash(ksources),
                "unit_of_launch": f"one {block}-column Hessian apply (a Lanczos block step)",
                "algo_bytes_per_launch": algo / max(launches, 1), "ms_per_launch": ms / max(launches, 1),
                "launches": launches,
                "sweep_ms_by_kernel": {KERNELS[kv][0]: ledger[kv][0] for kv in (1, 2)},
                "device_peaks_live": dev})
    if prof.get("ncu"):
        obj["ncu"] = prof["ncu"]
    return obj


def config3_leg(lrp, stream, peaks, peak_kind, dev):
    """The 3D workload (63^3 with the kappa field, nt = 1000, 400 sensors
    every 10th step) beside the headline: one 16-column Hessian apply (its
    Lanczos block) on the mixed path in the launch shape the autotuner picks
    for it (12-CTA clusters of 256 threads, time-step hierarchy cut at 4
    levels; fixed here to keep the bench short), timed by the sweep ledger's
    CUDA events, and its roofline object (generic kernel: HBM bound)."""
    import torch
    spec = synth.workload("heat3d_63")
    X = torch.from_numpy(synth.normal_block(spec.nx, 16, spec.seed + 31)).cuda()
    res = {}
    for bf in (0, 1):
        G = lrp.lrp_setup_problem(spec, precision=lrp.LRP_MIXED, stream=stream, team_ctas=12, team_cols=1,
                                  mg_levels=4, mg_bf16=bf)
        t = lrp.lrp_problem_tuning(G)
        t["threads"] = 256
        lrp.lrp_set_tuning(G, t)
        lrp.lrp_sweep_profile(G, 1)
        Y, st = lrp.lrp_hessian_apply(G, X)
        torch.cuda.synchronize()
        ledger = {kv: lrp.lrp_sweep_profile(G, -1, kv) for kv in (1, 2, 3, 4)}
        lrp.lrp_sweep_profile(G, 0)
        ms, n, algo = ledger[3]
        res[bf] = (Y.cpu().numpy(), st, ms, ledger, lrp.lrp_problem_tuning(G))
        G.close()
    Y0, st, ms, ledger, tune = res[0]
    roof = roofline_object(1, "heat3d_63", ledger, ledger[3], peaks, peak_kind, dev, 16)
    out = {"workload": "heat3d_63: 3D 63^3 (250047 dofs), kappa field, nt=1000, 400 sensors every 10th step, "
                        "sigma=1e-3; one 16-column Hessian apply (mixed)",
           "matvec_per_s": 16 / (ms / 1e3) if ms > 0 else None, "ms_apply": ms, "status": st["status"],
           "pcg_iters_mean": st["pcg_iters_mean"], "launch": tune, "roofline": roof}
    Y1, st1, ms1, ledger1, _ = res[1]
    ms_b, n_b, algo_b = ledger1[3]
    out["bf16_smoothing"] = {
        "what": "the same apply with the multigrid vectors of the global-memory levels stored in BF16 (mg_bf16)",
        "matvec_per_s": 16 / (ms1 / 1e3) if ms1 > 0 else None, "ms_apply": ms1, "status": st1["status"],
        "converged": st1["status"] == 0, "pcg_iters_mean": st1["pcg_iters_mean"],
        "max_rel_residual": st1["max_rel_residual"],
        "max_rel_diff_vs_fp32_smoothing": float(np.max(np.abs(Y1 - Y0)) / np.max(np.abs(Y0))),
        "algo_gbs": (algo_b / n_b) / (ms_b / n_b / 1e3) / 1e9 if ms_b > 0 else None}
    return out


def config_dict(args, nt: int, ws: int = 1) -> dict:
    """The workload configuration both arms print (identical dicts)."""
    return {"workload": workload_name(args.workload, nt),
            "step": ("block Lanczos to rank k + posterior factors + one query + the posterior mean's trajectory "
                     "in low-rank-in-time form" if args.mode == "posterior"
                     else "one Hessian apply to a block of columns"),
            "k": args.k, "block": args.block, "eig_tol": 1e-6, "query": "mean + variance@1024 + 8 samples",
            "parallelism": f"replicas x{max(ws, 1)}"}


def run_reference(args):
    """The oracle (FP64 SciPy, sparse LU or CG solves) timed on this host's
    cores: every step applies Htilde to one block of columns, one column per
    core (a bounded sample of the workload's matvecs; on the 3D workload each
    column is itself sampled over 10 steps and extrapolated)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    nt = args.nt or {"heat2d_127": 500, "heat3d_63": 1000}[args.workload]
    pool = OraclePool(args.workload, args.nt)
    try:
        for _ in range(args.warmup):
            pool.block()
        t_tot, cols = 0.0, 0
        t0 = time.perf_counter()
        for _ in range(args.steps):
            dt, c = pool.block()
            t_tot += dt
            cols += c
        wall = time.perf_counter() - t0
    finally:
        pool.close()
    value = cols / t_tot
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(args, nt, ws),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
                             "sample": pool.sample_text(args.steps, wall)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--workload", default="heat2d_127", choices=sorted(WORKLOAD_DEFAULTS))
    ap.add_argument("--k", type=int, default=0, help="rank (0: the workload's)")
    ap.add_argument("--block", type=int, default=0, help="Lanczos block (0: the workload's)")
    ap.add_argument("--nt", type=int, default=0, help="override nt (profiling of small cases only)")
    ap.add_argument("--team-ctas", type=int, default=0)
    ap.add_argument("--team-cols", type=int, default=0)
    ap.add_argument("--mg-nu", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0, help="threads per CTA (256 or 512; profiling)")
    ap.add_argument("--mg-levels", type=int, default=0, help="time-step hierarchy depth (profiling)")
    ap.add_argument("--mode", default="posterior", choices=["posterior", "apply", "serve", "batched", "paper", "als"],
                    help="posterior: the whole hot path per step; apply: one Hessian apply per step "
                         "(kernel-level measurement and profiling); serve: the serving workload alone")
    ap.add_argument("--als-rank", type=int, default=0,
                    help="--mode als: only this rank, the default preconditioner and --workload (profiling)")
    ap.add_argument("--als-cols", type=int, default=4, help="--mode als with --als-rank: columns per product")
    ap.add_argument("--instances", type=int, default=64)
    ap.add_argument("--batch-steps", type=int, default=2)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=1000)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-budget-gib", type=float, default=24.0)
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-batch", type=int, default=16)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-config3", action="store_true", help="skip the 3D workload's block apply beside the headline")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args()
    k0, b0 = WORKLOAD_DEFAULTS[args.workload]
    args.k = args.k or k0
    args.block = args.block or b0
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_1703_05638_gb300 as lrp
    from paper_1703_05638_gb300 import build as lrp_build

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or ws == 1:
        lrp_build.build()
    if dist:
        dist.barrier()
    lrp.load()

    if args.mode == "batched":
        if rank == 0:
            bt = batched_bench(lrp, args.instances, 16, args.batch_steps)
            print(json.dumps({"metric": "batched Hessian matvecs/s over independent instances",
                              "value": bt["matvec_per_s"], "unit": "matvec/s", "n_gpus": 1,
                              "higher_is_better": True, "data": "synthetic", "dtype": "f32/f64",
                              "config": {"workload": f"batched: {args.instances} 2D instances, grids 63/127/255, "
                                                     "nt 200-2000, k=50, block 16"},
                              "batched": bt}), flush=True)
        if dist:
            dist.destroy_process_group()
        return 0
    if args.mode == "paper":
        if rank == 0:
            prec = lrp.LRP_MIXED if args.precision == "mixed" else lrp.LRP_FP64
            runs = paper_bench(lrp, prec)
            print(json.dumps({"metric": "Lanczos steps to resolve every eigenvalue above epsilon",
                              "unit": "steps", "n_gpus": 1, "data": "synthetic", "dtype": args.precision,
                              "config": {"workload": "paper heat experiment (Sec. 6.1) on FD: 63^2 nodes, nt=30, "
                                                     "9 sensor patches, Gamma_prior=10 I; convection-diffusion "
                                                     "experiment (Sec. 6.2): 31^2 nodes, nt=90, upwind, FP64"},
                              "runs": runs}), flush=True)
        if dist:
            dist.destroy_process_group()
        return 0
    if args.mode == "als":
        if rank == 0:
            prec = lrp.LRP_MIXED if args.precision == "mixed" else lrp.LRP_FP64
            spec = synth.workload(args.workload)
            if args.nt:
                spec.nt, spec.T = args.nt, args.nt * spec.T / spec.nt
            if args.als_rank:
                runs = [als_bench(lrp, spec, prec, ranks=(args.als_rank,), prec=((0.0, 2),), ncols=args.als_cols)]
            else:
                runs = [als_bench(lrp, spec, prec), als_bench(lrp, synth.paper_heat_spec(1e6), prec)]
            print(json.dumps({"metric": "Hessian apply ms per column: alternating low-rank space-time solves "
                                        "vs time stepping", "unit": "ms", "n_gpus": 1, "data": "synthetic",
                              "dtype": args.precision, "higher_is_better": False,
                              "config": {"workload": f"{args.workload} and the paper heat experiment (63^2, nt=30)"},
                              "runs": runs}), flush=True)
        if dist:
            dist.destroy_process_group()
        return 0
    if args.mode == "serve":
        if rank == 0:
            sv = serve_bench(lrp, args.serve_requests, args.serve_rate, args.serve_budget_gib, args.serve_slots,
                             args.serve_batch)
            print(json.dumps({"metric": "serve latency p50 (p99 beside)", "value": sv["p50_ms"], "unit": "ms",
                              "n_gpus": 1, "higher_is_better": False, "data": "synthetic", "dtype": "f32/f64",
                              "config": {"workload": "serving: Poisson stream over 2D 127^2 and 3D 31^3/63^3"},
                              "serve": sv}), flush=True)
        if dist:
            dist.destroy_process_group()
        return 0
    spec = synth.workload(args.workload)
    if args.nt:
        # a shorter horizon with the workload's step size (profiling of small cases)
        spec.T = spec.T * args.nt / spec.nt
        spec.nt = args.nt
    precision = lrp.LRP_MIXED if args.precision == "mixed" else lrp.LRP_FP64
    stream = torch.cuda.current_stream()
    tuning = {}
    if args.team_ctas:
        tuning["team_ctas"] = args.team_ctas
    if args.team_cols:
        tuning["team_cols"] = args.team_cols
    if args.mg_nu:
        tuning["mg_nu"] = args.mg_nu
    if args.mg_levels:
        tuning["mg_levels"] = args.mg_levels
    G = lrp.lrp_setup_problem(spec, precision=precision, stream=stream, **tuning)
    if args.threads:
        t = lrp.lrp_problem_tuning(G)
        t["threads"] = args.threads
        lrp.lrp_set_tuning(G, t)
    if not args.no_autotune and not tuning:
        lrp.lrp_autotune(G, args.block)
    nx = G.nx
    seed = spec.seed + 101 * rank
    # synthetic inputs, resident in HBM: Lanczos start block, data, query nodes, sample draws
    start_h = synth.normal_block(nx, args.block, seed)
    u_true_h = synth.normal_block(nx, 1, seed + 1)
    u_true = lrp.lrp_prior_half(G, torch.from_numpy(u_true_h).cuda())[0]
    d_clean = lrp.lrp_forward_observe(G, u_true)[0]
    noise = torch.from_numpy(synth.normal_block(G.n_data, 1, seed + 2)).cuda()
    y_obs = (d_clean + spec.sigma * noise).reshape(-1).contiguous()
    nodes_h = synth.query_nodes(nx, 1024, seed + 3)
    xi_h = synth.normal_block(nx, 8, seed + 4)
    start_d = torch.from_numpy(start_h).cuda()
    nodes_d = torch.from_numpy(nodes_h).cuda()
    xi_d = torch.from_numpy(xi_h).cuda()
    y_obs_h = y_obs.cpu().numpy()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    kind = lrp.LRP_Q_MEAN | lrp.LRP_Q_VARIANCE | lrp.LRP_Q_SAMPLES

    def step(device=True):
        if args.mode == "apply":
            # kernel-level case: one Hessian apply to the Lanczos-sized block
            _, ast = lrp.lrp_hessian_apply(G, start_d if device else start_h)
            return {"n_matvec": args.block, "ms": ast["ms"], "n_iter": 1, "k_converged": 0,
                    "max_ritz_resid": 0.0, "ms_apply": ast["ms"]}, None
        if device:
            post, st = lrp.lrp_lowrank_posterior(G, k=args.k, block=args.block, eig_tol=1e-6, start=start_d)
            out = lrp.lrp_posterior_query(post, kind, y_obs=y_obs, points=nodes_d, xi=xi_d, device=True)
            mean = out["mean"].reshape(-1, 1)
        else:
            post, st = lrp.lrp_lowrank_posterior(G, k=args.k, block=args.block, eig_tol=1e-6, start=start_h)
            out = lrp.lrp_posterior_query(post, kind, y_obs=y_obs_h, points=nodes_h, xi=xi_h, device=False)
            out["lambda"] = post.eigs()
            mean = out["mean"].reshape(-1, 1)
        # the posterior mean's state trajectory in low-rank-in-time form
        facs, tst = lrp.lrp_trajectory_factors(G, mean)
        out["traj_rank"] = int(facs[0][0].shape[1])
        out["traj_err"] = tst["time_trunc_err"]
        post.close()
        return st, out

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    launches0 = lrp.lrp_kernel_launches()
    lrp.lrp_sweep_profile(G, 1)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats = []
    traj = None
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        st, out_i = step()
        ev[i][1].record(stream)
        stats.append(st)
        if out_i is not None and "traj_rank" in out_i:
            traj = {"rank": out_i["traj_rank"], "trunc_err_bound": out_i["traj_err"]}
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    # ledger: every sweep launch per kernel (1 generic, 2 band) and, per
    # kernel, the launches that run a whole Hessian apply (3, 4): the
    # Lanczos block applies, the unit of the roofline figures
    ledger = {kv: lrp.lrp_sweep_profile(G, -1, kv) for kv in (1, 2, 3, 4)}
    lrp.lrp_sweep_profile(G, 0)
    # the dominant sweep kernel of the timed region (most device time)
    kdom = max((1, 2), key=lambda kv: ledger[kv][0])
    sweep_ms, sweep_launches, sweep_bytes = ledger[kdom + 2]
    if sweep_launches == 0:  # no whole-apply launch of it: all its launches
        sweep_ms, sweep_launches, sweep_bytes = ledger[kdom]
    launches = lrp.lrp_kernel_launches() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = float(sum(step_ms))
    matvecs = sum(s["n_matvec"] for s in stats)
    value, total_ms, matvecs = aggregate_replicas(dist, total_ms, matvecs, "cuda")

    # end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        if args.mode == "apply":
            h2d, d2h = start_h.nbytes, start_h.nbytes
        else:
            h2d = start_h.nbytes + y_obs_h.nbytes + nodes_h.nbytes + xi_h.nbytes + 8 * nx
            d2h = 8 * (args.k + nx + nodes_h.size + nx * xi_h.shape[1]) + 8 * spec.time_rank_max * (nx + spec.nt)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mv = 0
        for _ in range(args.steps):
            st, _ = step(device=False)
            mv += st["n_matvec"]
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e2e = {"value": mv * max(ws, 1) / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}

    # the plain FP64 GPU method on the same workload and GPU: one full
    # time-to-rank-k run (the same Lanczos, every solve in FP64)
    fp64 = None
    if not args.no_fp64_compare and precision == lrp.LRP_MIXED and rank == 0 and args.mode == "posterior":
        G64 = lrp.lrp_setup_problem(spec, precision=lrp.LRP_FP64, stream=stream)
        if not args.no_autotune and not tuning:
            lrp.lrp_autotune(G64, args.block)  # tuned like the mixed path
        lrp.lrp_hessian_apply(G64, start_d[:, :2])
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        post64, st64 = lrp.lrp_lowrank_posterior(G64, k=args.k, block=args.block, eig_tol=1e-6, start=start_d)
        e1.record(stream)
        torch.cuda.synchronize()
        lam64 = post64.eigs()
        post64.close()
        post_m, _ = lrp.lrp_lowrank_posterior(G, k=args.k, block=args.block, eig_tol=1e-6, start=start_d)
        lam_m = post_m.eigs()
        post_m.close()
        kk = min(len(lam64), len(lam_m))
        ms64 = e0.elapsed_time(e1)
        fp64 = {"value": st64["n_matvec"] / (ms64 / 1e3), "unit": UNIT, "s_to_rank_k": ms64 / 1e3,
                "n_matvec": st64["n_matvec"], "tuning": lrp.lrp_problem_tuning(G64),
                "max_rel_eig_diff_vs_mixed": float(np.max(np.abs(lam_m[:kk] - lam64[:kk]) / lam64[0]))}
        G64.close()

    serve = None
    if not args.no_serve and args.mode == "posterior":
        serve = serve_bench(lrp, args.serve_requests, args.serve_rate, args.serve_budget_gib, args.serve_slots,
                            args.serve_batch)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    peaks, peak_kind = measured_peaks()
    dev = lrp.lrp_measure_device_peaks()
    tune = lrp.lrp_problem_tuning(G)
    roofline = roofline_object(kdom, args.workload, ledger, (sweep_ms, sweep_launches, sweep_bytes), peaks,
                               peak_kind, dev, args.block)
    lan = stats[-1]
    cfg3 = None
    if not args.no_config3 and args.mode == "posterior" and args.workload == "heat2d_127":
        cfg3 = config3_leg(lrp, stream, peaks, peak_kind, dev)
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        cpu = cpu_baseline(args.workload, args.nt, lan["n_matvec"] if args.mode == "posterior" else 0)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": max(ws, 1), "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32/f64" if precision == lrp.LRP_MIXED else "f64",
        "data": "synthetic",
        "config": config_dict(args, spec.nt, ws),
        "l2": "flushed (256 MB write) before every timed step",
        "precision": ("f32 MG-PCG inside f64 iterative refinement; f64 Lanczos, re-orthogonalisation, "
                      "eigensolve and posterior" if precision == lrp.LRP_MIXED else "f64 throughout"),
        "launch": tune, "autotuned": not args.no_autotune and not tuning,
        "s_to_rank_k": statistics.mean(s["ms"] for s in stats) / 1e3,
        "lanczos": {"n_iter": lan["n_iter"], "n_matvec": lan["n_matvec"], "k_converged": lan["k_converged"],
                    "max_ritz_resid": lan["max_ritz_resid"], "ms_apply": lan["ms_apply"]},
        "trajectory": traj,
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "fp64_gpu": fp64, "serve": serve,
        "heat3d_63": cfg3,
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
