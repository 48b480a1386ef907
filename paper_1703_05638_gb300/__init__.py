"""Python binding of the GB300 low-rank posterior library (C ABI in include/lrp.h).

Argument marshalling only: every step of the computation runs in the CUDA
library ``liblrp.so`` built in-tree for sm_103a. Importing this package does
not load the library; the first call does, and raises if it is missing.

Function names mirror the C entry points (``lrp_setup_problem``,
``lrp_hessian_apply``, ...). Arrays may be NumPy arrays (host memory) or
CUDA torch tensors (device memory); blocks of vectors have shape (rows, ncols)
and are passed column-major, as the C ABI expects.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblrp.so")

LRP_OK, LRP_EINVAL, LRP_ENOMEM, LRP_ENOCONV, LRP_ENONFINITE, LRP_ETIMEOUT, LRP_EBUDGET, LRP_ECUDA = range(8)
LRP_FP64, LRP_MIXED = 0, 1
LRP_PRIOR_LAPLACE, LRP_PRIOR_IDENTITY = 0, 1
LRP_PDE_HEAT, LRP_PDE_CONVDIFF = 0, 1
LRP_PRIOR_PRECOND, LRP_MISFIT_ONLY, LRP_KEEP_TRAJ_FACTORS, LRP_LOWRANK_SOURCE, LRP_ALS_SOLVES = 0, 1, 2, 4, 8
LRP_Q_MEAN, LRP_Q_VARIANCE, LRP_Q_SAMPLES = 1, 2, 4
STATUS_NAMES = {0: "LRP_OK", 1: "LRP_EINVAL", 2: "LRP_ENOMEM", 3: "LRP_ENOCONV", 4: "LRP_ENONFINITE",
                5: "LRP_ETIMEOUT", 6: "LRP_EBUDGET", 7: "LRP_ECUDA"}

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class lrp_problem_desc(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int), ("nt", C.c_int), ("T", C.c_double),
                ("kappa_faces", C.c_void_p), ("prior_alpha", C.c_double), ("n_obs", C.c_int),
                ("obs_xyz", C.c_void_p), ("obs_every", C.c_int), ("sigma", C.c_double),
                ("precision", C.c_int), ("time_trunc_tol", C.c_double), ("time_rank_max", C.c_int),
                ("time_chunk", C.c_int), ("solve_rtol", C.c_double), ("pcg_maxit", C.c_int),
                ("team_ctas", C.c_int), ("team_cols", C.c_int), ("mg_nu", C.c_int),
                ("inner_rtol", C.c_double), ("coarse_items", C.c_int), ("kernel_variant", C.c_int),
                ("mg_nu_coarse", C.c_int), ("prior_kind", C.c_int), ("prior_gamma", C.c_double),
                ("pde", C.c_int), ("conv_nu", C.c_double), ("wind", C.c_double * 3), ("mg_levels", C.c_int),
                ("als_rank", C.c_int), ("als_sweeps", C.c_int), ("als_tol", C.c_double),
                ("als_prec_rtol", C.c_double), ("als_prec_its", C.c_int), ("mg_bf16", C.c_int)]


class lrp_apply_stats(C.Structure):
    _fields_ = [("n_solves", C.c_int), ("pcg_iters_max", C.c_int), ("pcg_iters_mean", C.c_double),
                ("refine_max", C.c_int), ("max_rel_residual", C.c_double), ("time_rank_max", C.c_int),
                ("time_trunc_err", C.c_double), ("ms", C.c_double), ("adj_rank_max", C.c_int),
                ("adj_trunc_err", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class lrp_lanczos_stats(C.Structure):
    _fields_ = [("n_iter", C.c_int), ("n_matvec", C.c_int), ("k_converged", C.c_int),
                ("max_ritz_resid", C.c_double), ("ms", C.c_double), ("ms_apply", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class lrp_query(C.Structure):
    _fields_ = [("kind", C.c_uint), ("y_obs", C.c_void_p), ("sigma", C.c_double), ("n_points", C.c_int),
                ("points", C.c_void_p), ("n_samples", C.c_int), ("xi", C.c_void_p)]


class lrp_query_result(C.Structure):
    _fields_ = [("mean", C.c_void_p), ("variance", C.c_void_p), ("samples", C.c_void_p), ("ms", C.c_double)]


class lrp_server_config(C.Structure):
    _fields_ = [("hbm_budget", C.c_size_t), ("slots", C.c_int), ("max_batch", C.c_int),
                ("max_samples", C.c_int), ("max_points", C.c_int), ("autotune", C.c_int)]


class lrp_request_stats(C.Structure):
    _fields_ = [("t_submit_ms", C.c_double), ("t_start_ms", C.c_double), ("t_done_ms", C.c_double),
                ("batch", C.c_int), ("slot", C.c_int), ("admitted", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class lrp_server_stats(C.Structure):
    _fields_ = [("device_bytes", C.c_size_t), ("models", C.c_int), ("resident", C.c_int),
                ("admissions", C.c_longlong), ("evictions", C.c_longlong), ("batches", C.c_longlong),
                ("served", C.c_longlong), ("pending", C.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class lrp_batch_stats(C.Structure):
    _fields_ = [("steps", C.c_int), ("graph_nodes", C.c_longlong), ("n_matvec", C.c_longlong),
                ("ms_steps", C.c_double), ("ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class lrp_arnoldi_stats(C.Structure):
    _fields_ = [("n_steps", C.c_int), ("k_converged", C.c_int), ("n_complex", C.c_int), ("max_imag", C.c_double),
                ("hess_asym", C.c_double), ("max_ritz_resid", C.c_double), ("time_rank_max", C.c_int),
                ("adj_rank_max", C.c_int), ("ms", C.c_double), ("ms_apply", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class lrp_als_stats(C.Structure):
    _fields_ = [("sweeps", C.c_int), ("gmres_iters", C.c_int), ("gmres_iters_max", C.c_int),
                ("precond_solves", C.c_int), ("residual", C.c_double), ("ms", C.c_double), ("ms_space", C.c_double),
                ("ms_time", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class lrp_device_peaks(C.Structure):
    _fields_ = [("smem_gbs", C.c_double), ("fp64_fma_tflops", C.c_double), ("fp32_fma_tflops", C.c_double),
                ("sm_count", C.c_int), ("clock_mhz", C.c_double)]


class lrp_tuning(C.Structure):
    _fields_ = [("team_ctas", C.c_int), ("team_cols", C.c_int), ("mg_nu", C.c_int), ("mg_nu_coarse", C.c_int),
                ("inner_rtol", C.c_double), ("last_kernel", C.c_int), ("last_team_ctas", C.c_int),
                ("threads", C.c_int), ("waves", C.c_int), ("team_ctas_narrow", C.c_int), ("mg_levels", C.c_int)]


EXPORTS = {
    "lrp_setup_problem": (C.c_int, [C.POINTER(lrp_problem_desc), C.c_void_p, C.POINTER(C.c_void_p)]),
    "lrp_problem_destroy": (None, [C.c_void_p]),
    "lrp_problem_sizes": (C.c_int, [C.c_void_p, _ip, _ip, _ip, _ip]),
    "lrp_hessian_apply": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_uint,
                                    C.POINTER(lrp_apply_stats)]),
    "lrp_hessian_apply_noalloc": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_int,
                                            C.POINTER(lrp_apply_stats)]),
    "lrp_autotune": (C.c_int, [C.c_void_p, C.c_int, C.c_int, _dp]),
    "lrp_forward_observe": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_int,
                                      C.POINTER(lrp_apply_stats)]),
    "lrp_adjoint": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_int,
                              C.POINTER(lrp_apply_stats)]),
    "lrp_prior_half": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_int,
                                 C.POINTER(lrp_apply_stats)]),
    "lrp_trajectory_factors": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                                         C.c_void_p, C.POINTER(lrp_apply_stats)]),
    "lrp_lowrank_posterior": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int,
                                        C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(lrp_lanczos_stats)]),
    "lrp_arnoldi": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_double, C.c_uint, C.c_void_p,
                              C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p),
                              C.POINTER(lrp_arnoldi_stats)]),
    "lrp_hessenberg_eig": (C.c_int, [C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p]),
    "lrp_als_solve": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int,
                                C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_void_p, C.c_int, C.c_void_p, C.c_int,
                                C.c_void_p, C.POINTER(lrp_als_stats)]),
    "lrp_st_hessian_apply": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p,
                                       C.c_void_p, _ip, C.POINTER(lrp_apply_stats)]),
    "lrp_st_arnoldi": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int, C.c_void_p,
                                 C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.POINTER(lrp_arnoldi_stats)]),
    "lrp_posterior_destroy": (None, [C.c_void_p]),
    "lrp_posterior_eigs": (C.c_int, [C.c_void_p, _ip, C.c_void_p, C.c_void_p, C.c_int]),
    "lrp_posterior_query": (C.c_int, [C.c_void_p, C.POINTER(lrp_query), C.POINTER(lrp_query_result)]),
    "lrp_posterior_save": (C.c_int, [C.c_void_p, C.c_char_p]),
    "lrp_posterior_load": (C.c_int, [C.c_void_p, C.c_char_p, C.POINTER(C.c_void_p)]),
    "lrp_last_error": (C.c_char_p, []),
    "lrp_version": (C.c_char_p, []),
    "lrp_kernel_launches": (C.c_ulonglong, []),
    "lrp_debug_fail_alloc": (None, [C.c_longlong]),
    "lrp_measure_device_peaks": (C.c_int, [C.POINTER(lrp_device_peaks)]),
    "lrp_sweep_profile": (C.c_int, [C.c_void_p, C.c_int, C.c_int, _dp, C.POINTER(C.c_ulonglong), _dp]),
    "lrp_problem_tuning": (C.c_int, [C.c_void_p, C.POINTER(lrp_tuning)]),
    "lrp_batch_lowrank_posterior": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.c_int, C.c_double, C.c_int,
                                              C.c_int, C.POINTER(C.c_void_p), C.POINTER(lrp_lanczos_stats),
                                              C.POINTER(lrp_batch_stats)]),
    "lrp_set_tuning": (C.c_int, [C.c_void_p, C.POINTER(lrp_tuning)]),
    "lrp_server_create": (C.c_int, [C.POINTER(lrp_server_config), C.POINTER(C.c_void_p)]),
    "lrp_server_add_model": (C.c_int, [C.c_void_p, C.POINTER(lrp_problem_desc), C.c_int, C.c_int, C.c_double,
                                       C.c_char_p, C.POINTER(C.c_int), C.POINTER(lrp_lanczos_stats)]),
    "lrp_server_submit": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(lrp_query), C.POINTER(C.c_ulonglong)]),
    "lrp_server_wait": (C.c_int, [C.c_void_p, C.c_ulonglong, C.c_double, C.POINTER(lrp_query_result),
                                  C.POINTER(lrp_request_stats)]),
    "lrp_server_info": (C.c_int, [C.c_void_p, C.POINTER(lrp_server_stats)]),
    "lrp_server_destroy": (None, [C.c_void_p]),
}

_lib = None
_lock = threading.Lock()


def load(path: Optional[str] = None):
    """Load liblrp.so (building nothing). Raises if the library is missing."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"CUDA library {p} is missing: run __graft_entry__.build() "
                                   "(or python paper_1703_05638_gb300/build.py) first")
            lib = C.CDLL(p)
            for name, (res, args) in EXPORTS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


class LrpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(status, allow=(LRP_OK,)):
    if status not in allow:
        raise LrpError(status, load().lrp_last_error().decode())
    return status


# --------------------------------------------------------------------------- arrays
def _is_torch(x):
    return type(x).__module__.startswith("torch")


class _Arg:
    """A column-major view of a (rows, ncols) block as a raw pointer."""

    def __init__(self, x, rows: int, dtype=np.float64):
        self.keep = None
        if x is None:
            self.ptr, self.ld, self.ncols, self.kind = None, rows, 0, "none"
            return
        if _is_torch(x):
            import torch
            t = x if x.dim() == 2 else x.reshape(-1, 1)
            assert t.shape[0] == rows, (tuple(t.shape), rows)
            tdt = torch.float64 if dtype == np.float64 else torch.int32
            ct = t.t().contiguous().to(tdt)  # (ncols, rows) row-major == column-major block
            self.keep = ct
            self.ptr, self.ld, self.ncols, self.kind = ct.data_ptr(), rows, t.shape[1], "torch"
        else:
            a = np.asarray(x, dtype=dtype)
            if a.ndim == 1:
                a = a.reshape(-1, 1)
            assert a.shape[0] == rows, (a.shape, rows)
            a = np.asfortranarray(a)
            self.keep = a
            self.ptr, self.ld, self.ncols, self.kind = a.ctypes.data, rows, a.shape[1], "numpy"


def _out_like(arg: _Arg, rows: int, ncols: int, like):
    if arg.kind == "torch":
        import torch
        t = torch.empty((ncols, rows), dtype=torch.float64, device=like.device)
        return t, t.data_ptr(), lambda: t.t()
    a = np.empty((rows, ncols), dtype=np.float64, order="F")
    return a, a.ctypes.data, lambda: a


# --------------------------------------------------------------------------- problem
class Problem:
    """Owner of one lrp_problem handle."""

    def __init__(self, handle, desc):
        self.handle = handle
        self.desc = desc
        nx, no, ns, nd = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        _check(load().lrp_problem_sizes(handle, C.byref(nx), C.byref(no), C.byref(ns), C.byref(nd)))
        self.nx, self.n_obs, self.n_steps, self.n_data = nx.value, no.value, ns.value, nd.value
        self.nt = int(desc.nt)

    def close(self):
        if self.handle:
            load().lrp_problem_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _desc(spec, precision, tuning, keep):
    d = lrp_problem_desc()
    d.dim, d.n, d.nt, d.T = int(spec.dim), int(spec.n), int(spec.nt), float(spec.T)
    kap = getattr(spec, "kappa", None)
    if kap is not None:
        k = np.ascontiguousarray(np.concatenate([np.asarray(f, dtype=np.float64).ravel() for f in kap]))
        keep.append(k)
        d.kappa_faces = k.ctypes.data
    d.prior_alpha = float(spec.prior_alpha)
    d.prior_kind = int(getattr(spec, "prior_kind", 0) or 0)
    d.prior_gamma = float(getattr(spec, "prior_gamma", 0.0) or 0.0)
    if (getattr(spec, "pde", "heat") or "heat") == "convdiff":
        d.pde = LRP_PDE_CONVDIFF
        d.conv_nu = float(spec.conv_nu)
        for a, v in enumerate(spec.wind):
            d.wind[a] = float(v)
    sens = np.ascontiguousarray(np.asarray(spec.sensors, dtype=np.float64))
    keep.append(sens)
    d.n_obs = sens.shape[0]
    d.obs_xyz = sens.ctypes.data
    d.obs_every = int(spec.obs_every)
    d.sigma = float(spec.sigma)
    d.precision = int(precision)
    d.time_trunc_tol = float(getattr(spec, "time_trunc_tol", 1e-8) or 1e-8)
    d.time_rank_max = int(getattr(spec, "time_rank_max", 40) or 40)
    for key, val in tuning.items():
        setattr(d, key, val)
    return d


def lrp_setup_problem(spec, precision: int = LRP_FP64, stream=None, **tuning) -> Problem:
    """Set up a problem from an object with the attributes of synth.ProblemSpec
    (dim, n, nt, T, prior_alpha, sigma, obs_every, sensors, kappa)."""
    lib = load()
    keep = []
    d = _desc(spec, precision, tuning, keep)
    h = C.c_void_p()
    s = 0 if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(lib.lrp_setup_problem(C.byref(d), C.c_void_p(s), C.byref(h)))
    return Problem(h, d)


def _sweep(fn, prob: Problem, X, rows_in, rows_out, *extra):
    a = _Arg(X, rows_in)
    out, optr, view = _out_like(a, rows_out, a.ncols, X)
    st = lrp_apply_stats()
    status = fn(prob.handle, a.ncols, C.c_void_p(a.ptr), a.ld, C.c_void_p(optr), rows_out, *extra, C.byref(st))
    _check(status, allow=(LRP_OK, LRP_ENOCONV))
    d = st.as_dict()
    d["status"] = status
    return view(), d


def lrp_hessian_apply(prob: Problem, X, flags: int = 0):
    """Y = Htilde X (or H_mis X with LRP_MISFIT_ONLY). Returns (Y, stats)."""
    return _sweep(load().lrp_hessian_apply, prob, X, prob.nx, prob.nx, C.c_uint(flags))


def lrp_hessian_apply_noalloc(prob: Problem, X):
    """Y = Htilde X with the library's fixed workspace (no device allocation
    by the call). X must be a CUDA torch tensor (nx, ncols); returns (Y, stats)
    with Y a CUDA tensor. The output tensor is allocated here, by the caller
    side, not by the library."""
    if not _is_torch(X) or not X.is_cuda:
        raise ValueError("lrp_hessian_apply_noalloc needs a CUDA tensor")
    return _sweep(load().lrp_hessian_apply_noalloc, prob, X, prob.nx, prob.nx)


def lrp_autotune(prob: Problem, nvec: int, steps: int = 16) -> float:
    """Pick the fastest launch shape / multigrid setting for blocks of nvec
    columns (kept in the problem); returns the winner's Hessian-apply time
    in ms."""
    ms = C.c_double()
    _check(load().lrp_autotune(prob.handle, int(nvec), int(steps), C.byref(ms)))
    return ms.value


def lrp_forward_observe(prob: Problem, U):
    """D = F U. Returns (D, stats), D of shape (n_data, ncols)."""
    return _sweep(load().lrp_forward_observe, prob, U, prob.nx, prob.n_data)


def lrp_adjoint(prob: Problem, D):
    """U = F^T D. Returns (U, stats)."""
    return _sweep(load().lrp_adjoint, prob, D, prob.n_data, prob.nx)


def lrp_prior_half(prob: Problem, X):
    """Y = Gamma_prior^{1/2} X = (I + alpha L0)^{-1} X. Returns (Y, stats)."""
    return _sweep(load().lrp_prior_half, prob, X, prob.nx, prob.nx)


def lrp_trajectory_factors(prob: Problem, U):
    """Low-rank-in-time factors of the forward trajectories of the columns of
    U (NumPy, or a CUDA torch tensor: the factors then stay on the device):
    returns (list of (W, V) with Y_j ~ W V^T, stats)."""
    rmax = prob.desc.time_rank_max
    nt = prob.desc.nt
    if _is_torch(U):
        import torch
        a = _Arg(U, prob.nx)
        W = torch.zeros((a.ncols, rmax, prob.nx), dtype=torch.float64, device=U.device)
        V = torch.zeros((a.ncols, rmax, nt), dtype=torch.float64, device=U.device)
        ranks = np.zeros(a.ncols, dtype=np.int32)
        st = lrp_apply_stats()
        status = load().lrp_trajectory_factors(prob.handle, a.ncols, C.c_void_p(a.ptr), a.ld,
                                               C.c_void_p(W.data_ptr()), C.c_void_p(V.data_ptr()),
                                               C.c_void_p(ranks.ctypes.data), C.byref(st))
        _check(status, allow=(LRP_OK, LRP_ENOCONV))
        return [(W[j, :ranks[j]].T, V[j, :ranks[j]].T) for j in range(a.ncols)], st.as_dict()
    a = _Arg(np.asarray(U), prob.nx)
    W = np.zeros((a.ncols, rmax, prob.nx))
    V = np.zeros((a.ncols, rmax, nt))
    ranks = np.zeros(a.ncols, dtype=np.int32)
    st = lrp_apply_stats()
    status = load().lrp_trajectory_factors(prob.handle, a.ncols, C.c_void_p(a.ptr), a.ld,
                                           C.c_void_p(W.ctypes.data), C.c_void_p(V.ctypes.data),
                                           C.c_void_p(ranks.ctypes.data), C.byref(st))
    _check(status, allow=(LRP_OK, LRP_ENOCONV))
    out = [(W[j, :ranks[j]].T.copy(), V[j, :ranks[j]].T.copy()) for j in range(a.ncols)]
    return out, st.as_dict()


class Posterior:
    def __init__(self, handle, prob: Problem):
        self.handle = handle
        self.prob = prob

    def eigs(self, vectors: bool = False):
        r = C.c_int()
        lib = load()
        _check(lib.lrp_posterior_eigs(self.handle, C.byref(r), None, None, 0))
        lam = np.zeros(max(r.value, 1))
        V = np.zeros((self.prob.nx, max(r.value, 1)), order="F") if vectors else None
        _check(lib.lrp_posterior_eigs(self.handle, C.byref(r), C.c_void_p(lam.ctypes.data),
                                      C.c_void_p(V.ctypes.data) if vectors else None, self.prob.nx))
        lam = lam[:r.value]
        return (lam, V[:, :r.value]) if vectors else lam

    def close(self):
        if self.handle:
            load().lrp_posterior_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lrp_lowrank_posterior(prob: Problem, k: int, block: int = 1, eig_tol: float = 1e-6,
                          eig_threshold: float = 0.0, max_basis: int = 0, start=None):
    """Block Lanczos for the k leading eigenpairs of Htilde; returns (Posterior, stats)."""
    lib = load()
    a = _Arg(start, prob.nx) if start is not None else None
    h = C.c_void_p()
    st = lrp_lanczos_stats()
    status = lib.lrp_lowrank_posterior(prob.handle, int(k), int(block), float(eig_tol), float(eig_threshold),
                                       int(max_basis), C.c_void_p(a.ptr) if a else None, C.byref(h),
                                       C.byref(st))
    _check(status, allow=(LRP_OK, LRP_ENOCONV))
    d = st.as_dict()
    d["status"] = status
    return Posterior(h, prob), d


def lrp_arnoldi(prob: Problem, max_steps: int, k: int = 0, eig_tol: float = 1e-6, eig_threshold: float = 0.0,
                flags: int = 0, start=None, posterior: bool = False):
    """Arnoldi process of Algorithm 1 (modified Gram-Schmidt, Hessenberg H)
    on Htilde, H_mis (LRP_MISFIT_ONLY) or the truncated product
    (LRP_LOWRANK_SOURCE). Returns a dict: 'theta' (complex Ritz values by
    decreasing real part), 'H' ((m+1) x m), 'ranks_y', 'ranks_q' (per step),
    'posterior' (a Posterior or None), 'stats' (with 'status')."""
    mmax = int(max_steps)
    re = np.zeros(mmax)
    im = np.zeros(mmax)
    H = np.zeros((mmax + 1, mmax), order="F")
    ry = np.zeros(mmax, dtype=np.int32)
    rq = np.zeros(mmax, dtype=np.int32)
    keep = []
    sp = None
    if start is not None:
        if _is_torch(start):
            t = start.contiguous()
            keep.append(t)
            sp = t.data_ptr()
        else:
            a = np.ascontiguousarray(np.asarray(start, dtype=np.float64).ravel())
            keep.append(a)
            sp = a.ctypes.data
    h = C.c_void_p()
    st = lrp_arnoldi_stats()
    status = load().lrp_arnoldi(prob.handle, mmax, int(k), float(eig_tol), float(eig_threshold), C.c_uint(flags),
                                sp, re.ctypes.data, im.ctypes.data, H.ctypes.data, ry.ctypes.data, rq.ctypes.data,
                                C.byref(h) if posterior else None, C.byref(st))
    _check(status, allow=(LRP_OK, LRP_ENOCONV))
    m = st.n_steps
    d = st.as_dict()
    d["status"] = status
    return {"theta": re[:m] + 1j * im[:m], "H": np.array(H[:m + 1, :m]), "ranks_y": ry[:m].copy(),
            "ranks_q": rq[:m].copy(), "posterior": Posterior(h, prob) if posterior else None, "stats": d}


def lrp_st_hessian_apply(prob: Problem, W, V):
    """Htilde (W V^T) for the space-time source parameter; returns
    (Wout, Vout, stats) with Wout Vout^T the truncated product."""
    Wa = np.asfortranarray(np.asarray(W, dtype=np.float64).reshape(prob.nx, -1))
    Va = np.asfortranarray(np.asarray(V, dtype=np.float64).reshape(prob.nt, -1))
    rmax = prob.desc.time_rank_max
    Wo = np.zeros((prob.nx, rmax), order="F")
    Vo = np.zeros((prob.nt, rmax), order="F")
    r = C.c_int()
    st = lrp_apply_stats()
    status = load().lrp_st_hessian_apply(prob.handle, Wa.shape[1], Wa.ctypes.data, prob.nx, Va.ctypes.data, prob.nt,
                                         Wo.ctypes.data, Vo.ctypes.data, C.byref(r), C.byref(st))
    _check(status, allow=(LRP_OK, LRP_ENOCONV))
    d = st.as_dict()
    d["status"] = status
    return Wo[:, :r.value].copy(), Vo[:, :r.value].copy(), d


def lrp_als_solve(prob: Problem, Wf, Vf, V0, sweeps: int, tol: float = 0.0, transpose: bool = False):
    """Alternating low-rank solve of the space-time system with the source
    Wf Vf^T (Wf: nx x rf, Vf: nt x rf) from the start V0 (nt x r). Returns
    (W, V, residuals, stats) with Y ~ W V^T. NumPy arrays (host)."""
    Wa = np.asfortranarray(np.asarray(Wf, dtype=np.float64).reshape(prob.nx, -1))
    Va = np.asfortranarray(np.asarray(Vf, dtype=np.float64).reshape(prob.nt, -1))
    V0a = np.asfortranarray(np.asarray(V0, dtype=np.float64).reshape(prob.nt, -1))
    rf, r = Wa.shape[1], V0a.shape[1]
    W = np.zeros((prob.nx, r), order="F")
    V = np.zeros((prob.nt, r), order="F")
    res = np.zeros(int(sweeps))
    st = lrp_als_stats()
    status = load().lrp_als_solve(prob.handle, int(bool(transpose)), rf, Wa.ctypes.data, prob.nx, Va.ctypes.data,
                                  prob.nt, r, V0a.ctypes.data, prob.nt, int(sweeps), float(tol), W.ctypes.data,
                                  prob.nx, V.ctypes.data, prob.nt, res.ctypes.data, C.byref(st))
    _check(status, allow=(LRP_OK, LRP_ENOCONV))
    d = st.as_dict()
    d["status"] = status
    return W, V, res[:st.sweeps].copy(), d


def lrp_st_arnoldi(prob: Problem, max_steps: int, k: int = 0, eig_tol: float = 1e-6, eig_threshold: float = 0.0,
                   W0=None, V0=None):
    """Algorithm 1 on low-rank space-time vectors. Returns a dict: 'theta',
    'H', 'ranks' (rank of each new Krylov vector), 'stats'."""
    mmax = int(max_steps)
    re = np.zeros(mmax)
    im = np.zeros(mmax)
    H = np.zeros((mmax + 1, mmax), order="F")
    rk = np.zeros(mmax, dtype=np.int32)
    r0, wp, vp, keep = 0, None, None, []
    if W0 is not None:
        Wa = np.asfortranarray(np.asarray(W0, dtype=np.float64).reshape(prob.nx, -1))
        Va = np.asfortranarray(np.asarray(V0, dtype=np.float64).reshape(prob.nt, -1))
        keep += [Wa, Va]
        r0, wp, vp = Wa.shape[1], Wa.ctypes.data, Va.ctypes.data
    st = lrp_arnoldi_stats()
    status = load().lrp_st_arnoldi(prob.handle, mmax, int(k), float(eig_tol), float(eig_threshold), r0, wp, vp,
                                   re.ctypes.data, im.ctypes.data, H.ctypes.data, rk.ctypes.data, C.byref(st))
    _check(status, allow=(LRP_OK, LRP_ENOCONV))
    m = st.n_steps
    d = st.as_dict()
    d["status"] = status
    return {"theta": re[:m] + 1j * im[:m], "H": np.array(H[:m + 1, :m]), "ranks": rk[:m].copy(), "stats": d}


def lrp_hessenberg_eig(H, want_schur: bool = False):
    """Eigenvalues of an upper Hessenberg matrix (Francis double-shift QR on
    the GPU). Returns (wr + i wi in Schur-diagonal order) or, with want_schur,
    (eigenvalues, T, Z) with H = Z T Z^T."""
    A = np.asfortranarray(np.asarray(H, dtype=np.float64))
    m = A.shape[0]
    wr = np.zeros(m)
    wi = np.zeros(m)
    T = np.zeros((m, m), order="F") if want_schur else None
    Z = np.zeros((m, m), order="F") if want_schur else None
    _check(load().lrp_hessenberg_eig(m, A.ctypes.data, m, wr.ctypes.data, wi.ctypes.data,
                                     T.ctypes.data if want_schur else None, Z.ctypes.data if want_schur else None))
    lam = wr + 1j * wi
    return (lam, T, Z) if want_schur else lam


def lrp_posterior_query(post: Posterior, kind: int, y_obs=None, sigma: float = 0.0, points=None, xi=None,
                        device: bool = False):
    """Mean / pointwise variance / samples. Inputs may be NumPy (host) or CUDA
    torch tensors; outputs are NumPy arrays, or CUDA torch tensors if device.
    Returns a dict with 'mean', 'variance', 'samples', 'ms'."""
    lib = load()
    nx = post.prob.nx
    q = lrp_query()
    res = lrp_query_result()
    keep = []
    out = {}
    q.kind = kind
    q.sigma = float(sigma)

    def alloc(shape):
        if device:
            import torch
            t = torch.empty(shape[::-1] if len(shape) == 2 else shape, dtype=torch.float64, device="cuda")
            return (t.t() if len(shape) == 2 else t), t.data_ptr()
        a = np.zeros(shape, order="F")
        return a, a.ctypes.data

    def inp(x, dtype):
        if _is_torch(x):
            t = x.contiguous()
            keep.append(t)
            return t.data_ptr(), t.numel()
        a = np.ascontiguousarray(np.asarray(x, dtype=dtype).ravel())
        keep.append(a)
        return a.ctypes.data, a.size

    if y_obs is not None:
        q.y_obs, _ = inp(y_obs, np.float64)
    if kind & (LRP_Q_MEAN | LRP_Q_SAMPLES):
        out["mean"], res.mean = alloc((nx,))
    if kind & LRP_Q_VARIANCE:
        q.points, q.n_points = inp(points, np.int32)
        out["variance"], res.variance = alloc((q.n_points,))
    if kind & LRP_Q_SAMPLES:
        if _is_torch(xi):
            a = _Arg(xi, nx)
            keep.append(a)
            q.xi, q.n_samples = a.ptr, a.ncols
        else:
            x = np.asfortranarray(np.asarray(xi, dtype=np.float64).reshape(nx, -1))
            keep.append(x)
            q.xi, q.n_samples = x.ctypes.data, x.shape[1]
        out["samples"], res.samples = alloc((nx, q.n_samples))
    out["status"] = _check(lib.lrp_posterior_query(post.handle, C.byref(q), C.byref(res)),
                           allow=(LRP_OK, LRP_ENOCONV))
    out["ms"] = res.ms
    return out


def lrp_batch_lowrank_posterior(probs, k: int, block: int = 16, eig_tol: float = 1e-6, use_graph: bool = True,
                                max_steps: int = 0):
    """Block Lanczos on several problems at once (each on its own stream; one
    CUDA graph per block step with use_graph). Returns ([(Posterior, stats)],
    batch stats)."""
    n = len(probs)
    hs = (C.c_void_p * n)(*[p.handle for p in probs])
    outs = (C.c_void_p * n)()
    sts = (lrp_lanczos_stats * n)()
    bst = lrp_batch_stats()
    _check(load().lrp_batch_lowrank_posterior(hs, n, int(k), int(block), float(eig_tol), int(bool(use_graph)),
                                              int(max_steps), outs, sts, C.byref(bst)), allow=(LRP_OK, LRP_ENOCONV))
    return [(Posterior(C.c_void_p(outs[i]), probs[i]), sts[i].as_dict()) for i in range(n)], bst.as_dict()


def lrp_posterior_save(post: Posterior, path: str):
    _check(load().lrp_posterior_save(post.handle, path.encode()))


def lrp_posterior_load(prob: Problem, path: str) -> Posterior:
    h = C.c_void_p()
    _check(load().lrp_posterior_load(prob.handle, path.encode(), C.byref(h)))
    return Posterior(h, prob)


def lrp_last_error() -> str:
    return load().lrp_last_error().decode()


def lrp_version() -> str:
    return load().lrp_version().decode()


def lrp_sweep_profile(prob: "Problem", mode: int = -1, kernel: int = 0):
    """Sweep-kernel ledger: returns (ms, launches, algorithmic bytes) accumulated
    so far for kernel (0 all sweep launches, 1 generic team kernel, 2 band
    kernel); mode 1 resets and starts recording, 0 resets and stops, -1 reads."""
    ms, n, b = C.c_double(), C.c_ulonglong(), C.c_double()
    _check(load().lrp_sweep_profile(prob.handle, int(mode), int(kernel), C.byref(ms), C.byref(n), C.byref(b)))
    return ms.value, int(n.value), b.value


class Server:
    """Posterior-query server (continuous batching over several models on one
    GPU; see lrp_server_* in lrp.h). Results come back as NumPy arrays."""

    def __init__(self, hbm_budget: int = 0, slots: int = 0, max_batch: int = 0, max_samples: int = 0,
                 max_points: int = 0, autotune: bool = False):
        cfg = lrp_server_config(int(hbm_budget), int(slots), int(max_batch), int(max_samples), int(max_points),
                                int(bool(autotune)))
        h = C.c_void_p()
        _check(load().lrp_server_create(C.byref(cfg), C.byref(h)))
        self.handle = h
        self._nx = {}
        self._shape = {}

    def add_model(self, spec, k: int, precision: int = LRP_MIXED, block: int = 16, eig_tol: float = 1e-6,
                  factors_path=None, **tuning):
        """Returns (model id, Lanczos stats)."""
        keep = []
        d = _desc(spec, precision, tuning, keep)
        mid = C.c_int()
        st = lrp_lanczos_stats()
        path = factors_path.encode() if factors_path else None
        _check(load().lrp_server_add_model(self.handle, C.byref(d), int(k), int(block), float(eig_tol), path,
                                           C.byref(mid), C.byref(st)), allow=(LRP_OK, LRP_ENOCONV))
        self._nx[mid.value] = int(spec.n) ** int(spec.dim)
        return mid.value, st.as_dict()

    def submit(self, model: int, kind: int, y_obs=None, sigma: float = 0.0, points=None, xi=None) -> int:
        q = lrp_query()
        q.kind = kind
        q.sigma = float(sigma)
        keep = []
        nx = self._nx.get(model, 1)  # an unknown model is rejected by the library
        if y_obs is not None:
            y = np.ascontiguousarray(np.asarray(y_obs, dtype=np.float64).ravel())
            keep.append(y)
            q.y_obs = y.ctypes.data
        npts = ns = 0
        if points is not None:
            pt = np.ascontiguousarray(np.asarray(points, dtype=np.int32).ravel())
            keep.append(pt)
            q.points, q.n_points = pt.ctypes.data, pt.size
            npts = pt.size
        if xi is not None:
            x = np.asfortranarray(np.asarray(xi, dtype=np.float64).reshape(nx, -1))
            keep.append(x)
            q.xi, q.n_samples = x.ctypes.data, x.shape[1]
            ns = x.shape[1]
        t = C.c_ulonglong()
        _check(load().lrp_server_submit(self.handle, int(model), C.byref(q), C.byref(t)))
        self._shape[t.value] = (kind, nx, npts, ns)
        return t.value

    def wait(self, ticket: int, timeout: float = 0.0) -> dict:
        """Results of a request (NumPy arrays) with its stats and status
        (LRP_OK or LRP_ENOCONV); LRP_ETIMEOUT raises and keeps the ticket."""
        kind, nx, npts, ns = self._shape[ticket]
        res = lrp_query_result()
        out = {}
        if kind & (LRP_Q_MEAN | LRP_Q_SAMPLES):
            out["mean"] = np.zeros(nx)
            res.mean = out["mean"].ctypes.data
        if kind & LRP_Q_VARIANCE:
            out["variance"] = np.zeros(npts)
            res.variance = out["variance"].ctypes.data
        if kind & LRP_Q_SAMPLES:
            out["samples"] = np.zeros((nx, ns), order="F")
            res.samples = out["samples"].ctypes.data
        st = lrp_request_stats()
        status = load().lrp_server_wait(self.handle, C.c_ulonglong(ticket), float(timeout), C.byref(res),
                                        C.byref(st))
        if status != LRP_ETIMEOUT:
            self._shape.pop(ticket, None)
        out["status"] = _check(status, allow=(LRP_OK, LRP_ENOCONV))
        out["stats"] = st.as_dict()
        out["latency_ms"] = st.t_done_ms - st.t_submit_ms
        return out

    def info(self) -> dict:
        st = lrp_server_stats()
        _check(load().lrp_server_info(self.handle, C.byref(st)))
        return st.as_dict()

    def close(self):
        if self.handle:
            load().lrp_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lrp_problem_tuning(prob: "Problem") -> dict:
    """Current launch/multigrid settings and what the last sweep launch used
    (last_kernel: 1 generic team kernel, 2 band kernel, 0 none yet)."""
    t = lrp_tuning()
    _check(load().lrp_problem_tuning(prob.handle, C.byref(t)))
    return {f: getattr(t, f) for f, _ in lrp_tuning._fields_}


def lrp_set_tuning(prob: "Problem", tuning: dict):
    """Apply a setting read by lrp_problem_tuning (e.g. from an autotuned problem of the same size)."""
    t = lrp_tuning()
    for f, _ in lrp_tuning._fields_:
        if f in tuning:
            setattr(t, f, tuning[f])
    _check(load().lrp_set_tuning(prob.handle, C.byref(t)))


def lrp_kernel_launches() -> int:
    return int(load().lrp_kernel_launches())


def lrp_measure_device_peaks() -> dict:
    """Shared-memory bandwidth and FP64/FP32 FMA throughput of the current
    device, measured with the library's own kernels."""
    pk = lrp_device_peaks()
    _check(load().lrp_measure_device_peaks(C.byref(pk)))
    return {f: getattr(pk, f) for f, _ in lrp_device_peaks._fields_}


def lrp_debug_fail_alloc(after: int):
    """Test hook: the device allocation after `after` more successful ones
    fails as if the device were full (once); after < 0 disarms it."""
    load().lrp_debug_fail_alloc(int(after))
