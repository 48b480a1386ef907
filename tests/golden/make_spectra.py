"""Writes the oracle's reference values for the full-size workloads into
tests/golden/ (expected values of the GPU parity tests at sizes where the
oracle takes minutes to hours, so the tests read them instead of recomputing
them). Calls only the oracle (and the seeded raw inputs of ``synth``).

Files (text; '#' lines are the header, the rest whitespace-separated columns):

* ``spectrum_heat2d_127.txt`` — the 110 leading eigenvalues of the
  prior-preconditioned misfit Hessian (Sec. 2 Eq. (prior_pre); Sec. 6.1
  Eq. (misfit)) of the 127^2 workload (nt = 500, 400 uniform sensors at every
  step, sigma = 1e-3, alpha = 0.05), by ARPACK's Lanczos on the matrix-free
  oracle operator (sparse LU solves), with each pair's explicit residual
  ||Htilde v - lam v|| / lam_1 (for a symmetric operator |lam - lam*| is at
  most the residual norm, and at most its square over the gap to the rest of
  the spectrum).
* ``spectrum_heat3d_63_nt20.txt`` — the 24 leading eigenvalues of the 3D
  63^3 workload (kappa field, 400 uniform sensors every 10th step) cut to its
  first 20 implicit-Euler steps (tau = 1e-3 as in the full workload, T = 0.02),
  with the oracle's CG solves; same columns.
* ``apply_heat3d_63.txt`` — Htilde x for one seeded x (``synth.normal_block``
  seed 2027) on the full 3D workload (nt = 1000), sampled at 256 seeded nodes
  (``synth.query_nodes`` seed 2028), plus ||Htilde x||_max.

Run: ``python tests/golden/make_spectra.py [heat2d|heat3d_eigs|heat3d_apply]``
(all three by default, in parallel processes). The heat3d jobs take about an
hour each on one core; heat2d about 15 minutes.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import spectrum  # noqa: E402
from oracle.problem import Problem  # noqa: E402

APPLY_X_SEED = 2027
APPLY_NODES_SEED = 2028
HEAT3D_EIG_NT = 20
# ARPACK's test is ||r_i|| <= tol |lam_i|; the 110th eigenvalue of the 2D
# workload is ~2.5e-6 lam_1, so 1e-8 asks for residuals near 2.5e-14 lam_1,
# just above the rounding noise of the operator, and the eigenvalue error
# (at most ||r||^2 / gap for a symmetric operator) is far below 1e-10 lam_1
EIGSH_TOL = 1e-8


def heat3d_eig_spec():
    """The 3D workload cut to its first 20 steps (same tau = 1e-3)."""
    return synth.workload("heat3d_63", nt=HEAT3D_EIG_NT, T=HEAT3D_EIG_NT / 1000.0)


def _spectrum(P, k, tol):
    t0 = time.time()
    lam, V = spectrum.eigsh_top(P.hessian_apply, P.nx, k, tol=tol)
    res = np.linalg.norm(P.hessian_apply(V) - V * lam, axis=0) / lam[0]
    return lam, res, time.time() - t0


def _write_spectrum(path, header, lam, res):
    with open(path, "w") as f:
        for line in header:
            f.write(f"# {line}\n")
        f.write("# columns: index (1-based), eigenvalue, ||Htilde v - lam v|| / lam_1\n")
        for i, (l, r) in enumerate(zip(lam, res)):
            f.write(f"{i + 1} {l:.17e} {r:.3e}\n")


def job_heat2d():
    spec = synth.workload("heat2d_127")
    P = Problem(spec)
    lam, res, dt = _spectrum(P, 110, EIGSH_TOL)
    _write_spectrum(os.path.join(HERE, "spectrum_heat2d_127.txt"), [
        "Leading eigenvalues of Htilde = R^-1 F^T F R^-1 / sigma^2 (Sec. 2 Eq. (prior_pre); Sec. 6.1 Eq. (misfit))",
        "workload heat2d_127: 2D heat eq, 127^2 interior, nt=500, T=1, 400 uniform sensors at every step,",
        "sigma=1e-3, prior (I + 0.05 L0)^-2; synth.workload('heat2d_127')",
        f"oracle: sparse LU solves, ARPACK eigsh k=110 tol={EIGSH_TOL:g} (oracle.spectrum.eigsh_top); {dt:.0f} s wall",
        "written by tests/golden/make_spectra.py",
    ], lam, res)


def job_heat3d_eigs():
    spec = heat3d_eig_spec()
    P = Problem(spec, solver="cg")
    lam, res, dt = _spectrum(P, 24, EIGSH_TOL)
    _write_spectrum(os.path.join(HERE, "spectrum_heat3d_63_nt20.txt"), [
        "Leading eigenvalues of Htilde (Sec. 2 Eq. (prior_pre); Sec. 6.1 Eq. (misfit))",
        "workload heat3d_63 cut to its first 20 steps: 3D 63^3 interior, kappa = exp(g) field, tau = 1e-3",
        f"(nt={HEAT3D_EIG_NT}, T=0.02), 400 uniform sensors every 10th step, sigma=1e-3, prior (I + 0.05 L0)^-2",
        f"oracle: CG solves to 1e-14, ARPACK eigsh k=24 tol={EIGSH_TOL:g}; {dt:.0f} s wall",
        "written by tests/golden/make_spectra.py",
    ], lam, res)


def job_heat3d_apply():
    spec = synth.workload("heat3d_63")
    P = Problem(spec, solver="cg")
    t0 = time.time()
    x = synth.normal_block(P.nx, 1, APPLY_X_SEED)[:, 0]
    y = P.hessian_apply(x)
    dt = time.time() - t0
    nodes = synth.query_nodes(P.nx, 256, APPLY_NODES_SEED)
    with open(os.path.join(HERE, "apply_heat3d_63.txt"), "w") as f:
        f.write("# Htilde x (Sec. 2 Eq. (prior_pre); Sec. 6.1 Eq. (misfit)) on the full 3D workload heat3d_63:\n")
        f.write("# 63^3 interior, kappa = exp(g), nt=1000, 400 uniform sensors every 10th step, sigma=1e-3,\n")
        f.write(f"# prior (I + 0.05 L0)^-2; x = synth.normal_block(nx, 1, {APPLY_X_SEED})[:, 0],\n")
        f.write(f"# nodes = synth.query_nodes(nx, 256, {APPLY_NODES_SEED}); oracle CG solves to 1e-14, {dt:.0f} s\n")
        f.write("# written by tests/golden/make_spectra.py\n")
        f.write(f"# max_abs {np.max(np.abs(y)):.17e}\n")
        f.write("# columns: node, (Htilde x)[node]\n")
        for p in nodes:
            f.write(f"{int(p)} {y[p]:.17e}\n")


JOBS = {"heat2d": job_heat2d, "heat3d_eigs": job_heat3d_eigs, "heat3d_apply": job_heat3d_apply}


def main(argv):
    names = argv or list(JOBS)
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=JOBS[n], name=n) for n in names]
    for p in procs:
        p.start()
    rc = 0
    for p in procs:
        p.join()
        print(p.name, "exit", p.exitcode, flush=True)
        rc |= p.exitcode != 0
    return int(rc)


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
