"""Parity at the benchmark's full sizes, against values written by the
oracle ahead of time (tests/golden/make_spectra.py; the oracle needs minutes
to hours there, so the tests read its results):

* the 127^2 workload in the benchmark's exact configuration (autotuned,
  Lanczos blocks of 32, k = 100, Ritz residual 1e-6 theta_1): its 100
  leading eigenvalues against the oracle's, in both paths;
* the 3D 63^3 workload (kappa field) cut to its first 20 steps: the 16
  leading eigenvalues with blocks of 16, in both paths;
* the full 3D workload (nt = 1000): one Hessian apply sampled at 256 nodes.

Eigenvalue parity (the reading of the tolerance for a spectrum that spans
many orders): |lam_i - lam*_i| <= tol lam*_1 for every i <= k, and relative
error <= tol where lam*_i >= 1e-3 lam*_1 (mixed) or 1e-6 lam*_1 (FP64).
The Lanczos stopping tolerance bounds what any path can reach (for a
symmetric operator a Ritz value is within its residual norm of an
eigenvalue), so the FP64 runs stop at a residual of 1e-10 theta_1 and the
mixed runs at the benchmark's 1e-6.
"""
import os

import numpy as np
import pytest

import synth

lrp = pytest.importorskip("paper_1703_05638_gb300")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TOL = {lrp.LRP_FP64: 1e-10, lrp.LRP_MIXED: 1e-6}
RESOLVABLE = {lrp.LRP_FP64: 1e-6, lrp.LRP_MIXED: 1e-3}
EIG_TOL = {lrp.LRP_FP64: 1e-10, lrp.LRP_MIXED: 1e-6}


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_05638_gb300 import build
    build.build()
    lrp.load()


def _rows(name):
    rows, meta = [], {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line.startswith("#"):
                parts = line[1:].split()
                if len(parts) == 2 and parts[0] == "max_abs":
                    meta["max_abs"] = float(parts[1])
            elif line:
                rows.append(line.split())
    return rows, meta


def _golden_spectrum(name):
    rows, _ = _rows(name)
    lam = np.array([float(r[1]) for r in rows])
    res = np.array([float(r[2]) for r in rows])
    return lam, res


def _check(lam, lam_ref, tol, resolvable):
    k = len(lam)
    assert k == len(lam_ref)
    abs_err = np.max(np.abs(lam - lam_ref)) / lam_ref[0]
    big = lam_ref >= resolvable * lam_ref[0]
    rel_err = np.max(np.abs(lam[big] - lam_ref[big]) / lam_ref[big])
    assert abs_err <= tol and rel_err <= tol, (abs_err, rel_err)


@pytest.mark.parametrize("precision", [lrp.LRP_MIXED, lrp.LRP_FP64])
def test_heat2d_127_spectrum_in_bench_configuration(precision):
    lam_ref, res_ref = _golden_spectrum("spectrum_heat2d_127.txt")
    # the oracle's own pairs are resolved far below the compared tolerance
    assert np.max(res_ref[:100]) < 1e-9
    spec = synth.workload("heat2d_127")
    G = lrp.lrp_setup_problem(spec, precision=precision)
    lrp.lrp_autotune(G, 32)
    start = synth.normal_block(G.nx, 32, spec.seed)
    post, st = lrp.lrp_lowrank_posterior(G, k=100, block=32, eig_tol=EIG_TOL[precision], start=start)
    assert st["status"] == lrp.LRP_OK and st["k_converged"] == 100, st
    _check(post.eigs(), lam_ref[:100], TOL[precision], RESOLVABLE[precision])


@pytest.mark.parametrize("precision", [lrp.LRP_MIXED, lrp.LRP_FP64])
def test_heat3d_63_first_steps_spectrum(precision):
    lam_ref, res_ref = _golden_spectrum("spectrum_heat3d_63_nt20.txt")
    assert np.max(res_ref[:16]) < 1e-9
    spec = synth.workload("heat3d_63", nt=20, T=0.02)
    G = lrp.lrp_setup_problem(spec, precision=precision)
    post, st = lrp.lrp_lowrank_posterior(G, k=16, block=16, eig_tol=EIG_TOL[precision])
    assert st["status"] == lrp.LRP_OK and st["k_converged"] == 16, st
    _check(post.eigs(), lam_ref[:16], TOL[precision], RESOLVABLE[precision])


@pytest.mark.parametrize("precision", [lrp.LRP_MIXED, lrp.LRP_FP64])
def test_heat3d_63_full_apply_sampled(precision):
    rows, meta = _rows("apply_heat3d_63.txt")
    nodes = np.array([int(r[0]) for r in rows])
    want = np.array([float(r[1]) for r in rows])
    spec = synth.workload("heat3d_63")
    G = lrp.lrp_setup_problem(spec, precision=precision)
    x = synth.normal_block(G.nx, 1, 2027)
    assert np.array_equal(nodes, synth.query_nodes(G.nx, 256, 2028))
    H, st = lrp.lrp_hessian_apply(G, torch.from_numpy(x).cuda())
    assert st["status"] == lrp.LRP_OK, st
    got = H[:, 0].cpu().numpy()
    assert abs(np.max(np.abs(got)) - meta["max_abs"]) <= TOL[precision] * meta["max_abs"]
    assert np.max(np.abs(got[nodes] - want)) <= TOL[precision] * meta["max_abs"], st
