"""The heat experiment of the paper's numerical section (Sec. 6.1) on finite
differences: 63^2 interior nodes, nt = 30, 9 sensor patches of 1/256 of the
domain, Gamma_prior = 10 I, beta_noise = 10^6 beta_prior, eigenvalues kept
above the threshold epsilon = 1. The GPU's eigenvalues above the threshold
(Lanczos with the threshold stop) against the oracle's (ARPACK on the
matrix-free oracle), in both paths; and the identity prior's Hessian apply
and posterior queries element by element on a small problem."""
import numpy as np
import pytest

import synth
from oracle import posterior as opost
from oracle import spectrum as ospec
from oracle.problem import Problem as OProblem

lrp = pytest.importorskip("paper_1703_05638_gb300")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = {lrp.LRP_FP64: 1e-10, lrp.LRP_MIXED: 1e-6}


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_05638_gb300 import build
    build.build()
    lrp.load()


def relerr(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(np.asarray(b))), 1e-300))


@pytest.mark.parametrize("precision", [lrp.LRP_FP64, lrp.LRP_MIXED])
def test_identity_prior_apply_and_queries(precision):
    spec = synth.small_spec(dim=2, n=31, nt=20, obs_every=2, n_obs=12, sigma=0.05, seed=33)
    spec.prior_kind, spec.prior_gamma = lrp.LRP_PRIOR_IDENTITY, 10.0
    P = OProblem(spec)
    G = lrp.lrp_setup_problem(spec, precision=precision)
    X = synth.normal_block(P.nx, 3, 4)
    H, st = lrp.lrp_hessian_apply(G, X)
    assert relerr(H, P.hessian_apply(X)) < TOL[precision], st
    Z, _ = lrp.lrp_prior_half(G, X)
    # FP64 path: one FP64 product; mixed path (band kernel): a double-float
    # product, about 48 bits
    assert relerr(Z, np.sqrt(10.0) * X) < (1e-15 if precision == lrp.LRP_FP64 else 2e-14)
    lam_ref, V_ref = ospec.eig_dense(P.hessian_explicit())
    k = int(np.argmax(lam_ref[4:20] / lam_ref[5:21])) + 5  # at a spectral gap
    post, st = lrp.lrp_lowrank_posterior(G, k=k, block=4, eig_tol=TOL[precision] / 10)
    lam = post.eigs()
    assert np.max(np.abs(lam - lam_ref[:k])) <= TOL[precision] * lam_ref[0]
    y = synth.normal_block(P.n_data, 1, 5)[:, 0]
    nodes = synth.query_nodes(P.nx, 40, 6)
    xi = synth.normal_block(P.nx, 2, 7)
    out = lrp.lrp_posterior_query(post, lrp.LRP_Q_MEAN | lrp.LRP_Q_VARIANCE | lrp.LRP_Q_SAMPLES, y_obs=y,
                                  points=nodes, xi=xi)
    m_ref = opost.mean_lowrank(P, lam_ref[:k], V_ref[:, :k], y)
    assert relerr(out["mean"], m_ref) < TOL[precision]
    assert relerr(out["variance"], opost.variance_lowrank(P, lam_ref[:k], V_ref[:, :k], nodes)) < TOL[precision]
    assert relerr(out["samples"], opost.samples_lowrank(P, lam_ref[:k], V_ref[:, :k], m_ref, xi)) < TOL[precision]


@pytest.mark.parametrize("precision", [lrp.LRP_FP64, lrp.LRP_MIXED])
def test_paper_heat_threshold_spectrum(precision):
    spec = synth.paper_heat_spec(1e6)
    P = OProblem(spec)
    lam_ref, _ = ospec.eigsh_top(P.hessian_apply, P.nx, 48, tol=1e-12)
    eps = 1.0
    n_above = int(np.sum(lam_ref >= eps))
    assert 10 < n_above < 45
    G = lrp.lrp_setup_problem(spec, precision=precision)
    post, st = lrp.lrp_lowrank_posterior(G, k=400, block=1, eig_tol=TOL[precision] / 10, eig_threshold=eps)
    assert st["status"] == lrp.LRP_OK, st
    lam = post.eigs()
    # the count above the threshold, unless an eigenvalue sits within the
    # tolerance of it
    if not np.any(np.abs(lam_ref - eps) <= 10 * TOL[precision] * lam_ref[0]):
        assert len(lam) == n_above, (len(lam), n_above, st)
    m = min(len(lam), n_above)
    err = np.abs(lam[:m] - lam_ref[:m])
    assert np.max(err) <= TOL[precision] * lam_ref[0]
    # relative error for the resolvable ones (lam >= 1e-6 lam_1 FP64, 1e-3 lam_1 mixed)
    big = lam_ref[:m] >= (1e-6 if precision == lrp.LRP_FP64 else 1e-3) * lam_ref[0]
    assert np.max(err[big] / lam_ref[:m][big]) <= TOL[precision]
