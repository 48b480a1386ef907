"""The convection-diffusion operator of the paper's Sec. 6.2 (upwind
differences; not symmetric): every implicit-Euler step solved by
Jacobi-preconditioned BiCGStab, the adjoint sweep with the transposed
operator. The forward map, the adjoint and the Hessian apply against the
oracle element by element (FP64 path, 1e-10), for two viscosities and
several team shapes; the leading eigenvalues above the paper's thresholds
against the dense eigensolver of the explicit Hessian."""
import numpy as np
import pytest

import synth
from oracle import spectrum as ospec
from oracle.problem import Problem as OProblem

lrp = pytest.importorskip("paper_1703_05638_gb300")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_05638_gb300 import build
    build.build()
    lrp.load()


def relerr(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(np.asarray(b))), 1e-300))


@pytest.mark.parametrize("nu", [1e-2, 1e-3])
@pytest.mark.parametrize("team", [dict(team_ctas=1, team_cols=1), dict(team_ctas=4, team_cols=1),
                                  dict(team_ctas=2, team_cols=2)])
def test_convdiff_sweeps_match_oracle(nu, team):
    spec = synth.paper_convdiff_spec(nu, nt=30)
    P = OProblem(spec)
    G = lrp.lrp_setup_problem(spec, precision=lrp.LRP_FP64, **team)
    U = synth.normal_block(P.nx, 3, 5)
    D, st = lrp.lrp_forward_observe(G, U)
    assert st["status"] == lrp.LRP_OK, st
    assert relerr(D, P.forward(U)) < 1e-10, st
    W = synth.normal_block(P.n_data, 3, 6)
    X, st = lrp.lrp_adjoint(G, W)
    assert relerr(X, P.adjoint(W)) < 1e-10, st
    H, st = lrp.lrp_hessian_apply(G, U)
    assert relerr(H, P.hessian_apply(U)) < 1e-10, st


@pytest.mark.parametrize("nu,eps", [(1e-2, 10.0), (1e-3, 10.0), (1e-2, 1.0)])
def test_convdiff_threshold_spectrum(nu, eps):
    """Eigenvalues of Htilde above the threshold epsilon (Sec. 6.2's
    thresholds 10 and 1) on the paper's setting (31^2 nodes, nt = 90,
    beta_noise = 1e4 beta_prior), against the dense eigensolver."""
    spec = synth.paper_convdiff_spec(nu)
    P = OProblem(spec)
    lam_ref, _ = ospec.eig_dense(P.hessian_explicit())
    n_above = int(np.sum(lam_ref >= eps))
    G = lrp.lrp_setup_problem(spec, precision=lrp.LRP_FP64)
    post, st = lrp.lrp_lowrank_posterior(G, k=600, block=4, eig_tol=1e-11, eig_threshold=eps)
    assert st["status"] == lrp.LRP_OK, st
    lam = post.eigs()
    if not np.any(np.abs(lam_ref - eps) <= 1e-9 * lam_ref[0]):
        assert len(lam) == n_above, (len(lam), n_above)
    m = min(len(lam), n_above)
    err = np.abs(lam[:m] - lam_ref[:m])
    assert np.max(err) <= 1e-10 * lam_ref[0]
    # relative error for the resolvable ones (lam >= 1e-6 lam_1, the FP64 reading)
    big = lam_ref[:m] >= 1e-6 * lam_ref[0]
    assert np.max(err[big] / lam_ref[:m][big]) <= 1e-10


def test_convdiff_setup_limits():
    spec = synth.paper_convdiff_spec(1e-2, nt=10)
    with pytest.raises(lrp.LrpError) as e:
        lrp.lrp_setup_problem(spec, precision=lrp.LRP_MIXED)
    assert e.value.status == lrp.LRP_EINVAL
    spec.kappa = synth.kappa_faces(spec.n, 2, 3)
    with pytest.raises(lrp.LrpError) as e:
        lrp.lrp_setup_problem(spec, precision=lrp.LRP_FP64)
    assert e.value.status == lrp.LRP_EINVAL
