"""The alternating low-rank space-time solver (Sec. 6.1, Eq. (st_pde),
(amen_1), (amen_2), (pre_1)) against the oracle (``oracle.als``):

* ``lrp_als_solve`` (space step by flexible GMRES with the block-diagonal
  preconditioner, time step by the projected recurrence) against
  ``als.als_solve`` / ``als.als_adjoint`` (space step by a dense
  Bartels-Stewart solve) from the same start, as the dense product W V^T and
  the residual after every sweep: heat 2D (initial condition as the source),
  3D with the kappa field (a rank-2 source), convection-diffusion forward
  and adjoint;
* the Hessian product with both solves by the alternating solver
  (``LRP_ALS_SOLVES``) against ``als.als_hessian_apply``, and against the
  exact (time-stepping) product within the solves' accuracy;
* Algorithm 1 (``lrp_arnoldi``) on that product: Ritz values above a
  threshold against the dense eigenvalues of the explicit Hessian;
* argument checks, a zero source and the residual stop.
"""
import numpy as np
import pytest

import synth
from oracle import als
from oracle import spectrum
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


def _spec(case):
    if case == "heat2d":
        return synth.small_spec(dim=2, n=15, nt=40, obs_every=4, n_obs=6, sigma=1e-2, alpha=0.05, seed=101)
    if case == "heat3d_kappa":
        return synth.small_spec(dim=3, n=7, nt=20, obs_every=2, n_obs=5, sigma=1e-2, alpha=0.05, seed=102,
                                with_kappa=True)
    if case == "convdiff":
        spec = synth.small_spec(dim=2, n=15, nt=40, obs_every=4, n_obs=6, sigma=1e-2, alpha=0.05, seed=103)
        spec.pde, spec.conv_nu, spec.wind = "convdiff", 1e-2, (0.0, 1.0, 0.0)
        return spec
    raise KeyError(case)


CASES = [
    # (case, precision, transpose, source rank, r, sweeps)
    ("heat2d", lrp.LRP_FP64, False, 1, 6, 4),
    ("heat2d", lrp.LRP_MIXED, False, 1, 6, 4),
    ("heat2d", lrp.LRP_FP64, True, 2, 6, 3),
    ("heat3d_kappa", lrp.LRP_FP64, False, 2, 5, 3),
    ("heat3d_kappa", lrp.LRP_MIXED, True, 2, 5, 3),
    ("convdiff", lrp.LRP_FP64, False, 1, 8, 4),
    ("convdiff", lrp.LRP_FP64, True, 2, 8, 3),
]


@pytest.mark.parametrize("case,precision,transpose,rf,r,sweeps", CASES)
def test_als_solve_matches_oracle(case, precision, transpose, rf, r, sweeps):
    """Same source, same random orthonormal start, same number of sweeps:
    the GPU's iterates follow the oracle's (the space step converged to
    max(10 solve_rtol, 1e-12) instead of solved exactly)."""
    spec = _spec(case)
    P = OProblem(spec)
    A = P.K.toarray()
    g = synth.rng(104)
    if rf == 1:
        Wf = synth.normal_block(P.nx, 1, 105)
        Vf = np.zeros((P.nt, 1))
        Vf[0, 0] = 1.0
    else:
        Wf = g.standard_normal((P.nx, rf))
        Vf = g.standard_normal((P.nt, rf))
    V0, _ = np.linalg.qr(g.standard_normal((P.nt, r)))
    if transpose:
        Wo, Vo, ro = als.als_adjoint(A, Wf, Vf, V0, sweeps)
    else:
        Wo, Vo, ro = als.als_solve(A, Wf, Vf, V0, sweeps)
    G = lrp.lrp_setup_problem(spec, precision=precision)
    W, V, res, st = lrp.lrp_als_solve(G, Wf, Vf, V0, sweeps, transpose=transpose)
    assert st["status"] == lrp.LRP_OK, (st, lrp.lrp_last_error())
    assert st["sweeps"] == sweeps
    assert np.max(np.abs(V.T @ V - np.eye(r))) < 1e-12
    assert relerr(W @ V.T, Wo @ Vo.T) < TOL[precision], (relerr(W @ V.T, Wo @ Vo.T), st)
    np.testing.assert_allclose(res, ro, rtol=1e-3, atol=10 * TOL[precision])
    G.close()


@pytest.mark.parametrize("precision", [lrp.LRP_FP64, lrp.LRP_MIXED])
@pytest.mark.parametrize("case", ["heat2d", "heat3d_kappa", "convdiff"])
def test_als_hessian_matches_oracle(case, precision):
    """Htilde x with both space-time solves by the alternating solver (rank
    8, 3 sweeps from e_1..e_8) against the oracle's same composition, and
    against the time-stepping product within the solves' final residuals."""
    if case == "convdiff" and precision == lrp.LRP_MIXED:
        pytest.skip("the convection-diffusion operator runs on the FP64 path")
    spec = _spec(case)
    P = OProblem(spec)
    A = P.K.toarray()
    r, sweeps = 8, 3
    X = synth.normal_block(P.nx, 2, 106)
    G = lrp.lrp_setup_problem(spec, precision=precision, als_rank=r, als_sweeps=sweeps)
    for misfit in (False, True):
        flags = lrp.LRP_ALS_SOLVES | (lrp.LRP_MISFIT_ONLY if misfit else 0)
        Y, st = lrp.lrp_hessian_apply(G, X, flags=flags)
        assert st["status"] == lrp.LRP_OK, (st, lrp.lrp_last_error())
        assert st["time_rank_max"] == r and st["adj_rank_max"] == r
        for j in range(X.shape[1]):
            want, info = als.als_hessian_apply(P, X[:, j], r, sweeps, A=A, misfit_only=misfit)
            assert relerr(Y[:, j], want) < TOL[precision], (j, misfit, relerr(Y[:, j], want), st)
            exact = P.misfit_apply(X[:, j]) if misfit else P.hessian_apply(X[:, j])
            bound = 100 * max(info["res_f"][-1], info["res_a"][-1]) + TOL[precision]
            assert relerr(Y[:, j], exact) < bound, (j, misfit, relerr(Y[:, j], exact), info)
    G.close()


def test_arnoldi_on_als_product():
    """Algorithm 1 with the alternating solves in every product (the paper's
    arrangement: Arnoldi outside, low-rank space-time solves inside) on a
    31^2 grid (nt = 60, 12 random sensors every 5th step: no symmetry, so
    no repeated eigenvalues) at rank 16: the 6 Ritz values above
    2e-5 lambda_1 (in the gap between lambda_6 = 5.8e-5 and lambda_7 =
    6.3e-6 lambda_1) match the dense eigenvalues of the explicit Htilde to
    1e-8 lambda_1, the product's error being ~2e-10."""
    spec = synth.small_spec(dim=2, n=31, nt=60, obs_every=5, n_obs=12, sigma=1e-2, alpha=0.05, seed=108)
    P = OProblem(spec)
    lam = spectrum.eig_dense(P.hessian_explicit())[0]
    eps = 2e-5 * lam[0]
    G = lrp.lrp_setup_problem(spec, precision=lrp.LRP_FP64, als_rank=16, als_sweeps=3)
    out = lrp.lrp_arnoldi(G, max_steps=60, eig_tol=1e-9, eig_threshold=eps, flags=lrp.LRP_ALS_SOLVES)
    st = out["stats"]
    assert st["status"] == lrp.LRP_OK, (st, lrp.lrp_last_error())
    th = np.sort(out["theta"].real)[::-1]
    want = lam[lam >= eps]
    got = th[th >= eps]
    assert got.size == want.size, (got, want)
    assert np.max(np.abs(got - want)) <= 1e-8 * lam[0], (got - want)
    G.close()


def test_als_argument_checks_and_degenerate_source():
    spec = _spec("heat2d")
    P = OProblem(spec)
    G = lrp.lrp_setup_problem(spec, precision=lrp.LRP_FP64)
    Wf = synth.normal_block(P.nx, 1, 107)
    Vf = np.zeros((P.nt, 1))
    Vf[0, 0] = 1.0
    for r in (65, P.nt + 1):
        V0 = np.zeros((P.nt, r))
        with pytest.raises(lrp.LrpError) as e:
            lrp.lrp_als_solve(G, Wf, Vf, V0, 2)
        assert e.value.status == lrp.LRP_EINVAL
    V0 = np.eye(P.nt)[:, :4]
    with pytest.raises(lrp.LrpError) as e:
        lrp.lrp_als_solve(G, Wf, Vf, V0, 0)
    assert e.value.status == lrp.LRP_EINVAL
    # a zero source: a zero solution, residual 0
    W, V, res, st = lrp.lrp_als_solve(G, np.zeros((P.nx, 1)), Vf, V0, 2)
    assert st["status"] == lrp.LRP_OK and np.all(W == 0.0)
    # the residual stop: rank 8 from e_1..e_8 reaches 1.0e-7 after one sweep
    # and 3.1e-8 after the second (the oracle's history); stop at 5e-8
    V0 = np.eye(P.nt)[:, :8]
    W, V, res, st = lrp.lrp_als_solve(G, Wf, Vf, V0, 8, tol=5e-8)
    assert st["sweeps"] == 2 and res[-1] <= 5e-8, (res, st)
    assert np.all(res[:-1] > 5e-8)
    G.close()


def test_als_hessian_many_columns_equal_single_column_calls():
    """A block of 11 columns is solved as one batch (one preconditioner
    launch per GMRES iteration for all of them, a Hessenberg matrix per
    column); every column equals the same column applied alone to the
    solves' accuracy. The batch keeps iterating a column's GMRES until every
    column has converged, so a column can take more iterations than alone:
    the difference is of the order of the space step's GMRES tolerance
    propagated through the sweeps (~1e-11 relative), hence 1e-9 here; the
    comparisons with the oracle keep 1e-10."""
    spec = _spec("heat2d")
    P = OProblem(spec)
    X = synth.normal_block(P.nx, 11, 113)
    G = lrp.lrp_setup_problem(spec, precision=lrp.LRP_FP64, als_rank=8, als_sweeps=3)
    Y, st = lrp.lrp_hessian_apply(G, X, flags=lrp.LRP_ALS_SOLVES)
    assert st["status"] == lrp.LRP_OK, (st, lrp.lrp_last_error())
    for j in (0, 5, 8, 10):
        y1, st1 = lrp.lrp_hessian_apply(G, X[:, j:j + 1], flags=lrp.LRP_ALS_SOLVES)
        assert st1["status"] == lrp.LRP_OK
        assert relerr(Y[:, j], y1[:, 0]) < 1e-9, (j, relerr(Y[:, j], y1[:, 0]))
    G.close()
