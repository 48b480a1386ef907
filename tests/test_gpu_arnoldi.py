"""The Arnoldi path of Sec. 4 Algorithm 1 against the oracle:

* the Hessenberg eigensolver (Francis double-shift QR) against the library
  eigensolver of NumPy on random, nearly symmetric and graded Hessenberg
  matrices, with the Schur factorisation H = Z T Z^T checked;
* the truncated product (LRP_LOWRANK_SOURCE: state and adjoint trajectories
  in low-rank-in-time form, the adjoint's data observed from the truncated
  state) element by element against ``oracle.lowrank.lowrank_hessian_apply``
  with the same chunking and tolerance, in both paths, for the heat and the
  convection-diffusion operator; without truncation it is the exact apply;
* Arnoldi on the exact operator: its Hessenberg matrix against the oracle's
  Algorithm 1 from the same start vector, the eigenvalues above a threshold
  against the dense eigensolver, and a posterior built from it against the
  oracle's low-rank formulas;
* Arnoldi on the truncated product (the paper's setting of Sec. 6.2 with
  nt = 30, so that the oracle's Arnoldi finishes in seconds): Ritz values
  above the threshold against the oracle's Arnoldi on its truncated product
  and against the exact eigenvalues, the Hessenberg matrix's asymmetry of the
  order of the truncation tolerance, the trajectory ranks per step.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import synth
from oracle import lowrank as olr
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


def _match_multiset(got, want):
    """Largest distance after pairing each wanted eigenvalue with the nearest
    unused computed one (both complex arrays of the same length)."""
    got = list(got)
    worst = 0.0
    for w in want:
        j = int(np.argmin([abs(g - w) for g in got]))
        worst = max(worst, abs(got[j] - w))
        got.pop(j)
    return worst


@pytest.mark.parametrize("m", [1, 2, 3, 17, 64, 150, 300])
@pytest.mark.parametrize("kind", ["random", "near_symmetric", "graded"])
def test_hessenberg_eig_matches_numpy(m, kind):
    r = synth.rng(100 + m)
    if kind == "random":
        A = r.standard_normal((m, m))
        tol = 1e-8  # nonnormal: eigenvalue condition numbers well above 1
    elif kind == "near_symmetric":
        A = r.standard_normal((m, m))
        A = A + A.T + 1e-7 * r.standard_normal((m, m))
        tol = 1e-11
    else:
        Q, _ = np.linalg.qr(r.standard_normal((m, m)))
        A = (Q * 10.0 ** -np.linspace(0, 12, m)) @ Q.T
        tol = 1e-12
    H = sla.hessenberg(A)
    lam, T, Z = lrp.lrp_hessenberg_eig(H, want_schur=True)
    ref = np.linalg.eigvals(H)
    scale = max(1.0, np.abs(ref).max()) if kind == "random" else np.abs(ref).max()
    assert _match_multiset(lam, ref) <= tol * scale
    assert np.max(np.abs(Z @ T @ Z.T - H)) <= 1e-12 * np.abs(H).max() * max(1, m / 50)
    assert np.max(np.abs(Z.T @ Z - np.eye(m))) <= 1e-12 * max(1, m / 50)
    assert np.all(np.tril(T, -2) == 0)
    # complex pairs sit in 2x2 blocks, in conjugate order
    for i in range(m):
        if lam[i].imag > 0:
            assert lam[i + 1] == np.conj(lam[i]) and T[i + 1, i] != 0


def _heat_spec():
    return synth.small_spec(dim=2, n=15, nt=40, obs_every=2, n_obs=12, sigma=1e-2, alpha=0.05, seed=81)


def _convdiff_spec(nt=30):
    return synth.paper_convdiff_spec(1e-2, nt=nt)


@pytest.mark.parametrize("precision", [lrp.LRP_FP64, lrp.LRP_MIXED])
@pytest.mark.parametrize("pde", ["heat", "convdiff"])
def test_lowrank_source_apply_matches_oracle(precision, pde):
    if pde == "convdiff" and precision == lrp.LRP_MIXED:
        pytest.skip("the convection-diffusion operator runs on the FP64 path")
    spec = _convdiff_spec() if pde == "convdiff" else _heat_spec()
    P = OProblem(spec)
    tol, rmax, s = 1e-6, 40, 8
    G = lrp.lrp_setup_problem(spec, precision=precision, time_trunc_tol=tol, time_rank_max=rmax, time_chunk=s)
    X = synth.normal_block(P.nx, 2, 82)
    Y, st = lrp.lrp_hessian_apply(G, X, lrp.LRP_LOWRANK_SOURCE)
    assert st["status"] == lrp.LRP_OK, st
    for j in range(2):
        want, info = olr.lowrank_hessian_apply(P, X[:, j], tol, rmax, s)
        assert relerr(Y[:, j], want) < TOL[precision], (j, st, info)
    assert st["time_rank_max"] == max(olr.lowrank_hessian_apply(P, X[:, j], tol, rmax, s)[1]["rank_y"]
                                      for j in range(2))
    assert 0 < st["adj_rank_max"] <= rmax and st["time_trunc_err"] <= tol and st["adj_trunc_err"] <= tol
    # H_mis form
    Ym, st = lrp.lrp_hessian_apply(G, X[:, :1], lrp.LRP_LOWRANK_SOURCE | lrp.LRP_MISFIT_ONLY)
    want, _ = olr.lowrank_hessian_apply(P, X[:, 0], tol, rmax, s, misfit_only=True)
    assert relerr(Ym[:, 0], want) < TOL[precision], st


@pytest.mark.parametrize("precision", [lrp.LRP_FP64, lrp.LRP_MIXED])
def test_lowrank_source_without_truncation_is_exact(precision):
    """time_trunc_tol = 1e-15 and a rank cap above nt: nothing of
    significance is discarded and the truncated product is the exact Hessian
    apply."""
    spec = synth.small_spec(dim=2, n=15, nt=12, obs_every=3, n_obs=8, sigma=1e-2, seed=83)
    P = OProblem(spec)
    G = lrp.lrp_setup_problem(spec, precision=precision, time_trunc_tol=1e-15, time_rank_max=16, time_chunk=5)
    X = synth.normal_block(P.nx, 3, 84)
    Y, st = lrp.lrp_hessian_apply(G, X, lrp.LRP_LOWRANK_SOURCE)
    assert relerr(Y, P.hessian_apply(X)) < TOL[precision], st


def test_lowrank_source_rejects_keep_traj():
    G = lrp.lrp_setup_problem(_heat_spec())
    with pytest.raises(lrp.LrpError) as e:
        lrp.lrp_hessian_apply(G, np.zeros((G.nx, 1)), lrp.LRP_LOWRANK_SOURCE | lrp.LRP_KEEP_TRAJ_FACTORS)
    assert e.value.status == lrp.LRP_EINVAL


def test_arnoldi_exact_operator_matches_oracle():
    """Algorithm 1 on the exact Htilde (FP64): the Hessenberg matrix of the
    first steps equals the oracle's from the same start vector, the Ritz
    values above the threshold are the dense eigenvalues above it, every one
    is real, and the posterior from the Ritz pairs answers queries like the
    oracle's low-rank formulas with the dense eigenpairs."""
    spec = _heat_spec()
    P = OProblem(spec)
    G = lrp.lrp_setup_problem(spec, precision=lrp.LRP_FP64)
    lam, V = ospec.eig_dense(P.hessian_explicit())
    eps = 0.5 * (lam[9] + lam[10])
    v1 = synth.normal_block(P.nx, 1, 85)[:, 0]
    res = lrp.lrp_arnoldi(G, 120, eig_tol=1e-11, eig_threshold=eps, start=v1, posterior=True)
    st = res["stats"]
    assert st["status"] == lrp.LRP_OK and st["k_converged"] == 10, st
    theta = res["theta"]
    above = theta.real >= eps
    assert int(np.sum(above)) == 10
    assert np.max(np.abs(theta.real[above] - lam[:10])) <= 1e-10 * lam[0]
    # H of a symmetric operator is symmetric up to the orthogonality that
    # single modified Gram-Schmidt loses as Ritz values converge (rounding
    # amplified by the spectrum's range; the oracle's Algorithm 1 loses the
    # same, ~1e-7 in V^T V here)
    assert st["n_complex"] == 0 and st["hess_asym"] < 1e-7
    _, Ho = ospec.arnoldi_mgs(P.hessian_apply, v1, 8)
    assert np.max(np.abs(res["H"][:9, :8] - Ho)) <= 1e-9 * lam[0]
    post = res["posterior"]
    lam_p, Vp = post.eigs(vectors=True)
    assert np.max(np.abs(lam_p - lam[:10])) <= 1e-10 * lam[0]
    assert np.max(np.abs(Vp.T @ Vp - np.eye(10))) < 1e-12
    # a Ritz vector is accurate to its residual over the gap to the rest of
    # the spectrum (here ~1e-11 lam_1 / 4e-5 lam_1): the queries to 1e-7
    nodes = synth.query_nodes(P.nx, 30, 86)
    y = synth.normal_block(P.n_data, 1, 87)[:, 0]
    out = lrp.lrp_posterior_query(post, lrp.LRP_Q_MEAN | lrp.LRP_Q_VARIANCE, y_obs=y, points=nodes)
    assert relerr(out["variance"], opost.variance_lowrank(P, lam[:10], V[:, :10], nodes)) < 1e-7
    assert relerr(out["mean"], opost.mean_lowrank(P, lam[:10], V[:, :10], y)) < 1e-7


@pytest.mark.parametrize("precision", [lrp.LRP_FP64, lrp.LRP_MIXED])
def test_arnoldi_k_leading_stop(precision):
    """Without a threshold the run stops once the k leading Ritz values meet
    the residual test; they are the k leading eigenvalues."""
    spec = _heat_spec()
    P = OProblem(spec)
    G = lrp.lrp_setup_problem(spec, precision=precision)
    lam, _ = ospec.eig_dense(P.hessian_explicit())
    res = lrp.lrp_arnoldi(G, 100, k=6, eig_tol=TOL[precision] / 10)
    st = res["stats"]
    assert st["status"] == lrp.LRP_OK and st["k_converged"] == 6, st
    assert np.max(np.abs(res["theta"].real[:6] - lam[:6])) <= TOL[precision] * lam[0]


def test_arnoldi_lowrank_source_convdiff_matches_oracle():
    """Sec. 6.2's setting (31^2 nodes, nu = 1e-2, threshold epsilon = 1) with
    nt = 30 so that the oracle's Arnoldi finishes in seconds: Algorithm 1 with the truncated product (eps_0 = 1e-8, the
    paper's truncation threshold). The Ritz values above epsilon agree with
    the oracle's Arnoldi on its own truncated product and with the exact
    eigenvalues to the residual tolerance plus the truncation's effect; they
    stay real; H is not symmetric, but only at the level of the truncation;
    the ranks per step stay below the cap."""
    spec = _convdiff_spec()
    P = OProblem(spec)
    tol0, rmax, s = 1e-8, 40, 16
    G = lrp.lrp_setup_problem(spec, precision=lrp.LRP_FP64, time_trunc_tol=tol0, time_rank_max=rmax,
                              time_chunk=s)
    lam, _ = ospec.eig_dense(P.hessian_explicit())
    eps, eig_tol = 1.0, 1e-9
    v1 = synth.normal_block(P.nx, 1, 88)[:, 0]
    res = lrp.lrp_arnoldi(G, 150, eig_tol=eig_tol, eig_threshold=eps, flags=lrp.LRP_LOWRANK_SOURCE, start=v1)
    st = res["stats"]
    assert st["status"] == lrp.LRP_OK, st
    theta = res["theta"]
    n_above = int(np.sum(lam >= eps))
    assert 10 <= n_above < 120
    above = theta.real >= eps
    assert int(np.sum(above)) == n_above
    assert st["n_complex"] == 0 or st["max_imag"] < 1e-7
    assert np.max(np.abs(theta.real[above] - lam[:n_above])) <= (eig_tol + 100 * tol0) * lam[0]
    assert 0.0 < st["hess_asym"] < 1e-5
    assert 0 < st["time_rank_max"] <= rmax and 0 < st["adj_rank_max"] <= rmax
    assert np.all(res["ranks_y"] > 0) and np.all(res["ranks_y"] <= rmax)
    m, _, _, th_o, _ = olr.arnoldi_threshold(lambda x: olr.lowrank_hessian_apply(P, x, tol0, rmax, s)[0], v1,
                                             eps, eig_tol, 150)
    ab_o = th_o.real >= eps
    assert int(np.sum(ab_o)) == n_above
    assert np.max(np.abs(theta.real[above] - th_o.real[ab_o])) <= 2 * eig_tol * lam[0] + 1e-12 * lam[0]
