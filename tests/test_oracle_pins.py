"""Pins of the FP64 oracle against closed forms, invariants, brute force and
hand-worked values (no GPU). Each test names the passage it instantiates and
the mistake it would catch."""
import math
import os
from fractions import Fraction
from types import SimpleNamespace

import numpy as np
import pytest

import synth
from oracle import als, lowrank, operators, observe, posterior, spacetime, spectrum, timefactors
from oracle.problem import Problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _spec(**kw):
    base = dict(dim=2, n=7, nt=12, T=1.0, prior_alpha=0.1, sigma=0.05, obs_every=3,
                sensors=synth.uniform_sensors(5, 2, 3), kappa=None)
    base.update(kw)
    return SimpleNamespace(**base)


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------- operators
@pytest.mark.parametrize("dim,n,modes", [(1, 15, (3,)), (2, 7, (1, 2)), (2, 15, (4, 1)),
                                          (3, 7, (2, 1, 3))])
def test_laplacian_sine_modes(dim, n, modes):
    """Sec. 5: sine modes are eigenfunctions of the Dirichlet Laplacian; the
    discrete eigenvalue is sum (4/h^2) sin^2(m pi h/2). Catches a wrong h
    scaling, a missing boundary term or a wrong neighbour index."""
    L = operators.laplacian(n, dim)
    phi = operators.sine_mode(n, dim, modes)
    mu = operators.sine_eigenvalue(n, modes)
    np.testing.assert_allclose(L @ phi, mu * phi, rtol=0, atol=1e-10 * mu)


def test_laplacian_golden_1d():
    rows = _read_golden("laplace1d_n3.txt")
    L = operators.laplacian(3, 1).toarray()
    lam = np.sort(np.linalg.eigvalsh(L))
    want = np.array([float(r[1]) for r in rows])
    np.testing.assert_allclose(lam, want, rtol=1e-14)


def test_laplacian_flux_form_faces():
    """Variable kappa (flux form): for u = x-coordinate at an interior node,
    (L u)_p = (kappa_west - kappa_east)/h exactly. Catches swapped faces, a
    sign error or faces read along the wrong axis."""
    n, dim = 9, 2
    kap = synth.kappa_faces(n, dim, seed=5)
    L = operators.laplacian(n, dim, kap)
    h = 1.0 / (n + 1)
    x = np.tile((np.arange(n) + 1.0) * h, n)          # first coordinate fastest
    y = np.repeat((np.arange(n) + 1.0) * h, n)
    kx, ky = kap
    Lx, Ly = L @ x, L @ y
    for (i, j) in [(3, 4), (1, 1), (5, 7)]:
        p = i + n * j
        assert abs(Lx[p] - (kx[j, i] - kx[j, i + 1]) / h) < 1e-9
        assert abs(Ly[p] - (ky[j, i] - ky[j + 1, i]) / h) < 1e-9
    assert abs(L - L.T).max() < 1e-12


def test_laplacian_constant_kappa_scales():
    n, dim = 5, 3
    kap = [np.full(s.shape, 2.5) for s in synth.kappa_faces(n, dim, seed=1)]
    L = operators.laplacian(n, dim, kap)
    L0 = operators.laplacian(n, dim)
    assert abs(L - 2.5 * L0).max() < 1e-9


def test_kappa_field_statistics():
    """Input recipe check: log(kappa) has mean ~0 and std ~0.5."""
    kap = synth.kappa_faces(31, 2, seed=11)
    g = np.log(np.concatenate([k.ravel() for k in kap]))
    assert abs(g.mean()) < 0.5
    assert 0.2 < g.std() < 0.9


# ---------------------------------------------------------------- time stepping
@pytest.mark.parametrize("dim,n,modes", [(1, 31, (2,)), (2, 7, (2, 3)), (3, 7, (1, 1, 2))])
def test_modal_decay(dim, n, modes):
    """Implicit Euler on a sine mode: y_n = (1 + tau mu)^{-n} phi exactly.
    Catches an explicit-Euler step, an off-by-one step count or a wrong tau."""
    P = Problem(_spec(dim=dim, n=n, nt=9, sensors=synth.uniform_sensors(3, dim, 1)))
    phi = operators.sine_mode(n, dim, modes)
    mu = operators.sine_eigenvalue(n, modes)
    Y = P.trajectory(phi)
    for k in range(P.nt):
        np.testing.assert_allclose(Y[:, k], (1 + P.tau * mu) ** -(k + 1) * phi,
                                   rtol=1e-12, atol=1e-14)


def test_heat_1d_continuum_decay():
    """1D heat equation u_t = u_xx, u(0)=sin(pi x): the exact solution decays
    as exp(-pi^2 t). The implicit-Euler/FD error is O(tau + h^2): halving tau
    (h fixed and small) must roughly halve the error."""
    errs = []
    for nt in (200, 400, 800):
        P = Problem(_spec(dim=1, n=255, nt=nt, sensors=synth.uniform_sensors(2, 1, 1)))
        phi = operators.sine_mode(255, 1, (1,))
        y = P.trajectory(phi)[:, -1]
        errs.append(np.max(np.abs(y - math.exp(-math.pi ** 2) * phi)))
    assert errs[0] < 5e-4
    assert 1.8 < errs[0] / errs[1] < 2.2 and 1.8 < errs[1] / errs[2] < 2.2


# ---------------------------------------------------------------- observation
def test_lattice_sensors_select_nodes():
    """The tiny workload's 7x7 lattice (i/8, j/8) on the 31-grid hits nodes
    (4i-1, 4j-1) exactly: B is a 0/1 selection."""
    B = observe.observation_matrix(31, 2, synth.lattice_sensors(7, 2)).toarray()
    assert B.shape == (49, 961)
    for s in range(49):
        i, j = s % 7 + 1, s // 7 + 1
        row = np.zeros(961)
        row[(4 * i - 1) + 31 * (4 * j - 1)] = 1.0
        np.testing.assert_array_equal(B[s], row)


@pytest.mark.parametrize("dim", [2, 3])
def test_interpolation_reproduces_multilinear(dim):
    """Bilinear/trilinear interpolation reproduces f = prod_a x_a exactly
    (it vanishes on the faces x_a = 0, so cells touching those faces count
    too); weights of interior cells sum to 1."""
    n = 9
    h = 1.0 / (n + 1)
    r = synth.rng(3)
    pts = r.uniform(0.0, 0.6, size=(40, dim))
    B = observe.observation_matrix(n, dim, pts)
    coords = np.meshgrid(*[(np.arange(n) + 1.0) * h] * dim, indexing="ij")
    f_nodes = np.ones([n] * dim)
    for c in coords:
        f_nodes = f_nodes * c
    f_nodes = f_nodes.transpose(tuple(range(dim))[::-1]).ravel()   # first coord fastest
    np.testing.assert_allclose(B @ f_nodes, np.prod(pts, axis=1), rtol=1e-12, atol=1e-15)
    inner = np.all((pts > h) & (pts < 1 - h), axis=1)
    np.testing.assert_allclose(np.asarray(B.sum(axis=1)).ravel()[inner], 1.0, rtol=1e-14)


# ---------------------------------------------------------------- forward / adjoint
@pytest.mark.parametrize("dim,kappa", [(2, False), (3, True)])
def test_adjoint_identity(dim, kappa):
    """<F u, w> = <u, F^T w> to 1e-12: F (forward stepping) and F^T (backward
    recursion) are written independently."""
    n = 7 if dim == 2 else 5
    spec = _spec(dim=dim, n=n, nt=10, obs_every=2, sensors=synth.uniform_sensors(6, dim, 2),
                 kappa=synth.kappa_faces(n, dim, 4) if kappa else None)
    P = Problem(spec)
    r = synth.rng(9)
    u = r.standard_normal((P.nx, 3))
    w = r.standard_normal((P.n_data, 3))
    lhs = np.sum(P.forward(u) * w, axis=0)
    rhs = np.sum(u * P.adjoint(w), axis=0)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_forward_brute_force(dim):
    """F from dense matrix powers B (I + tau L)^{-n} on an n=3 grid."""
    spec = _spec(dim=dim, n=3, nt=6, obs_every=2, sensors=synth.uniform_sensors(4, dim, 6),
                 kappa=synth.kappa_faces(3, dim, 8))
    P = Problem(spec)
    L = operators.laplacian(3, dim, spec.kappa).toarray()
    Sinv = np.linalg.inv(np.eye(P.nx) + P.tau * L)
    B = observe.observation_matrix(3, dim, spec.sensors).toarray()
    rows = [B @ np.linalg.matrix_power(Sinv, s) for s in (2, 4, 6)]
    np.testing.assert_allclose(P.forward_explicit(), np.vstack(rows), rtol=1e-12, atol=1e-15)


def test_hessian_matrix_free_symmetric():
    """Htilde applied column by column (matrix-free path) is symmetric to 1e-12."""
    P = Problem(_spec(n=5, nt=8, obs_every=2, sensors=synth.uniform_sensors(4, 2, 12)))
    H = P.hessian_apply(np.eye(P.nx))
    assert np.max(np.abs(H - H.T)) <= 1e-12 * np.max(np.abs(H))


def test_hessian_modal_closed_form():
    """Full observation (a sensor on every node, every step) and constant
    kappa: a sine mode is an exact eigenvector of Htilde with eigenvalue
    (1+alpha mu)^-2 sigma^-2 sum_n (1+tau mu)^-2n (discrete analogue of the
    Sec. 5 modal analysis). Catches a missing prior factor, sigma^-1 instead
    of sigma^-2, or a mis-indexed observed step."""
    n = 7
    spec = _spec(n=n, nt=10, obs_every=1, sensors=synth.lattice_sensors(n, 2),
                 sigma=0.3, prior_alpha=0.02)
    P = Problem(spec)
    assert np.allclose(P.B.toarray(), np.eye(P.nx))
    for modes in [(1, 1), (2, 3), (5, 2)]:
        phi = operators.sine_mode(n, 2, modes)
        mu = operators.sine_eigenvalue(n, modes)
        lam = (1 + P.alpha * mu) ** -2 / P.sigma ** 2 * sum(
            (1 + P.tau * mu) ** (-2 * k) for k in range(1, P.nt + 1))
        np.testing.assert_allclose(P.hessian_apply(phi), lam * phi, rtol=1e-11, atol=1e-14)


def test_identity_prior_modal_closed_form():
    """The prior of the experiments of Sec. 6.1, Gamma_prior = gamma I: with
    full observation a sine mode is an eigenvector of Htilde with eigenvalue
    gamma sigma^-2 sum_n (1+tau mu)^-2n; the exact posterior covariance is
    (H_mis + I/gamma)^-1 and the prior variance is gamma at every node.
    Catches sqrt(gamma) applied once instead of twice, or 1/gamma in place of
    gamma."""
    n = 7
    spec = _spec(n=n, nt=10, obs_every=1, sensors=synth.lattice_sensors(n, 2), sigma=0.3,
                 prior_kind=1, prior_gamma=10.0)
    P = Problem(spec)
    for modes in [(1, 1), (2, 3), (5, 2)]:
        phi = operators.sine_mode(n, 2, modes)
        mu = operators.sine_eigenvalue(n, modes)
        lam = 10.0 / P.sigma ** 2 * sum((1 + P.tau * mu) ** (-2 * k) for k in range(1, P.nt + 1))
        np.testing.assert_allclose(P.hessian_apply(phi), lam * phi, rtol=1e-11, atol=1e-14)
    Hm = P.misfit_explicit()
    want = np.linalg.inv(Hm + np.eye(P.nx) / 10.0)
    np.testing.assert_allclose(posterior.post_cov_exact(P), want, rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(posterior.prior_diag(P, np.arange(P.nx)), 10.0, rtol=1e-15)
    lam, V = spectrum.eig_dense(P.hessian_explicit())
    G_lr = posterior.post_cov_lowrank(P, lam, V)
    assert np.max(np.abs(G_lr - want)) <= 1e-10 * np.max(np.abs(want))


def test_one_node_golden():
    rows = {r[0]: Fraction(r[1]) for r in _read_golden("one_node_problem.txt")}
    spec = _spec(n=1, nt=2, prior_alpha=1 / 16, sigma=1.0, obs_every=1,
                 sensors=np.array([[0.5, 0.5]]))
    P = Problem(spec)
    assert abs(P.misfit_explicit()[0, 0] - float(rows["H_mis"])) < 1e-16
    assert abs(P.hessian_explicit()[0, 0] - float(rows["Htilde"])) < 1e-16
    assert abs(posterior.post_cov_exact(P)[0, 0] - float(rows["Gamma_post"])) < 1e-15
    m = posterior.mean_exact(P, np.array([1.0, 1.0]))
    assert abs(m[0] - float(rows["mean"])) < 1e-15


# ---------------------------------------------------------------- spectrum
def test_sigma_rescaling():
    """Gamma_noise = sigma^2 I: eigenvalues scale as 1/sigma^2."""
    s1 = _spec(n=5, nt=6, obs_every=2, sigma=1.0, sensors=synth.uniform_sensors(4, 2, 1))
    s2 = _spec(n=5, nt=6, obs_every=2, sigma=0.01, sensors=synth.uniform_sensors(4, 2, 1))
    l1, _ = spectrum.eig_dense(Problem(s1).hessian_explicit())
    l2, _ = spectrum.eig_dense(Problem(s2).hessian_explicit())
    np.testing.assert_allclose(l2, l1 / 0.01 ** 2, rtol=1e-9, atol=1e-9 * l2[0])


def test_arnoldi_matches_dense():
    """Algorithm 1 (Arnoldi + MGS) recovers the leading eigenvalues of the
    explicit Htilde (the check of Sec. 6.1 against a dense eigensolver)."""
    P = Problem(_spec(n=7, nt=12, obs_every=3, sensors=synth.uniform_sensors(6, 2, 5)))
    lam, _ = spectrum.eig_dense(P.hessian_explicit())
    v1 = synth.normal_block(P.nx, 1, 3)[:, 0]
    V, H = spectrum.arnoldi_mgs(P.hessian_apply, v1, 30)
    ritz, Y = spectrum.ritz_from_arnoldi(V, H, 5)
    np.testing.assert_allclose(ritz, lam[:5], rtol=1e-10)
    for i in range(3):
        r = P.hessian_apply(Y[:, i]) - ritz[i] * Y[:, i]
        assert np.linalg.norm(r) < 1e-8 * lam[0]


def test_eigsh_top_matches_dense():
    """The matrix-free ARPACK cross-check returns the leading eigenpairs of the
    explicit Htilde (the check of Sec. 6.1 against a dense eigensolver):
    eigenvalues to 1e-10 lam_1, eigenvectors of simple eigenvalues up to sign.
    Catches a wrong ordering, the wrong end of the spectrum or a reshaped
    operand."""
    P = Problem(_spec(n=7, nt=12, obs_every=3, sensors=synth.uniform_sensors(6, 2, 5)))
    lam, V = spectrum.eig_dense(P.hessian_explicit())
    got, W = spectrum.eigsh_top(P.hessian_apply, P.nx, 6, tol=1e-13)
    assert np.all(np.diff(got) <= 0)
    assert np.max(np.abs(got - lam[:6])) <= 1e-10 * lam[0]
    for i in range(6):
        if min(abs(lam[i] - lam[j]) for j in range(7) if j != i) > 1e-6 * lam[0]:
            assert abs(abs(W[:, i] @ V[:, i]) - 1.0) < 1e-8


# ---------------------------------------------------------------- posterior
def _tiny_problem():
    return Problem(_spec(n=5, nt=8, obs_every=2, sensors=synth.uniform_sensors(5, 2, 21),
                         sigma=0.02, prior_alpha=0.05))


def test_smw_full_rank_equals_exact():
    """With all nx eigenpairs the low-rank form equals the exact inverse
    (Sherman-Morrison-Woodbury, Sec. 2)."""
    P = _tiny_problem()
    lam, V = spectrum.eig_dense(P.hessian_explicit())
    G_lr = posterior.post_cov_lowrank(P, lam, V)
    G_ex = posterior.post_cov_exact(P)
    assert np.max(np.abs(G_lr - G_ex)) <= 1e-10 * np.max(np.abs(G_ex))
    Ht = P.hessian_explicit()
    np.testing.assert_allclose(posterior.smw_inner(lam, V), np.linalg.inv(np.eye(P.nx) + Ht),
                               rtol=1e-9, atol=1e-12)


def test_mean_is_map_point():
    """The exact mean zeroes the gradient of the MAP objective
    1/2 u^T Gamma_prior^{-1} u + 1/2 |y - F u|^2 / sigma^2 (Sec. 2), and the
    full-rank low-rank mean equals it."""
    P = _tiny_problem()
    y = synth.normal_block(P.n_data, 1, 4)[:, 0]
    m = posterior.mean_exact(P, y)
    R = P.R.toarray()
    grad = R @ (R @ m) - P.adjoint(y - P.forward(m)) / P.sigma ** 2
    assert np.linalg.norm(grad) <= 1e-9 * np.linalg.norm(P.adjoint(y)) / P.sigma ** 2
    lam, V = spectrum.eig_dense(P.hessian_explicit())
    np.testing.assert_allclose(posterior.mean_lowrank(P, lam, V, y), m, rtol=1e-8,
                               atol=1e-10 * np.abs(m).max())


def test_sample_map_covariance():
    """M = R^{-1}(I + V((1+lam)^-1/2 - 1)V^T) satisfies M M^T = low-rank
    Gamma_post for a partial spectrum too."""
    P = _tiny_problem()
    lam, V = spectrum.eig_dense(P.hessian_explicit())
    k = 6
    mean = np.zeros(P.nx)
    M = posterior.samples_lowrank(P, lam[:k], V[:, :k], mean, np.eye(P.nx))
    np.testing.assert_allclose(M @ M.T, posterior.post_cov_lowrank(P, lam[:k], V[:, :k]),
                               rtol=1e-10, atol=1e-14)


def test_variance_matches_dense_diag():
    P = _tiny_problem()
    lam, V = spectrum.eig_dense(P.hessian_explicit())
    nodes = np.array([0, 3, 12, 24])
    want = np.diag(posterior.post_cov_lowrank(P, lam[:5], V[:, :5]))[nodes]
    np.testing.assert_allclose(posterior.variance_lowrank(P, lam[:5], V[:, :5], nodes), want,
                               rtol=1e-11)


@pytest.mark.parametrize("dim,n", [(2, 7), (3, 5)])
def test_prior_diag_dst_closed_form(dim, n):
    """(Gamma_prior)_ii for the constant-coefficient prior equals the
    spectral sum over orthonormal discrete sine vectors
    sum_m prod_a s_{m_a}(i_a)^2 / (1 + alpha mu_m)^2."""
    alpha = 0.07
    P = Problem(_spec(dim=dim, n=n, prior_alpha=alpha, sensors=synth.uniform_sensors(2, dim, 1)))
    nodes = np.arange(P.nx)
    got = posterior.prior_diag(P, nodes)
    x = np.arange(1, n + 1)
    S = np.sqrt(2.0 / (n + 1)) * np.sin(np.outer(np.arange(1, n + 1), x) * np.pi / (n + 1))
    h = 1.0 / (n + 1)
    mu1 = 4 / h ** 2 * np.sin(np.arange(1, n + 1) * np.pi * h / 2) ** 2
    want = np.zeros(P.nx)
    for p in range(P.nx):
        idx = [(p // n ** a) % n for a in range(dim)]
        tot = 0.0
        for m in np.ndindex(*([n] * dim)):
            mu = sum(mu1[mi] for mi in m)
            w = np.prod([S[m[a], idx[a]] ** 2 for a in range(dim)])
            tot += w / (1 + alpha * mu) ** 2
        want[p] = tot
    np.testing.assert_allclose(got, want, rtol=1e-12)


# ---------------------------------------------------------------- time factors
def test_truncate_known_spectrum():
    """Eckart-Young on a matrix with prescribed singular values: the chosen
    rank is the smallest meeting the tail bound and the error is the tail."""
    r = synth.rng(2)
    U, _ = np.linalg.qr(r.standard_normal((60, 12)))
    Z, _ = np.linalg.qr(r.standard_normal((40, 12)))
    s = 10.0 ** -np.arange(12)
    Y = (U * s) @ Z.T
    W, V, err = timefactors.truncate(Y, 3e-6, 40)
    fro = np.linalg.norm(Y)
    # tail from s_6 = 1e-6 on is ~1.005e-6 <= 3e-6 |Y|; from s_5 it is ~1e-5 > 3e-6 |Y|
    assert W.shape[1] == 6
    assert abs(err - np.sqrt(np.sum(s[6:] ** 2))) < 1e-12
    assert np.linalg.norm(Y - W @ V.T) <= 3e-6 * fro


def test_streaming_exact_low_rank():
    r = synth.rng(3)
    Y = r.standard_normal((50, 3)) @ r.standard_normal((3, 37))
    W, V, ranks = timefactors.streaming(Y, 8, 1e-10, 40)
    assert W.shape[1] == 3 and max(ranks) == 3
    np.testing.assert_allclose(W @ V.T, Y, rtol=0, atol=1e-10 * np.abs(Y).max())


def test_streaming_trajectory_error_bound():
    """Low-rank-in-time factors of a real heat trajectory meet the tolerance
    and their rank stays close to the optimal SVD rank (Sec. 3)."""
    P = Problem(_spec(n=15, nt=120, sensors=synth.uniform_sensors(3, 2, 1)))
    u = P.prior_half(synth.normal_block(P.nx, 1, 8)[:, 0])
    Y = P.trajectory(u)
    tol = 1e-8
    W, V, ranks = timefactors.streaming(Y, 20, tol, 40)
    assert np.linalg.norm(Y - W @ V.T) <= tol * np.linalg.norm(Y)
    Wo, Vo, _ = timefactors.truncate(Y, tol, 40)
    assert Wo.shape[1] <= W.shape[1] <= Wo.shape[1] + 6


@pytest.mark.parametrize("k", [None, 6])
def test_sigma_override_equals_problem_at_that_sigma(k):
    """Gamma_noise = sigma^2 I (Sec. 2): the posterior queries of a problem
    set up at sigma0 and asked at sigma (eigenvalues rescaled by
    sigma0^2/sigma^2, data weighted by 1/sigma^2) equal those of the same
    problem set up at sigma with its own eigenpairs. k = None uses every
    eigenpair (then the mean is also the exact posterior mean at sigma);
    k = 6 sits at a spectral gap (lam_6 / lam_7 ~ 100), so the rank-k projector is unique. Catches a
    swapped sigma0/sigma in the rescaling or the data weighted at sigma0."""
    s0, s1 = 0.02, 0.005
    sens = synth.uniform_sensors(5, 2, 21)
    P0 = Problem(_spec(n=5, nt=8, obs_every=2, sensors=sens, sigma=s0, prior_alpha=0.05))
    P1 = Problem(_spec(n=5, nt=8, obs_every=2, sensors=sens, sigma=s1, prior_alpha=0.05))
    l0, V0 = spectrum.eig_dense(P0.hessian_explicit())
    l1, V1 = spectrum.eig_dense(P1.hessian_explicit())
    if k is not None:
        assert l0[k - 1] > 10 * l0[k]
        l0, V0, l1, V1 = l0[:k], V0[:, :k], l1[:k], V1[:, :k]
    np.testing.assert_allclose(posterior.rescale_eigs(l0, s0, s1), l1, rtol=1e-9, atol=1e-12 * l1[0])
    y = synth.normal_block(P0.n_data, 1, 4)[:, 0]
    m0 = posterior.mean_lowrank(P0, l0, V0, y, sigma=s1)
    m1 = posterior.mean_lowrank(P1, l1, V1, y)
    np.testing.assert_allclose(m0, m1, rtol=0, atol=1e-9 * np.abs(m1).max())
    if k is None:
        me = posterior.mean_exact(P1, y)
        np.testing.assert_allclose(m0, me, rtol=0, atol=1e-8 * np.abs(me).max())
    nodes = np.array([0, 6, 12, 18, 24])
    v0 = posterior.variance_lowrank(P0, l0, V0, nodes, sigma=s1)
    v1 = posterior.variance_lowrank(P1, l1, V1, nodes)
    np.testing.assert_allclose(v0, v1, rtol=1e-9)
    # samples: the maps xi -> sample agree through their covariance (the
    # eigenvector bases differ by rotations inside degenerate spaces)
    E = np.eye(P0.nx)
    S0 = posterior.samples_lowrank(P0, l0, V0, np.zeros(P0.nx), E, sigma=s1)
    S1 = posterior.samples_lowrank(P1, l1, V1, np.zeros(P1.nx), E)
    np.testing.assert_allclose(S0 @ S0.T, S1 @ S1.T, rtol=0, atol=1e-9 * np.abs(S1 @ S1.T).max())
    # and the sample map at the override is the low-rank covariance at sigma
    C1 = posterior.post_cov_lowrank(P1, l1, V1)
    np.testing.assert_allclose(S0 @ S0.T, C1, rtol=0, atol=1e-9 * np.abs(C1).max())


def test_cg_solver_matches_lu():
    """The oracle's CG solves (used where sparse LU fill-in is prohibitive)
    reach the stated relative residual 1e-14 of the operator itself, and give
    the same forward map, adjoint and Hessian as the LU solves on a 3D
    problem with a variable kappa."""
    spec = synth.small_spec(dim=3, n=7, nt=6, obs_every=2, n_obs=6, with_kappa=True, seed=12)
    Pl, Pc = Problem(spec), Problem(spec, solver="cg")
    b = synth.normal_block(Pl.nx, 2, 3)
    for A, solver in ((Pl.K, Pc._K_lu), (Pl.R, Pc._R_lu)):
        x = solver.solve(b)
        assert np.max(np.linalg.norm(b - A @ x, axis=0) / np.linalg.norm(b, axis=0)) <= 2e-14
    X = synth.normal_block(Pl.nx, 2, 5)
    for f in ("forward", "hessian_apply"):
        want = getattr(Pl, f)(X)
        np.testing.assert_allclose(getattr(Pc, f)(X), want, rtol=0, atol=1e-11 * np.abs(want).max())
    W = synth.normal_block(Pl.n_data, 2, 6)
    want = Pl.adjoint(W)
    np.testing.assert_allclose(Pc.adjoint(W), want, rtol=0, atol=1e-11 * np.abs(want).max())


def test_golden_files_are_consistent():
    """The oracle-written full-size reference values (tests/golden/make_spectra.py)
    are what their headers say: decreasing eigenvalues with explicit residuals
    far below the compared tolerances, and the sampled apply at the seeded
    nodes of the 63^3 grid."""
    for name, k in (("spectrum_heat2d_127.txt", 110), ("spectrum_heat3d_63_nt20.txt", 24)):
        rows = _read_golden(name)
        lam = np.array([float(r[1]) for r in rows])
        res = np.array([float(r[2]) for r in rows])
        assert len(lam) == k and np.all(np.diff(lam) <= 0) and lam[-1] > 0
        assert np.max(res) < 1e-12
    rows = _read_golden("apply_heat3d_63.txt")
    nodes = np.array([int(r[0]) for r in rows])
    assert np.array_equal(nodes, synth.query_nodes(63 ** 3, 256, 2028))


# ------------------------------------------------- convection-diffusion (Sec. 6.2)
@pytest.mark.parametrize("wind", [(0.0, 1.0), (-1.0, 0.5)])
def test_upwind_convection_linear_field(wind):
    """Upwind w . grad_h of the coordinate field x_a is w_a at every node whose
    upstream neighbour is inside the grid or the inflow boundary (where the
    Dirichlet value 0 equals x_a); the upwind direction is the low side for
    w_a > 0. Catches a downwind stencil, a wrong sign or a missing 1/h."""
    n = 9
    W = operators.upwind_convection(n, 2, wind)
    x = (np.arange(n) + 1.0) / (n + 1)
    for a in range(2):
        field = np.kron(np.ones(n), x) if a == 0 else np.kron(x, np.ones(n))  # x_0 fastest
        got = (W @ field).reshape(n, n)  # [i1, i0]
        other = 1 - a
        want_part = wind[a]
        # contributions of the other axis vanish on this field except at its
        # outflow/inflow nodes; compare where both axes see interior upstream data
        if wind[a] > 0:
            sl_a = slice(0, n)
        else:
            sl_a = slice(0, n - 1)
        if wind[other] == 0:
            sl_o = slice(0, n)
        elif wind[other] > 0:
            sl_o = slice(1, n)
        else:
            sl_o = slice(0, n - 1)
        sub = got[sl_a, sl_o] if a == 1 else got[sl_o, sl_a]
        np.testing.assert_allclose(sub, want_part, rtol=1e-12, atol=1e-12)


def test_upwind_step_closed_form():
    """Pure advection (nu = 0) in 1D: one implicit-Euler upwind step
    (1 + c) y_i - c y_{i-1} = y0_i, c = tau w / h, from a unit pulse at j has
    y_i = c^(i-j) / (1 + c)^(i-j+1) for i >= j and 0 upstream of j."""
    n, j, tau, w = 15, 4, 0.05, 1.0
    A = operators.convection_diffusion(n, 1, 0.0, (w,)).toarray()
    y0 = np.zeros(n)
    y0[j] = 1.0
    y = np.linalg.solve(np.eye(n) + tau * A, y0)
    c = tau * w * (n + 1)
    want = np.array([c ** (i - j) / (1 + c) ** (i - j + 1) if i >= j else 0.0 for i in range(n)])
    np.testing.assert_allclose(y, want, rtol=1e-12, atol=1e-15)


def _convdiff_spec(**kw):
    base = dict(dim=2, n=7, nt=10, obs_every=2, sensors=synth.uniform_sensors(6, 2, 2),
                pde="convdiff", conv_nu=1e-2, wind=(0.0, 1.0))
    base.update(kw)
    return _spec(**base)


def test_convdiff_adjoint_and_brute_force():
    """The nonsymmetric operator: <F u, w> = <u, F^T w> to 1e-12 (the adjoint
    steps solve with the transpose), F equals dense powers B (I + tau L)^-n,
    and the explicit F^T equals the transpose of the explicit F. Catches a
    forgotten transpose in the adjoint sweep."""
    P = Problem(_convdiff_spec())
    assert abs(P.L - P.L.T).max() > 1.0  # genuinely nonsymmetric
    r = synth.rng(19)
    u = r.standard_normal((P.nx, 3))
    w = r.standard_normal((P.n_data, 3))
    np.testing.assert_allclose(np.sum(P.forward(u) * w, axis=0), np.sum(u * P.adjoint(w), axis=0), rtol=1e-12)
    Sinv = np.linalg.inv(np.eye(P.nx) + P.tau * P.L.toarray())
    B = P.B.toarray()
    rows = [B @ np.linalg.matrix_power(Sinv, s) for s in P.steps]
    F = P.forward_explicit()
    np.testing.assert_allclose(F, np.vstack(rows), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(P.adjoint(np.eye(P.n_data)), F.T, rtol=1e-12, atol=1e-15)
    H = P.hessian_apply(np.eye(P.nx))
    assert np.max(np.abs(H - H.T)) <= 1e-12 * np.max(np.abs(H))


# ---------------------------------------------------------------- low-rank product, Arnoldi (Sec. 4)
def _norm2(A):
    return float(np.linalg.norm(np.asarray(A), 2))


@pytest.mark.parametrize("pde", ["heat", "convdiff"])
def test_lowrank_apply_exact_without_truncation(pde):
    """Sec. 4 Algorithm 1's product with nothing discarded (eps_0 = 0, no
    rank cap) is the exact Htilde x and H_mis x (Sec. 2 Eq. (prior_pre)).
    Catches a wrong step of the pipeline: an off-by-one time index in the
    observed rows of the truncated trajectory, the wrong column of the
    adjoint trajectory, a missing 1/sigma^2 or prior factor."""
    P = Problem(_convdiff_spec() if pde == "convdiff" else _spec(n=7, nt=12, obs_every=3))
    x = synth.normal_block(P.nx, 1, 41)[:, 0]
    got, info = lowrank.lowrank_hessian_apply(P, x, 0.0, 10 ** 6, 5)
    want = P.hessian_apply(x)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))
    assert info["err_y"] <= 1e-14 and info["err_q"] <= 1e-14
    got_m, _ = lowrank.lowrank_hessian_apply(P, x, 0.0, 10 ** 6, 4, misfit_only=True)
    want_m = P.misfit_apply(x)
    assert np.max(np.abs(got_m - want_m)) <= 1e-12 * np.max(np.abs(want_m))


def test_adjoint_trajectory_first_column_is_adjoint():
    """q_1 of the backward recursion is F^T d (Sec. 6 Eq. (postvar) with
    K^{-T}), and the columns past the last observed step are zero."""
    P = Problem(_spec(n=7, nt=13, obs_every=3))
    d = synth.normal_block(P.n_data, 1, 42)[:, 0]
    Q = lowrank.adjoint_trajectory(P, d)
    np.testing.assert_allclose(Q[:, 0], P.adjoint(d), rtol=1e-13, atol=1e-15)
    assert not np.any(Q[:, P.steps[-1]:])
    assert np.all(np.linalg.norm(Q[:, :P.steps[-1]], axis=0) > 0)


@pytest.mark.parametrize("tol", [1e-4, 1e-6])
def test_lowrank_apply_error_bound(tol):
    """With truncation the product differs from Htilde x by at most
    ||R^-1|| (||F|| ||B|| tol ||Y||_F / sigma^2 + tol ||Q||_F) (the streaming
    truncation keeps ||Y - W V^T||_F <= tol ||Y||_F for both trajectories;
    ||Q||_F of the truncated data is within O(tol) of the exact one, a 1 %
    margin). The error is genuinely there, and the product is no longer
    symmetric (the reason for Arnoldi in Sec. 4), by at most twice the bound.
    An off-by-one time index in the adjoint's data or a wrong row of V makes
    the error O(||Htilde x||) and fails the bound."""
    P = Problem(_spec(n=7, nt=40, obs_every=2, sensors=synth.uniform_sensors(8, 2, 4)))
    x = synth.normal_block(P.nx, 2, 43)
    got, info = lowrank.lowrank_hessian_apply(P, x[:, 0], tol, 40, 8)
    want = P.hessian_apply(x[:, 0])
    z = P.prior_half(x[:, 0])
    Y = P.trajectory(z)
    Q = lowrank.adjoint_trajectory(P, P.forward(z) / P.sigma ** 2)
    Rinv = P.prior_half(np.eye(P.nx))
    F = P.forward_explicit()
    bound = _norm2(Rinv) * (_norm2(F) * _norm2(P.B.toarray()) * tol * np.linalg.norm(Y) / P.sigma ** 2
                            + 1.01 * tol * np.linalg.norm(Q))
    err = np.linalg.norm(got - want)
    assert 0.0 < err <= bound, (err, bound)
    assert info["err_y"] <= tol and info["err_q"] <= tol and info["rank_y"] < P.nx
    got2, _ = lowrank.lowrank_hessian_apply(P, x[:, 1], tol, 40, 8)
    asym = abs(x[:, 1] @ got - x[:, 0] @ got2)
    assert 0.0 < asym <= 2 * bound * max(np.linalg.norm(x[:, 0]), np.linalg.norm(x[:, 1])) * 1.5


def test_ritz_nonsym_known_spectrum_and_residual_estimate():
    """Algorithm 1 on a nonsymmetric matrix with a prescribed spectrum (a
    complex pair included): after n steps the Ritz values are that spectrum;
    after m < n steps the estimate |h_{m+1,m}| |e_m^T y| equals the true
    residual ||A V_m y - theta V_m y|| of every real Ritz pair (the Arnoldi
    relation A V_m = V_{m+1} H). Catches a transposed H, a wrong row of the
    estimate or an unsorted spectrum."""
    r = synth.rng(44)
    n = 12
    lam = np.array([9.0, 7.5, 6.0, 4.0, 3.0, 2.0, 1.0, 0.5, 0.25, 0.125])
    T = np.zeros((n, n))
    T[:10, :10] = np.diag(lam)
    T[10:, 10:] = [[-1.0, 2.0], [-2.0, -1.0]]  # eigenvalues -1 +- 2i
    S = r.standard_normal((n, n)) + 3 * np.eye(n)
    A = S @ T @ np.linalg.inv(S)
    v1 = r.standard_normal(n)
    V, H = spectrum.arnoldi_mgs(lambda v: A @ v, v1, n)
    got, _, _ = lowrank.ritz_nonsym(H, n)
    want = np.concatenate([lam, [-1 + 2j, -1 - 2j]])
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-8)
    m = 6
    V, H = spectrum.arnoldi_mgs(lambda v: A @ v, v1, m)
    theta, Yv, res = lowrank.ritz_nonsym(H, m)
    for i in range(m):
        if abs(theta[i].imag) > 0:
            continue
        y = V[:, :m] @ Yv[:, i].real
        true = np.linalg.norm(A @ y - theta[i].real * y)
        assert abs(true - res[i]) <= 1e-9 * np.abs(A).max()


def test_arnoldi_threshold_rule_symmetric_operator():
    """The threshold stop of Sec. 6.1 on the exact (symmetric) Htilde: the
    Ritz values above eps are the eigenvalues above eps of the explicit
    matrix, in number and value, every Ritz value is real, and the Arnoldi
    relation Htilde V_m = V_{m+1} H holds."""
    P = Problem(_spec(n=7, nt=12, obs_every=3, sensors=synth.uniform_sensors(6, 2, 5)))
    lam, _ = spectrum.eig_dense(P.hessian_explicit())
    eps = lam[4] * 0.5 + lam[5] * 0.5  # between the 5th and 6th eigenvalue
    v1 = synth.normal_block(P.nx, 1, 45)[:, 0]
    m, V, H, theta, res = lowrank.arnoldi_threshold(P.hessian_apply, v1, eps, 1e-10, 40)
    above = theta.real >= eps
    assert m < 40 and int(np.sum(above)) == 5
    np.testing.assert_allclose(theta.real[above], lam[:5], rtol=1e-9)
    assert np.max(np.abs(theta.imag)) <= 1e-10 * lam[0]
    # the Arnoldi relation holds to rounding (single MGS lets orthogonality
    # decay as Ritz values converge; the relation does not depend on it)
    AV = np.column_stack([P.hessian_apply(V[:, j]) for j in range(m)])
    assert np.max(np.abs(AV - V @ H)) <= 1e-12 * lam[0]


# ---------------------------------------------------------------- space-time parameter (Sec. 4)
def _st_problem(**kw):
    base = dict(n=3, nt=5, obs_every=2, sensors=synth.uniform_sensors(4, 2, 31), sigma=0.05, prior_alpha=0.1)
    base.update(kw)
    return Problem(_spec(**base))


@pytest.mark.parametrize("pde", ["heat", "convdiff"])
def test_source_forward_brute_force_and_adjoint(pde):
    """y_n = sum_{m<=n} S^{n-m+1} tau u_m: the explicit F of the source map
    equals the block matrix [tau B S^{n_k - m + 1}] (m <= n_k), and
    <F U, d> = <U, F^T d>. Catches a source added after the solve, a wrong
    tau, or an adjoint trajectory shifted by one step."""
    kw = dict(pde="convdiff", conv_nu=1e-2, wind=(0.0, 1.0)) if pde == "convdiff" else {}
    P = _st_problem(**kw)
    S = np.linalg.inv(np.eye(P.nx) + P.tau * P.L.toarray())
    B = P.B.toarray()
    F = np.zeros((P.n_data, P.nx * P.nt))
    for k, nk in enumerate(P.steps):
        for m in range(1, nk + 1):
            F[k * P.n_obs:(k + 1) * P.n_obs, (m - 1) * P.nx:m * P.nx] = P.tau * B @ np.linalg.matrix_power(S, nk - m + 1)
    Fo = np.column_stack([spacetime.forward_source(P, np.eye(P.nx * P.nt)[:, c].reshape(P.nt, P.nx).T)
                          for c in range(P.nx * P.nt)])
    np.testing.assert_allclose(Fo, F, rtol=1e-12, atol=1e-15)
    r = synth.rng(32)
    U = r.standard_normal((P.nx, P.nt))
    d = r.standard_normal(P.n_data)
    lhs = spacetime.forward_source(P, U) @ d
    rhs = np.sum(U * spacetime.adjoint_source(P, d))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    np.testing.assert_allclose(np.column_stack([spacetime.vec(spacetime.adjoint_source(P, e))
                                                for e in np.eye(P.n_data)]), F.T, rtol=1e-12, atol=1e-15)


def test_spacetime_hessian_symmetric_psd():
    """Htilde = R^-1 F^T F R^-1 / sigma^2 on vec(U) is symmetric positive
    semi-definite (before the symmetrisation of the explicit matrix) and
    equals the product of its explicit factors."""
    P = _st_problem()
    N = P.nx * P.nt
    cols = [spacetime.vec(spacetime.hessian_st(P, e.reshape(P.nt, P.nx).T)) for e in np.eye(N)]
    H = np.column_stack(cols)
    assert np.max(np.abs(H - H.T)) <= 1e-12 * np.abs(H).max()
    assert np.linalg.eigvalsh(0.5 * (H + H.T)).min() >= -1e-12 * np.abs(H).max()
    F = np.column_stack([spacetime.forward_source(P, e.reshape(P.nt, P.nx).T) for e in np.eye(N)])
    Rinv = np.kron(np.eye(P.nt), P.prior_half(np.eye(P.nx)))
    np.testing.assert_allclose(H, Rinv @ F.T @ F @ Rinv / P.sigma ** 2, rtol=1e-11, atol=1e-12 * np.abs(H).max())


def test_lowrank_vector_ops():
    """Truncation of a factored matrix: exact without a tolerance; with
    prescribed singular values it keeps the smallest rank meeting the
    Frobenius tail bound (Eckart-Young); the factored inner product equals the
    dense one."""
    r = synth.rng(33)
    A = r.standard_normal((30, 7))
    B = r.standard_normal((20, 7))
    A2, B2 = spacetime.truncate(A, B, 0.0, 100)
    np.testing.assert_allclose(A2 @ B2.T, A @ B.T, rtol=0, atol=1e-12 * np.abs(A @ B.T).max())
    U, _ = np.linalg.qr(r.standard_normal((30, 8)))
    Z, _ = np.linalg.qr(r.standard_normal((20, 8)))
    s = 10.0 ** -np.arange(8)
    # split into two factored terms that sum to U diag(s) Z^T
    A = np.hstack([U[:, :4] * s[:4], U[:, 4:] * s[4:]])
    B = np.hstack([Z[:, :4], Z[:, 4:]])
    At, Bt = spacetime.truncate(A, B, 3e-4, 100)
    assert At.shape[1] == 4  # tail from s_4 = 1e-4 is ~1.005e-4 <= 3e-4 ||.||; from s_3 it is 1e-3
    err = np.linalg.norm(A @ B.T - At @ Bt.T)
    assert abs(err - np.sqrt(np.sum(s[4:] ** 2))) < 1e-13
    X = (r.standard_normal((30, 3)), r.standard_normal((20, 3)))
    Y = (r.standard_normal((30, 5)), r.standard_normal((20, 5)))
    assert abs(spacetime.dot(X, Y) - np.sum((X[0] @ X[1].T) * (Y[0] @ Y[1].T))) < 1e-10


def test_lr_hessian_apply_exact_without_truncation():
    P = _st_problem(n=7, nt=12, obs_every=3)
    r = synth.rng(34)
    A = r.standard_normal((P.nx, 3))
    B = r.standard_normal((P.nt, 3))
    Ao, Bo = spacetime.lr_hessian_apply(P, A, B, 0.0, 100, 5)
    want = spacetime.hessian_st(P, A @ B.T)
    assert np.max(np.abs(Ao @ Bo.T - want)) <= 1e-12 * np.abs(want).max()


def test_lr_arnoldi_equals_dense_arnoldi():
    """Algorithm 1 on factored vectors with nothing truncated is Algorithm 1
    on vec(U) with the explicit space-time Htilde: the same Hessenberg matrix
    from the same start vector, and its Ritz values converge to the dense
    eigenvalues. With the paper's truncation (1e-8) the leading Ritz values
    stay within 1e-7 of them and every vector keeps unit norm."""
    P = _st_problem(n=7, nt=16, obs_every=2, sensors=synth.uniform_sensors(6, 2, 35))
    Hd = spacetime.hessian_st_explicit(P)
    lam = np.sort(np.linalg.eigvalsh(Hd))[::-1]
    r = synth.rng(36)
    A0 = r.standard_normal((P.nx, 2))
    B0 = r.standard_normal((P.nt, 2))
    m = 24
    H, ranks, _ = spacetime.lr_arnoldi(P, A0, B0, m, 0.0, 1000, 4)
    v1 = spacetime.vec(A0 @ B0.T)
    _, Hdense = spectrum.arnoldi_mgs(lambda x: Hd @ x, v1, m)
    # the leading columns (later ones amplify rounding once the fast-decaying
    # spectrum is resolved, in either form)
    assert np.max(np.abs(H[:9, :8] - Hdense[:9, :8])) <= 1e-10 * lam[0]
    theta, _, _ = lowrank.ritz_nonsym(H, m)
    np.testing.assert_allclose(theta.real[:4], lam[:4], rtol=1e-9)
    Ht, ranks_t, basis = spacetime.lr_arnoldi(P, A0, B0, m, 1e-8, 40, 4)
    th_t, _, _ = lowrank.ritz_nonsym(Ht, m)
    np.testing.assert_allclose(th_t.real[:4], lam[:4], rtol=1e-7)
    assert max(ranks_t) <= min(P.nx, P.nt, 40)
    assert abs(spacetime.dot(basis[3], basis[3]) - 1.0) < 1e-12


# ---------------------------------------------------------------- alternating space-time solve (Sec. 6.1)
def _als_setup(n=7, nt=20, dim=2):
    P = Problem(_spec(n=n, nt=nt, dim=dim))
    A = P.K.toarray()
    return P, A


def test_als_full_rank_is_time_stepping():
    """With r = nt the time basis spans everything: one sweep solves the
    space-time system (Eq. (st_pde)) exactly and reproduces the
    implicit-Euler trajectory of the initial condition (f_1 = u)."""
    P, A = _als_setup()
    u = synth.normal_block(P.nx, 1, 51)[:, 0]
    Wf = u[:, None]
    Vf = np.zeros((P.nt, 1))
    Vf[0, 0] = 1.0
    V0, _ = np.linalg.qr(synth.normal_block(P.nt, P.nt, 52))
    W, V, res = als.als_solve(A, Wf, Vf, V0, 1)
    Y = P.trajectory(u)
    assert res[0] < 1e-12
    assert np.max(np.abs(W @ V.T - Y)) <= 1e-12 * np.abs(Y).max()


@pytest.mark.parametrize("modes", [[(1, 1)], [(1, 1), (2, 3)]])
def test_als_recovers_exact_low_rank_solution(modes):
    """u a sum of k sine modes (eigenvectors of the Dirichlet Laplacian,
    Sec. 5): y_n = sum_k (1 + tau mu_k)^-n u_k has rank k, and the
    alternating solve with r = k from a random start converges to it."""
    P, A = _als_setup(n=15, nt=40)
    n = P.n
    x = np.arange(1, n + 1) / (n + 1)
    u = np.zeros(P.nx)
    for a, b in modes:
        u += np.kron(np.sin(b * np.pi * x), np.sin(a * np.pi * x))
    Wf = u[:, None]
    Vf = np.zeros((P.nt, 1))
    Vf[0, 0] = 1.0
    V0, _ = np.linalg.qr(synth.normal_block(P.nt, len(modes), 53))
    W, V, res = als.als_solve(A, Wf, Vf, V0, 6)
    Y = P.trajectory(u)
    assert res[-1] < 1e-12, res
    assert np.max(np.abs(W @ V.T - Y)) <= 1e-11 * np.abs(Y).max()


def test_als_galerkin_conditions():
    """The two half steps are Galerkin projections: after the time step the
    residual R = A Y - Y S^T - F is orthogonal to the space basis (Q^T R = 0);
    after the space step it is orthogonal to the time basis (R V = 0). A
    transposed T or a shift in the wrong direction breaks one of them. The
    block forward substitution equals the dense block-bidiagonal solve."""
    P, A = _als_setup(n=7, nt=16)
    r = synth.rng(54)
    Wf = r.standard_normal((P.nx, 2))
    Vf = r.standard_normal((P.nt, 2))
    V, _ = np.linalg.qr(r.standard_normal((P.nt, 3)))
    F = Wf @ Vf.T

    def R_of(Y):
        YS = np.zeros_like(Y)
        YS[:, 1:] = Y[:, :-1]
        return A @ Y - YS - F

    T = als.shift_gram(V)
    W = sla_solve_sylvester(A, -T, Wf @ (Vf.T @ V))
    assert np.max(np.abs(R_of(W @ V.T) @ V)) <= 1e-12 * np.abs(F).max()
    Q, _ = np.linalg.qr(W)
    G = (Q.T @ Wf) @ Vf.T
    Z = als.time_step(Q.T @ A @ Q, G)
    assert np.max(np.abs(Q.T @ R_of(Q @ Z.T))) <= 1e-12 * np.abs(F).max()
    k = Q.shape[1]
    Ah = Q.T @ A @ Q
    big = np.kron(np.eye(P.nt), Ah) - np.kron(np.eye(P.nt, k=-1), np.eye(k))
    z = np.linalg.solve(big, G.T.reshape(-1))
    np.testing.assert_allclose(Z.reshape(-1), z, rtol=1e-12, atol=1e-14)


def sla_solve_sylvester(A, B, C):
    import scipy.linalg
    return scipy.linalg.solve_sylvester(A, B, C)


def test_als_adjoint_full_rank_is_backward_recursion():
    """The adjoint system A^T q_n = q_{n+1} + f_n in reversed time: with
    r = nt one sweep reproduces the backward recursion of the Hessian's
    adjoint sweep (lowrank.adjoint_trajectory, itself pinned to F^T d)."""
    P, A = _als_setup(n=7, nt=12)
    r = synth.rng(55)
    D = r.standard_normal(P.n_data)
    Q = lowrank.adjoint_trajectory(P, D)
    F = np.zeros((P.nx, P.nt))
    Bt = P.B.T.toarray()
    for k, n in enumerate(P.steps):
        F[:, n - 1] = Bt @ D[k * P.n_obs:(k + 1) * P.n_obs]
    U, s, Vt = np.linalg.svd(F, full_matrices=False)
    V0, _ = np.linalg.qr(r.standard_normal((P.nt, P.nt)))
    W, V, res = als.als_adjoint(A, U * s, Vt.T, V0, 1)
    assert res[0] < 1e-12
    assert np.max(np.abs(W @ V.T - Q)) <= 1e-12 * np.abs(Q).max()


@pytest.mark.parametrize("misfit", [False, True])
def test_als_hessian_full_rank_is_exact(misfit):
    """With r = nt both alternating solves are exact after one sweep, so the
    product is Htilde x (H_mis x) of the time-stepping oracle; with r below
    nt it differs by about the solves' residuals."""
    P, A = _als_setup(n=7, nt=12)
    x = synth.normal_block(P.nx, 1, 56)[:, 0]
    ref = P.misfit_apply(x) if misfit else P.hessian_apply(x)
    out, info = als.als_hessian_apply(P, x, P.nt, 1, A=A, misfit_only=misfit)
    assert info["res_f"][0] < 1e-12 and info["res_a"][0] < 1e-12
    assert np.max(np.abs(out - ref)) <= 1e-11 * np.abs(ref).max()
    out4, info4 = als.als_hessian_apply(P, x, 4, 3, A=A, misfit_only=misfit)
    err = np.linalg.norm(out4 - ref) / np.linalg.norm(ref)
    assert 0 < err < 1e-2


def _als_setup_convdiff(n=7, nt=12):
    """The upwind convection-diffusion operator (Sec. 6.2): A = I + tau L is
    not symmetric, so a transposed A anywhere in the alternating solve or its
    adjoint changes the result."""
    spec = _spec(n=n, nt=nt, pde="convdiff", conv_nu=1e-2, wind=(0.0, 1.0, 0.0))
    P = Problem(spec)
    A = P.K.toarray()
    assert np.abs(A - A.T).max() > 1e-3
    return P, A


def test_als_convdiff_full_rank_forward_and_adjoint():
    """Nonsymmetric operator: with r = nt one sweep of the forward solve
    reproduces implicit Euler with (I + tau L) and one sweep of the adjoint
    solve the backward recursion with (I + tau L)^T; swapping the two
    operators fails both."""
    P, A = _als_setup_convdiff()
    g = synth.rng(57)
    u = g.standard_normal(P.nx)
    e1 = np.zeros((P.nt, 1))
    e1[0, 0] = 1.0
    V0, _ = np.linalg.qr(g.standard_normal((P.nt, P.nt)))
    W, V, res = als.als_solve(A, u[:, None], e1, V0, 1)
    Y = P.trajectory(u)
    assert res[0] < 1e-12
    assert np.max(np.abs(W @ V.T - Y)) <= 1e-12 * np.abs(Y).max()
    Wt, Vt, _ = als.als_solve(A.T.copy(), u[:, None], e1, V0, 1)
    assert np.max(np.abs(Wt @ Vt.T - Y)) > 1e-6 * np.abs(Y).max()
    D = g.standard_normal(P.n_data)
    Q = lowrank.adjoint_trajectory(P, D)
    F = np.zeros((P.nx, P.nt))
    Bt = P.B.T.toarray()
    for k, n in enumerate(P.steps):
        F[:, n - 1] = Bt @ D[k * P.n_obs:(k + 1) * P.n_obs]
    U, s, Vt2 = np.linalg.svd(F, full_matrices=False)
    Wq, Vq, resq = als.als_adjoint(A, U * s, Vt2.T, V0, 1)
    assert resq[0] < 1e-12
    assert np.max(np.abs(Wq @ Vq.T - Q)) <= 1e-12 * np.abs(Q).max()
    Wx, Vx, _ = als.als_adjoint(A.T.copy(), U * s, Vt2.T, V0, 1)
    assert np.max(np.abs(Wx @ Vx.T - Q)) > 1e-6 * np.abs(Q).max()


def test_als_convdiff_hessian_full_rank_is_exact():
    """The product on the nonsymmetric operator with r = nt equals the
    time-stepping Htilde (forward with A, adjoint with A^T)."""
    P, A = _als_setup_convdiff()
    x = synth.normal_block(P.nx, 1, 58)[:, 0]
    ref = P.hessian_apply(x)
    out, info = als.als_hessian_apply(P, x, P.nt, 1, A=A)
    assert np.max(np.abs(out - ref)) <= 1e-11 * np.abs(ref).max()
