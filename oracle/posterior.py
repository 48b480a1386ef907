"""Posterior covariance, mean, pointwise variance and samples (FP64).

Definitions (prior mean 0, noise mean 0):

* Gamma_post = (F^T Gamma_noise^{-1} F + Gamma_prior^{-1})^{-1}
  (Sec. 2 Eq. (postcov1); Sec. 6 Eq. (postvar)) with Gamma_prior^{-1} = R^2.
* MAP point / posterior mean u_post = Gamma_post F^T Gamma_noise^{-1} y_obs
  (Sec. 2, Eq. (map1) and the least-squares problem after it).
* Low-rank form: with Htilde ~ V Lambda V^T,
  Gamma_post ~ R^{-1} (I - V D V^T) R^{-1}, D = diag(lambda/(lambda+1))
  (Sec. 2: factorisation through Gamma_prior^{1/2} and the
  Sherman-Morrison-Woodbury step).
* Samples: u_post + R^{-1} (I + V Lambda V^T)^{-1/2} xi with
  (I + V Lambda V^T)^{-1/2} = I + V ((I+Lambda)^{-1/2} - I) V^T for
  orthonormal V (spectral calculus); their covariance is the low-rank
  Gamma_post.
* Noise rescaling: Htilde(sigma) = Htilde(sigma0) sigma0^2 / sigma^2, so the
  eigenvectors are unchanged and lambda(sigma) = lambda(sigma0) sigma0^2/sigma^2.
"""
from __future__ import annotations

import numpy as np


def rescale_eigs(lam, sigma0: float, sigma: float):
    return np.asarray(lam) * (sigma0 ** 2 / sigma ** 2)


def post_cov_exact(P) -> np.ndarray:
    """(H_mis + R^2)^{-1} by a dense inverse (tiny sizes)."""
    H = P.misfit_explicit()
    R = P.R.toarray()
    M = H + R @ R
    return np.linalg.inv(0.5 * (M + M.T))


def smw_inner(lam, V) -> np.ndarray:
    """I - V diag(lam/(lam+1)) V^T (dense)."""
    d = lam / (lam + 1.0)
    return np.eye(V.shape[0]) - (V * d) @ V.T


def post_cov_lowrank(P, lam, V) -> np.ndarray:
    """R^{-1} (I - V D V^T) R^{-1} (dense, tiny sizes)."""
    Rinv = P.prior_half(np.eye(P.nx))
    return Rinv @ smw_inner(lam, V) @ Rinv


def mean_lowrank(P, lam, V, yobs, sigma=None):
    """R^{-1} (I - V D V^T) R^{-1} F^T y_obs / sigma^2 with the eigenvalues
    rescaled to the requested noise level."""
    sigma = P.sigma if sigma is None else float(sigma)
    lam_s = rescale_eigs(lam, P.sigma, sigma)
    d = lam_s / (lam_s + 1.0)
    g = P.adjoint(np.asarray(yobs, dtype=np.float64)) / sigma ** 2
    z = P.prior_half(g)
    z = z - V @ (d * (V.T @ z))
    return P.prior_half(z)


def mean_exact(P, yobs) -> np.ndarray:
    """Gamma_post F^T y_obs / sigma^2 with the dense exact Gamma_post."""
    g = P.adjoint(np.asarray(yobs, dtype=np.float64)) / P.sigma ** 2
    return post_cov_exact(P) @ g


def prior_diag(P, nodes) -> np.ndarray:
    """(Gamma_prior)_{ii} = ||R^{-1} e_i||^2 by direct solves."""
    nodes = np.asarray(nodes)
    E = np.zeros((P.nx, len(nodes)))
    E[nodes, np.arange(len(nodes))] = 1.0
    X = P.prior_half(E)
    return np.sum(X * X, axis=0)


def variance_lowrank(P, lam, V, nodes, sigma=None, G=None) -> np.ndarray:
    """diag(Gamma_post) at the given nodes from the low-rank form:
    (Gamma_prior)_ii - sum_j D_j (R^{-1} V)_{ij}^2."""
    sigma = P.sigma if sigma is None else float(sigma)
    lam_s = rescale_eigs(lam, P.sigma, sigma)
    d = lam_s / (lam_s + 1.0)
    if G is None:
        G = P.prior_half(V)
    g = G[np.asarray(nodes)]
    return prior_diag(P, nodes) - (g * g) @ d


def samples_lowrank(P, lam, V, mean, xi, sigma=None) -> np.ndarray:
    """mean + R^{-1} (xi + V ((1+lambda)^{-1/2} - 1) V^T xi) for a block xi
    (nx, s) of standard normals."""
    sigma = P.sigma if sigma is None else float(sigma)
    lam_s = rescale_eigs(lam, P.sigma, sigma)
    c = 1.0 / np.sqrt(1.0 + lam_s) - 1.0
    xi = np.asarray(xi, dtype=np.float64)
    z = xi + V @ (c[:, None] * (V.T @ xi))
    return mean.reshape(-1, 1) + P.prior_half(z)
