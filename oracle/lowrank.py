"""The low-rank matrix-vector product of Sec. 4 Algorithm 1 and the Arnoldi
run around it (FP64). TEST INFRASTRUCTURE ONLY (see the package docstring).

Algorithm 1 applies Htilde "up to the truncation tolerance eps_0": the
space-time solutions the product passes through are kept in low-rank form
and truncated, which makes the computed product non-symmetric (the reason
the paper uses Arnoldi rather than Lanczos, Sec. 4). With the initial
condition as parameter (Sec. 6) the space-time objects are the state and
adjoint trajectories, so the product is, for one column x:

1. z = Gamma_prior^{1/2} x (skipped for H_mis);
2. forward trajectory Y = [y_1 .. y_nt] of z, truncated to W_Y V_Y^T by the
   streaming recompression of ``timefactors.streaming`` (chunks of s steps,
   tolerance eps_0, rank cap rmax);
3. the adjoint's data are the observations of the truncated trajectory,
   d_n = B (W_Y V_Y^T)[:, n-1] / sigma^2 at every observed step n;
4. adjoint trajectory Q = [q_1 .. q_nt], q_{nt+1} = 0,
   q_n = (I + tau L)^{-T} (q_{n+1} + B^T d_n) (d_n = 0 at unobserved steps),
   truncated the same way to W_Q V_Q^T;
5. result Gamma_prior^{1/2} (W_Q V_Q^T)[:, 0] (the truncated q_1, which is
   F^T d in the untruncated case).

With eps_0 = 0 (nothing discarded) every step is exact and the result is
``Problem.hessian_apply``.

* ``adjoint_trajectory`` — step 4 before truncation.
* ``lowrank_hessian_apply`` — steps 1-5.
* ``ritz_nonsym`` — eigenvalues of the leading square block of Arnoldi's H
  (a library eigensolver; they may be complex), sorted by decreasing real
  part, with the residual estimate |h_{m+1,m}| |e_m^T y| (||y|| = 1) of each
  real one.
* ``arnoldi_threshold`` — Algorithm 1 (``spectrum.arnoldi_mgs`` one step at
  a time) stopped by the threshold rule of Sec. 6.1: once every Ritz value
  whose real part is at least eps has a residual estimate of at most
  tol * |theta_1| and some Ritz value lies below eps, from step 8 on (or
  m_max steps).
"""
from __future__ import annotations

import numpy as np

from . import timefactors


def adjoint_trajectory(P, D):
    """Q = [q_1 .. q_nt] of the backward recursion for data D (n_data,)."""
    D = np.asarray(D, dtype=np.float64).reshape(-1)
    Bt = P.B.T.tocsr()
    Q = np.zeros((P.nx, P.nt))
    q = np.zeros(P.nx)
    for n in range(P.nt, 0, -1):
        k = P._obs_index.get(n)
        rhs = q if k is None else q + Bt @ D[k * P.n_obs:(k + 1) * P.n_obs]
        q = P.step_adjoint(rhs)
        Q[:, n - 1] = q
    return Q


def lowrank_hessian_apply(P, x, tol, rmax, s, misfit_only=False):
    """Steps 1-5 for one column x (nx,). Returns (result, info) with info the
    ranks and the relative Frobenius truncation errors of both trajectories."""
    x = np.asarray(x, dtype=np.float64).reshape(-1)
    z = x if misfit_only else P.prior_half(x)
    Y = P.trajectory(z)
    Wy, Vy, _ = timefactors.streaming(Y, s, tol, rmax)
    Yt = Wy @ Vy.T
    D = np.zeros(P.n_data)
    for k, n in enumerate(P.steps):
        D[k * P.n_obs:(k + 1) * P.n_obs] = P.B @ Yt[:, n - 1]
    D /= P.sigma ** 2
    Q = adjoint_trajectory(P, D)
    Wq, Vq, _ = timefactors.streaming(Q, s, tol, rmax)
    q1 = Wq @ Vq[0, :]
    out = q1 if misfit_only else P.prior_half(q1)

    def rel(A, B):
        n = np.linalg.norm(A)
        return float(np.linalg.norm(A - B) / n) if n > 0 else 0.0

    info = dict(rank_y=Wy.shape[1], rank_q=Wq.shape[1], err_y=rel(Y, Yt), err_q=rel(Q, Wq @ Vq.T))
    return out, info


def ritz_nonsym(H: np.ndarray, m: int):
    """Eigenvalues of H[:m, :m] by decreasing real part, the normalised
    eigenvectors, and the residual estimates |H[m, m-1]| |y_m|."""
    lam, S = np.linalg.eig(H[:m, :m])
    order = np.lexsort((-lam.imag, -lam.real))
    lam = lam[order]
    S = S[:, order]
    S = S / np.linalg.norm(S, axis=0)
    beta = abs(H[m, m - 1]) if H.shape[0] > m else 0.0
    res = beta * np.abs(S[m - 1, :])
    return lam, S, res


def arnoldi_threshold(apply, v1, eps, tol, m_max):
    """Arnoldi (MGS) until the threshold rule holds or m_max steps.
    Returns (m, V, H, ritz values, residual estimates)."""
    nx = v1.shape[0]
    V = np.zeros((nx, m_max + 1))
    H = np.zeros((m_max + 1, m_max))
    V[:, 0] = v1 / np.linalg.norm(v1)
    m = 0
    for j in range(m_max):
        w = apply(V[:, j])
        for i in range(j + 1):
            H[i, j] = w @ V[:, i]
            w = w - H[i, j] * V[:, i]
        H[j + 1, j] = np.linalg.norm(w)
        m = j + 1
        if H[j + 1, j] == 0.0:
            break
        V[:, j + 1] = w / H[j + 1, j]
        if m < 8:
            continue  # a short Krylov space has not found the dominant eigenvalues yet
        lam, _, res = ritz_nonsym(H[:m + 1, :m], m)
        above = lam.real >= eps
        if np.any(~above) and np.all(res[above] <= tol * abs(lam[0])):
            break
    lam, _, res = ritz_nonsym(H[:m + 1, :m], m)
    return m, V[:, :m + 1], H[:m + 1, :m], lam, res
