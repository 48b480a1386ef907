"""A space-time parameter and Algorithm 1 on low-rank space-time vectors
(Sec. 4, Eq. (lanczos1)-(lanczos2)), FP64. TEST INFRASTRUCTURE ONLY (see the
package docstring).

The parameter is a source u(x, t) of the state equation (Sec. 4 names a
space-time right-hand side as the case where the low-rank form pays most):
y_t + L y = u, y(0) = 0; implicit Euler with tau = T / nt:
(I + tau L) y_n = y_{n-1} + tau u_n, n = 1..nt. The parameter vector is
U = [u_1 .. u_nt] (nx x nt; vec(U) stacks the columns).

* F U = [B y_n] at the observed steps;
* F^T d = tau [q_1 .. q_nt] with the adjoint recursion q_{nt+1} = 0,
  q_n = (I + tau L)^{-T} (q_{n+1} + B^T d_n) (d_n = 0 at unobserved steps),
  since y_n = sum_{m <= n} S^{n-m+1} tau u_m with S = (I + tau L)^{-1};
* Gamma_prior = I_nt (x) Gamma_x, Gamma_x as for the initial condition, so
  Gamma_prior^{1/2} U = R^{-1} U (column by column);
* Htilde U = R^{-1} F^T F R^{-1} U / sigma^2.

Low-rank vectors (Sec. 4): U ~ A B^T (A: nx x r, B: nt x r).

* ``truncate`` — thin QR of both factors, SVD of the small R_A R_B^T, the
  smallest rank whose discarded Frobenius tail is at most tol ||A B^T||_F
  (capped at rmax); returns (Q_A U_r S_r, Q_B Z_r);
* ``dot`` — <X, Y> = trace(A_X^T A_Y B_Y^T B_X);
* ``lr_hessian_apply`` — Htilde (A B^T) with the adjoint trajectory Q
  truncated by ``timefactors.streaming`` (chunks of s steps, tolerance tol,
  cap rmax) and returned as factors (tau R^{-1} W_Q, V_Q); with tol = 0
  (nothing discarded) it is the exact product;
* ``lr_arnoldi`` — Algorithm 1 on factored vectors: w = Htilde v_j (factored);
  for i = 1..j: h_ij = <w, v_i>, w <- truncate(w - h_ij v_i) (Eq.
  (lanczos2): the factors are concatenated, then truncated); h_{j+1,j} =
  ||w||_F, v_{j+1} = w / h_{j+1,j}. Returns H, the ranks of the vectors and
  the Ritz values (``lowrank.ritz_nonsym``).
"""
from __future__ import annotations

import numpy as np

from . import lowrank, timefactors


def forward_source(P, U):
    """F U for a source U (nx, nt) -> (n_data,)."""
    U = np.asarray(U, dtype=np.float64).reshape(P.nx, P.nt)
    y = np.zeros(P.nx)
    D = np.zeros(P.n_data)
    for n in range(1, P.nt + 1):
        y = P.step(y + P.tau * U[:, n - 1])
        k = P._obs_index.get(n)
        if k is not None:
            D[k * P.n_obs:(k + 1) * P.n_obs] = P.B @ y
    return D


def adjoint_source(P, D):
    """F^T D -> (nx, nt) = tau [q_1 .. q_nt]."""
    return P.tau * lowrank.adjoint_trajectory(P, D)


def prior_half_st(P, U):
    return P.prior_half(np.asarray(U, dtype=np.float64).reshape(P.nx, P.nt))


def hessian_st(P, U):
    """Htilde U (nx, nt) for the space-time parameter."""
    Z = prior_half_st(P, U)
    return prior_half_st(P, adjoint_source(P, forward_source(P, Z) / P.sigma ** 2))


def hessian_st_explicit(P):
    """Dense Htilde on vec(U) (tiny sizes only), symmetrised."""
    N = P.nx * P.nt
    H = np.zeros((N, N))
    for c in range(N):
        e = np.zeros(N)
        e[c] = 1.0
        H[:, c] = hessian_st(P, e.reshape(P.nt, P.nx).T).T.reshape(-1)
    return 0.5 * (H + H.T)


def vec(U):
    """vec(U): the columns u_1 .. u_nt stacked."""
    return np.asarray(U).T.reshape(-1)


def truncate(A, B, tol, rmax):
    """Rounded factors of A B^T (see the module docstring)."""
    if A.shape[1] == 0:
        return A, B
    Qa, Ra = np.linalg.qr(A)
    Qb, Rb = np.linalg.qr(B)
    Uc, s, Zt = np.linalg.svd(Ra @ Rb.T)
    fro2 = float(np.sum(s ** 2))
    tail = np.concatenate([np.cumsum((s ** 2)[::-1])[::-1], [0.0]])
    r = int(np.argmax(tail <= tol ** 2 * fro2))
    if s.size and s[0] > 0.0:
        r = max(r, 1)
    r = min(r, rmax)
    return (Qa @ Uc[:, :r]) * s[:r], Qb @ Zt[:r].T


def dot(X, Y):
    return float(np.sum((X[0].T @ Y[0]) * (X[1].T @ Y[1])))


def lr_hessian_apply(P, A, B, tol, rmax, s):
    """Htilde (A B^T) with the adjoint trajectory truncated; returns factors."""
    Z = P.prior_half(A) @ B.T
    D = forward_source(P, Z) / P.sigma ** 2
    Q = lowrank.adjoint_trajectory(P, D)
    Wq, Vq, _ = timefactors.streaming(Q, s, tol, rmax)
    return P.tau * P.prior_half(Wq), Vq


def lr_arnoldi(P, A0, B0, m, tol, rmax, s):
    """m steps of Algorithm 1 on factored vectors. Returns (H, ranks, basis)
    with basis the list of (A, B) factors of v_1 .. v_{m+1}."""
    nrm = np.sqrt(dot((A0, B0), (A0, B0)))
    basis = [(A0 / nrm, B0)]
    H = np.zeros((m + 1, m))
    ranks = []
    for j in range(m):
        Aw, Bw = lr_hessian_apply(P, basis[j][0], basis[j][1], tol, rmax, s)
        for i in range(j + 1):
            H[i, j] = dot((Aw, Bw), basis[i])
            Aw, Bw = truncate(np.hstack([Aw, -H[i, j] * basis[i][0]]), np.hstack([Bw, basis[i][1]]), tol, rmax)
        H[j + 1, j] = np.sqrt(max(dot((Aw, Bw), (Aw, Bw)), 0.0))
        ranks.append(Aw.shape[1])
        if H[j + 1, j] == 0.0:
            return H[:j + 2, :j + 1], ranks, basis
        basis.append((Aw / H[j + 1, j], Bw))
    return H, ranks, basis
