"""Alternating low-rank solve of the space-time system (Sec. 6.1, Eq.
(st_pde), (amen_1), (amen_2), (pre_1)), FP64. TEST INFRASTRUCTURE ONLY (see
the package docstring).

The implicit-Euler sweep y_n = A^{-1} (y_{n-1} + f_n), n = 1..nt, A = I + tau L
(y_0 = 0; an initial condition u enters as f_1 = u), is the space-time system
A Y - Y S^T = F with Y = [y_1 .. y_nt], F = [f_1 .. f_nt] and (Y S^T)[:, n] =
y_{n-1} (Eq. (st_pde) with M = I, scaled by tau). In the two-factor format
Y ~ W V^T (nx x r, nt x r) the alternating solve takes, in turn:

* the space step (Eq. (amen_1)): V fixed with orthonormal columns, the
  Galerkin projection onto span(V) in time: A W - W T = F V with
  T = V^T S^T V, T[i, j] = sum_{n >= 1} V[n-1, i] V[n, j] (an nx r system;
  here solved exactly by the Bartels-Stewart routine of SciPy, a library
  step; the GPU solves it by right-preconditioned GMRES with the block
  diagonal of Eq. (pre_1), blocks (1 - T[j, j]) I + tau L);
* the time step (Eq. (amen_2)): W orthonormalised to Q, the Galerkin
  projection onto span(Q) in space: Ahat z_n - z_{n-1} = Q^T f_n with
  Ahat = Q^T A Q (r x r), z_0 = 0, solved directly step by step; then
  Y = Q Z^T and V = the orthonormalised Z.

``als_solve`` runs a fixed number of such sweeps from a given orthonormal
start V0 and returns the factors and the relative residual
||A Y - Y S^T - F||_F / ||F||_F after each sweep.

``als_adjoint`` solves the adjoint system A^T q_n = q_{n+1} + f_n,
n = nt..1, q_{nt+1} = 0 (the backward recursion of the Hessian's adjoint
sweep) as the same system with A^T in reversed time.

``als_hessian_apply`` is the prior-preconditioned Hessian product (Sec. 2
Eq. (prior_pre), Sec. 6.1 Eq. (misfit)) with both space-time solves done by
``als_solve`` at rank r from the first r unit time vectors:
z = Gamma_prior^{1/2} x; the state Y ~ W_Y V_Y^T of A Y - Y S^T = z e_1^T;
the adjoint's source at the observed steps n, B^T B y_n / sigma^2, i.e. the
factors (B^T B W_Y / sigma^2, V_Y with the unobserved rows zeroed); the
adjoint solution's first step q_1; the result Gamma_prior^{1/2} q_1.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def shift_gram(V):
    """T = V^T S^T V: T[i, j] = sum_{n>=1} V[n-1, i] V[n, j]."""
    return V[:-1].T @ V[1:]


def residual(A, W, V, Wf, Vf):
    """||A W V^T - W (S V)^T - Wf Vf^T||_F / ||Wf Vf^T||_F (dense)."""
    Y = W @ V.T
    YS = np.zeros_like(Y)
    YS[:, 1:] = Y[:, :-1]
    F = Wf @ Vf.T
    return float(np.linalg.norm(A @ Y - YS - F) / np.linalg.norm(F))


def time_step(Ahat, G):
    """Z (nt x r) with Ahat z_n - z_{n-1} = G[:, n], z_{-1} = 0 (G: r x nt)."""
    r, nt = G.shape
    Z = np.zeros((nt, r))
    lu = sla.lu_factor(Ahat)
    z = np.zeros(r)
    for n in range(nt):
        z = sla.lu_solve(lu, z + G[:, n])
        Z[n] = z
    return Z


def als_solve(A, Wf, Vf, V0, sweeps):
    """sweeps alternating sweeps from the orthonormal start V0 (nt x r).
    A: dense nx x nx. Returns (W, V, residuals) with Y ~ W V^T."""
    V = V0.copy()
    res = []
    W = None
    for _ in range(sweeps):
        T = shift_gram(V)
        G = Wf @ (Vf.T @ V)
        # A W - W T = G  <=>  A W + W (-T) = G
        W = sla.solve_sylvester(A, -T, G)
        Q, _ = np.linalg.qr(W)
        Ahat = Q.T @ A @ Q
        Z = time_step(Ahat, (Q.T @ Wf) @ Vf.T)
        Vn, Rz = np.linalg.qr(Z)
        W = Q @ Rz.T
        V = Vn
        res.append(residual(A, W, V, Wf, Vf))
    return W, V, res


def als_adjoint(A, Wf, Vf, V0, sweeps):
    """A^T q_n = q_{n+1} + f_n (n = nt..1, q_{nt+1} = 0), F = Wf Vf^T with
    row n-1 of Vf and V0 = step n. Returns (W, V, residuals), Q ~ W V^T in
    natural time order."""
    W, Vr, res = als_solve(A.T.copy(), Wf, Vf[::-1].copy(), V0[::-1].copy(), sweeps)
    return W, Vr[::-1].copy(), res


def als_hessian_apply(P, x, r, sweeps, A=None, misfit_only=False):
    """Htilde x (H_mis x) with both solves by ``als_solve`` at rank r and
    ``sweeps`` sweeps from the unit vectors e_1..e_r in each solve's own
    time direction. P: an oracle Problem; A: its dense time-step matrix
    (built if None). Returns (result, info) with the final residuals."""
    A = P.K.toarray() if A is None else A
    x = np.asarray(x, dtype=np.float64).reshape(-1)
    nt = P.nt
    z = x if misfit_only else P.prior_half(x)
    start = np.eye(nt)[:, :r]
    e1 = np.zeros((nt, 1))
    e1[0, 0] = 1.0
    Wy, Vy, res_f = als_solve(A, z[:, None], e1, start, sweeps)
    B = P.B.toarray()
    Wa = B.T @ (B @ Wy) / P.sigma ** 2
    mask = np.zeros((nt, 1))
    for n in P.steps:
        mask[n - 1, 0] = 1.0
    Va = Vy * mask
    # the adjoint starts from e_1..e_r of its own (reversed) time
    Wq, Vq, res_a = als_adjoint(A, Wa, Va, start[::-1].copy(), sweeps)
    q1 = Wq @ Vq[0, :]
    out = q1 if misfit_only else P.prior_half(q1)
    return out, dict(res_f=res_f, res_a=res_a)
