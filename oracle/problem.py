"""Forward map, adjoint and prior-preconditioned misfit Hessian (FP64).

The parameter u is the initial condition of y_t + L y = 0 (Sec. 6, Eq. (pde));
L = -div(kappa grad) (the heat equation) or -nu Laplace + w . grad (the
convection-diffusion equation of Sec. 6.2, upwind; not symmetric, so the
adjoint steps solve with (I + tau L)^T).
Implicit Euler with tau = T/nt gives (I + tau L) y_n = y_{n-1}, y_0 = u
(one block row of the space-time system Eq. (st_pde) with M = I), so
y_n = S^n u with S = (I + tau L)^{-1}.

* F u     = [B y_n]_{n in observed steps}         (the parameter-to-observable
  map A of Sec. 2 realised as B K^{-1} C, Sec. 6 Eq. (dis_obj))
* F^T w   = sum_n (S^T)^n B^T w_n, evaluated by the backward recursion
  q_{nt+1} = 0, q_n = (I + tau L)^{-T} (q_{n+1} + B^T w_n), F^T w = q_1
  (w_n = 0 at unobserved steps)
* Gamma_noise = sigma^2 I, Gamma_prior = R^{-2} with R = I + alpha L0
  (L0: the constant-coefficient Laplacian), so Gamma_prior^{1/2} = R^{-1};
  or (prior_kind 1, the prior of the experiments of Sec. 6.1) Gamma_prior =
  gamma I, i.e. R = gamma^{-1/2} I
* H_mis = F^T F / sigma^2,  Htilde = R^{-1} H_mis R^{-1}
  (Sec. 2 Eq. (prior_pre); Sec. 6.1 Eq. (misfit))

Observation vectors are laid out step-major: entry (k, s) of step k (k-th
observed step) and sensor s sits at row k*n_obs + s.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.sparse.linalg import cg, splu

from .operators import convection_diffusion, laplacian, shifted
from .observe import observation_matrix, observed_steps


class _CGSolver:
    """x = A^{-1} b for a symmetric positive definite sparse A by conjugate
    gradients with the Jacobi preconditioner, to a relative residual of
    1e-14, column by column (a plain library step in place of a sparse LU
    whose fill-in is prohibitive on 3D grids of 63^3 nodes). Both operators
    solved here, I + tau L and I + alpha L0, are symmetric (L is in flux
    form), so the transposed solve is the same solve."""

    RTOL = 1e-14

    def __init__(self, A):
        self.A = sp.csr_matrix(A)
        self.M = sp.diags(1.0 / self.A.diagonal())

    def solve(self, B, trans="N"):
        B = np.asarray(B, dtype=np.float64)
        cols = B.reshape(B.shape[0], -1)
        out = np.empty_like(cols)
        for j in range(cols.shape[1]):
            if not np.any(cols[:, j]):
                out[:, j] = 0.0
                continue
            x, info = cg(self.A, cols[:, j], rtol=self.RTOL, atol=0.0, M=self.M, maxiter=100000)
            if info != 0:
                raise RuntimeError(f"oracle CG did not reach {self.RTOL} (info {info})")
            out[:, j] = x
        return out.reshape(B.shape)


class _ScaledIdentity:
    """x = s b (Gamma_prior^{1/2} = sqrt(gamma) I)."""

    def __init__(self, s):
        self.s = float(s)

    def solve(self, B, trans="N"):
        return self.s * np.asarray(B, dtype=np.float64)


class Problem:
    """All operators of one inverse problem. ``spec`` is any object with the
    attributes of ``synth.ProblemSpec`` (dim, n, nt, T, prior_alpha, sigma,
    obs_every, sensors, kappa). ``solver``: "lu" (sparse LU factors of
    I + tau L and I + alpha L0, the default) or "cg" (conjugate gradients to
    a relative residual of 1e-14, for grids too large to factor)."""

    def __init__(self, spec, solver: str = "lu"):
        self.spec = spec
        self.dim = int(spec.dim)
        self.n = int(spec.n)
        self.nx = self.n ** self.dim
        self.nt = int(spec.nt)
        self.tau = float(spec.T) / self.nt
        self.alpha = float(spec.prior_alpha)
        self.sigma = float(spec.sigma)
        self.pde = str(getattr(spec, "pde", "heat") or "heat")
        if self.pde == "convdiff":
            # Sec. 6.2: L = -nu Laplace + w . grad (upwind); not symmetric
            self.L = convection_diffusion(self.n, self.dim, float(spec.conv_nu), spec.wind)
        else:
            self.L = laplacian(self.n, self.dim, spec.kappa)
        self.L0 = laplacian(self.n, self.dim, None)
        self.prior_kind = int(getattr(spec, "prior_kind", 0) or 0)
        if self.prior_kind == 1:
            self.gamma = float(spec.prior_gamma)
            self.R = (sp.identity(self.nx, format="csc") / np.sqrt(self.gamma)).tocsc()
        else:
            self.R = shifted(self.L0, self.alpha)
        self.K = shifted(self.L, self.tau)
        if solver == "lu":
            self._R_lu = splu(self.R)
            self._K_lu = splu(self.K)
        elif solver == "cg":
            if self.pde != "heat":
                raise ValueError("the CG solves need a symmetric operator")
            self._R_lu = _CGSolver(self.R)
            self._K_lu = _CGSolver(self.K)
        else:
            raise ValueError(solver)
        if self.prior_kind == 1:
            self._R_lu = _ScaledIdentity(np.sqrt(self.gamma))
        self.B = observation_matrix(self.n, self.dim, spec.sensors)
        self.n_obs = self.B.shape[0]
        self.steps = observed_steps(self.nt, int(spec.obs_every))
        self._obs_index = {s: k for k, s in enumerate(self.steps)}
        self.n_data = self.n_obs * len(self.steps)

    # -- prior -----------------------------------------------------------
    def prior_half(self, X):
        """Gamma_prior^{1/2} X = R^{-1} X."""
        return self._R_lu.solve(np.asarray(X, dtype=np.float64))

    # -- forward / adjoint ------------------------------------------------
    def step(self, Y):
        """One implicit-Euler step: solve (I + tau L) y_n = y_{n-1}."""
        return self._K_lu.solve(Y)

    def step_adjoint(self, Y):
        """(I + tau L)^{-T} Y."""
        return self._K_lu.solve(Y, trans="T")

    def trajectory(self, u):
        """Y = [y_1, ..., y_nt] for one initial condition u (nx,) -> (nx, nt)."""
        y = np.asarray(u, dtype=np.float64).copy()
        out = np.empty((self.nx, self.nt))
        for n in range(1, self.nt + 1):
            y = self.step(y)
            out[:, n - 1] = y
        return out

    def forward(self, U):
        """F U for a block U (nx, b) -> (n_data, b)."""
        U = np.asarray(U, dtype=np.float64)
        squeeze = U.ndim == 1
        Y = U.reshape(self.nx, -1).copy()
        D = np.zeros((self.n_data, Y.shape[1]))
        for n in range(1, self.nt + 1):
            Y = self.step(Y)
            k = self._obs_index.get(n)
            if k is not None:
                D[k * self.n_obs:(k + 1) * self.n_obs] = self.B @ Y
        return D[:, 0] if squeeze else D

    def adjoint(self, W):
        """F^T W for a block W (n_data, b) -> (nx, b) by the backward recursion."""
        W = np.asarray(W, dtype=np.float64)
        squeeze = W.ndim == 1
        W = W.reshape(self.n_data, -1)
        Q = np.zeros((self.nx, W.shape[1]))
        Bt = self.B.T.tocsr()
        for n in range(self.nt, 0, -1):
            k = self._obs_index.get(n)
            rhs = Q if k is None else Q + Bt @ W[k * self.n_obs:(k + 1) * self.n_obs]
            Q = self.step_adjoint(rhs)
        return Q[:, 0] if squeeze else Q

    # -- Hessians -----------------------------------------------------------
    def misfit_apply(self, X):
        """H_mis X = F^T Gamma_noise^{-1} F X."""
        return self.adjoint(self.forward(X) / self.sigma ** 2)

    def hessian_apply(self, X):
        """Htilde X = R^{-1} F^T F R^{-1} X / sigma^2."""
        return self.prior_half(self.misfit_apply(self.prior_half(X)))

    def forward_explicit(self):
        """The dense (n_data, nx) matrix of F (tiny sizes only)."""
        return self.forward(np.eye(self.nx))

    def hessian_explicit(self):
        """Dense Htilde, symmetrised (tiny sizes only)."""
        F = self.forward_explicit()
        Rinv = self.prior_half(np.eye(self.nx))
        G = F @ Rinv
        H = G.T @ G / self.sigma ** 2
        return 0.5 * (H + H.T)

    def misfit_explicit(self):
        F = self.forward_explicit()
        H = F.T @ F / self.sigma ** 2
        return 0.5 * (H + H.T)
