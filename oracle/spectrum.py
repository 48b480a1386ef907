"""Leading spectrum of the prior-preconditioned misfit Hessian (FP64).

* ``eig_dense`` — the definition: all eigenpairs of the explicit symmetric
  Htilde (tiny sizes), sorted by decreasing eigenvalue.
* ``arnoldi_mgs`` — the Arnoldi process of Sec. 4, Algorithm 1: for each
  step, apply the operator to the newest basis vector, orthogonalise the
  result against every previous basis vector one at a time (modified
  Gram-Schmidt), record the coefficients in the Hessenberg matrix, normalise.
  The Ritz values are the eigenvalues of the leading square block of H.
* ``eigsh_top`` — SciPy's ARPACK Lanczos on a LinearOperator (matrix-free
  cross-check at medium sizes).
"""
from __future__ import annotations

import numpy as np
from scipy.sparse.linalg import LinearOperator, eigsh


def eig_dense(H: np.ndarray):
    """Eigenpairs of a symmetric matrix, eigenvalues in decreasing order."""
    lam, V = np.linalg.eigh(0.5 * (H + H.T))
    order = np.argsort(lam)[::-1]
    return lam[order], V[:, order]


def arnoldi_mgs(apply, v1: np.ndarray, m: int):
    """m steps of Algorithm 1 (Sec. 4) with modified Gram-Schmidt.

    apply: x (nx,) -> operator times x. Returns (V, H) with V of shape
    (nx, m+1) (orthonormal columns) and H of shape (m+1, m) upper Hessenberg,
    so that apply(V[:, :m]) = V @ H up to rounding. Stops early (returning
    truncated arrays) if the new vector vanishes.
    """
    nx = v1.shape[0]
    V = np.zeros((nx, m + 1))
    H = np.zeros((m + 1, m))
    V[:, 0] = v1 / np.linalg.norm(v1)
    for j in range(m):
        w = apply(V[:, j])
        for i in range(j + 1):
            H[i, j] = w @ V[:, i]
            w = w - H[i, j] * V[:, i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] == 0.0:
            return V[:, :j + 1], H[:j + 1, :j + 1]
        V[:, j + 1] = w / H[j + 1, j]
    return V, H


def ritz_from_arnoldi(V: np.ndarray, H: np.ndarray, k: int):
    """Top-k Ritz values/vectors of the Arnoldi factorisation (real parts;
    the operator here is symmetric, so H's square block is symmetric up to
    rounding)."""
    m = H.shape[1]
    Hm = H[:m, :m]
    lam, S = np.linalg.eig(Hm)
    lam = lam.real
    S = S.real
    order = np.argsort(lam)[::-1][:k]
    Y = V[:, :m] @ S[:, order]
    Y /= np.linalg.norm(Y, axis=0)
    return lam[order], Y


def eigsh_top(apply, nx: int, k: int, tol: float = 1e-13, v0=None):
    """Top-k eigenpairs by ARPACK on a LinearOperator (decreasing order)."""
    op = LinearOperator((nx, nx), matvec=lambda x: apply(x.reshape(-1)), dtype=np.float64)
    lam, V = eigsh(op, k=k, which="LA", tol=tol, v0=v0)
    order = np.argsort(lam)[::-1]
    return lam[order], V[:, order]
