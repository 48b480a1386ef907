"""Low-rank-in-time trajectory factors Y = [y_1 ... y_nt] ~ W V^T (FP64).

Sec. 3 stores state, control and adjoint trajectories as W_Y V_Y^T with small
rank; Sec. 4 controls the rank of such factored sums by truncation (skinny QR
or truncated SVD). Two restatements:

* ``truncate`` — the definition: SVD of the full trajectory, keep the
  smallest rank r whose discarded Frobenius tail is at most tol*||Y||_F
  (optimal by Eckart-Young), capped at rmax.
* ``streaming`` — the recompression the GPU performs while stepping: after
  every chunk of s new columns, orthogonalise the chunk against the current
  space factor W (orthonormal), take a thin QR of the remainder, form the
  small core [[diag(sig), C], [0, R]], take its SVD and keep the leading
  singular triplets whose discarded tail is at most (tol/K) times the core's
  Frobenius norm, K = number of chunks. By the triangle inequality the total
  error is at most tol * ||Y||_F.
"""
from __future__ import annotations

import math

import numpy as np


def _rank_for(sv: np.ndarray, thresh_sq: float, rmax: int) -> int:
    """Smallest r with sum_{i>=r} sv_i^2 <= thresh_sq, capped at rmax (and >= 1
    when any singular value is nonzero)."""
    tail = np.concatenate([np.cumsum((sv ** 2)[::-1])[::-1], [0.0]])
    r = int(np.argmax(tail <= thresh_sq))
    if sv.size and sv[0] > 0.0:
        r = max(r, 1)
    return min(r, rmax)


def truncate(Y: np.ndarray, tol: float, rmax: int):
    """Optimal truncation: returns (W, V, err) with W = U_r diag(s_r), V = Z_r."""
    U, s, Zt = np.linalg.svd(Y, full_matrices=False)
    fro2 = float(np.sum(s ** 2))
    r = _rank_for(s, tol ** 2 * fro2, rmax)
    W = U[:, :r] * s[:r]
    V = Zt[:r].T
    err = math.sqrt(float(np.sum(s[r:] ** 2)))
    return W, V, err


def streaming(Y: np.ndarray, s: int, tol: float, rmax: int):
    """Streaming recompression over chunks of s columns of Y (nx, nt).

    Returns (W, V, rank history) with Y ~ W V^T, W = Q diag(sig).
    """
    nx, nt = Y.shape
    K = int(math.ceil(nt / s))
    tol_k = tol / K
    Q = np.zeros((nx, 0))
    sig = np.zeros(0)
    V = np.zeros((0, 0))
    ranks = []
    for c0 in range(0, nt, s):
        Bk = Y[:, c0:c0 + s]
        sk = Bk.shape[1]
        r = Q.shape[1]
        # block classical Gram-Schmidt, twice
        C = Q.T @ Bk
        Bp = Bk - Q @ C
        C2 = Q.T @ Bp
        Bp = Bp - Q @ C2
        C = C + C2
        Q2, R2 = np.linalg.qr(Bp)
        core = np.zeros((r + sk, r + sk))
        core[:r, :r] = np.diag(sig)
        core[:r, r:] = C
        core[r:, r:] = R2
        Uc, sc, Zct = np.linalg.svd(core)
        fro2 = float(np.sum(sc ** 2))
        rn = _rank_for(sc, tol_k ** 2 * fro2, rmax)
        Q = np.hstack([Q, Q2]) @ Uc[:, :rn]
        sig = sc[:rn]
        Vext = np.zeros((V.shape[0] + sk, r + sk))
        Vext[:V.shape[0], :r] = V
        Vext[V.shape[0]:, r:] = np.eye(sk)
        V = Vext @ Zct[:rn].T
        ranks.append(rn)
    return Q * sig, V, ranks
