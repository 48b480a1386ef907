"""FP64 CPU oracle for the low-rank posterior-covariance method.

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, obviously-correct
restatement of what the GPU path computes, written from the paper (Benner,
Qiu, Stoll, "Low-rank computation of posterior covariance matrices in
Bayesian inverse problems"). It exists to check the CUDA library. Only the
test suite, the smoke check and the benchmark's CPU-baseline leg may import
it; the product path never does, and it shares no code with the library.

Modules and the passages they follow:

* ``operators``  — the spatial operator L = -div(kappa grad) by finite
  differences with zero Dirichlet data (Sec. 6, Eq. (pde) with L=-Laplace),
  the implicit-Euler step matrix I + tau*L (Sec. 6.1, Eq. (st_pde) realised
  step by step with M = I), the prior Gamma_prior = (I + alpha*L0)^-2.
* ``observe``    — the sparse observation operator B (Sec. 6, Eq. (obj) and
  (dis_obj)) as point sensors interpolated bilinearly/trilinearly.
* ``problem``    — forward map F (parameter -> observations), adjoint F^T,
  prior-preconditioned misfit Hessian (Sec. 2 Eq. (prior_pre); Sec. 6.1
  Eq. (misfit)), explicit matrices on tiny sizes.
* ``spectrum``   — dense eigendecomposition of the explicit Hessian, and the
  Arnoldi process with modified Gram-Schmidt (Sec. 4, Algorithm 1).
* ``posterior``  — exact posterior covariance (Sec. 2 Eq. (postcov1); Sec. 6
  Eq. (postvar)), the Sherman-Morrison-Woodbury low-rank form (Sec. 2), the
  posterior mean, pointwise variance and samples.
* ``lowrank``    — the low-rank matrix-vector product of Sec. 4
  Algorithm 1 (state and adjoint trajectories truncated to eps_0, the
  adjoint's data observed from the truncated state), the Ritz values of a
  nonsymmetric Hessenberg matrix and the threshold-stopped Arnoldi run.
* ``spacetime``  — a space-time source as the parameter (Sec. 4): its
  forward map, adjoint and Hessian, low-rank space-time vectors (truncation,
  inner product) and Algorithm 1 on them (Eq. (lanczos1)-(lanczos2)).
* ``als``        — the alternating low-rank solve of the space-time system
  (Sec. 6.1, Eq. (st_pde), (amen_1), (amen_2)): space steps by Galerkin
  projection in time (a Sylvester equation), time steps by Galerkin
  projection in space (block forward substitution).
* ``timefactors``— the low-rank-in-time factorisation Y ~ W V^T (Sec. 3) by
  truncated SVD of the full trajectory, and the streaming recompression the
  GPU uses (thin QR of [W | new columns], small SVD, truncation; Sec. 4).

Parity: every function is pinned by a test in ``tests/test_oracle_*.py``
against a closed form, an invariant or brute force, except where its
docstring says "parity unpinned".
"""
