"""A space-time source as the parameter (Sec. 4) and Algorithm 1 on low-rank
space-time vectors (Eq. (lanczos1)-(lanczos2)) against the oracle
(``oracle.spacetime``):

* the factored Hessian product (forward sweep with the factored source,
  adjoint sweep storing its trajectory, streaming truncation, prior factors)
  against the oracle's on the same factors, as dense nx x nt matrices, with
  nothing truncated (exact) and at a tolerance (same streaming recompression,
  same ranks), for the heat and the convection-diffusion operator;
* Algorithm 1 on factored vectors: the leading columns of H against the
  oracle's run from the same start factors, the ranks of the vectors, and the
  Ritz values above a threshold against the dense eigenvalues of the
  explicit space-time Hessian.
"""
import numpy as np
import pytest

import synth
from oracle import lowrank as olr
from oracle import spacetime as ost
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


def _spec(pde="heat", n=15, nt=60, obs_every=12, n_obs=4):
    spec = synth.small_spec(dim=2, n=n, nt=nt, obs_every=obs_every, n_obs=n_obs, sigma=1e-2, alpha=0.05, seed=91)
    if pde == "convdiff":
        spec.pde, spec.conv_nu, spec.wind = "convdiff", 1e-2, (0.0, 1.0, 0.0)
    return spec


@pytest.mark.parametrize("precision", [lrp.LRP_FP64, lrp.LRP_MIXED])
@pytest.mark.parametrize("pde", ["heat", "convdiff"])
@pytest.mark.parametrize("tol,rmax", [(1e-15, 64), (1e-6, 40)])
def test_st_hessian_apply_matches_oracle(precision, pde, tol, rmax):
    """nt = 60 observed every 12th step by 4 sensors: the adjoint trajectory
    has numerical rank 24 (heat) / 30 (convection-diffusion) at 1e-6, with
    the singular values at the cut a factor 2-3 apart (a stable rank
    decision); at tolerance 1e-15 with the rank cap 64 >= nt nothing of
    significance is discarded and the product is the exact one."""
    if pde == "convdiff" and precision == lrp.LRP_MIXED:
        pytest.skip("the convection-diffusion operator runs on the FP64 path")
    spec = _spec(pde)
    P = OProblem(spec)
    s = 8
    G = lrp.lrp_setup_problem(spec, precision=precision, time_trunc_tol=tol, time_rank_max=rmax, time_chunk=s)
    r = synth.rng(92)
    A = r.standard_normal((P.nx, 3))
    B = r.standard_normal((P.nt, 3))
    Ao, Bo, st = lrp.lrp_st_hessian_apply(G, A, B)
    assert st["status"] == lrp.LRP_OK, st
    got = Ao @ Bo.T
    if tol < 1e-14:
        want = ost.hessian_st(P, A @ B.T)
    else:
        Aw, Bw = ost.lr_hessian_apply(P, A, B, tol, rmax, s)
        want = Aw @ Bw.T
        assert Ao.shape[1] == Aw.shape[1]
    assert relerr(got, want) < TOL[precision], st


@pytest.mark.parametrize("precision", [lrp.LRP_FP64, lrp.LRP_MIXED])
def test_st_arnoldi_matches_oracle(precision):
    spec = _spec(n=7, nt=16, obs_every=2, n_obs=10)
    P = OProblem(spec)
    tol, rmax, s = 1e-8, 40, 4
    G = lrp.lrp_setup_problem(spec, precision=precision, time_trunc_tol=tol, time_rank_max=rmax, time_chunk=s)
    r = synth.rng(93)
    A0 = r.standard_normal((P.nx, 2))
    B0 = r.standard_normal((P.nt, 2))
    Hd = ost.hessian_st_explicit(P)
    lam = np.sort(np.linalg.eigvalsh(Hd))[::-1]
    eps = 0.5 * (lam[5] + lam[6])
    res = lrp.lrp_st_arnoldi(G, 60, eig_tol=TOL[precision] / 10, eig_threshold=eps, W0=A0, V0=B0)
    st = res["stats"]
    assert st["status"] == lrp.LRP_OK, st
    theta = res["theta"]
    above = theta.real >= eps
    assert int(np.sum(above)) == 6
    assert np.max(np.abs(theta.real[above] - lam[:6])) <= (TOL[precision] + 100 * tol) * lam[0]
    Ho, ranks_o, _ = ost.lr_arnoldi(P, A0, B0, 6, tol, rmax, s)
    assert np.max(np.abs(res["H"][:7, :6] - Ho)) <= 10 * TOL[precision] * lam[0]
    if precision == lrp.LRP_FP64:
        assert list(res["ranks"][:6]) == ranks_o
