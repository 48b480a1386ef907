"""BF16 storage of the multigrid vectors (mg_bf16, mixed path, generic sweep
kernel): the smoother iterates and coarse right-hand sides of the levels in
global memory are rounded to BF16, the arithmetic stays FP32 inside FP64
iterative refinement. The V-cycle is then a slightly different operator in
every application, so the test is whether the solves still converge to the
path's tolerance: element by element against the oracle at the mixed path's
1e-6 (3D with the kappa field, 2D with several columns per team), the
solves' own statistics (no LRP_ENOCONV), and the same columns with FP32
storage agreeing to the same tolerance.
"""
import numpy as np
import pytest

import synth
from oracle.problem import Problem as OProblem

lrp = pytest.importorskip("paper_1703_05638_gb300")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_05638_gb300 import build
    build.build()
    lrp.load()


def relerr(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(np.asarray(b))), 1e-300))


@pytest.mark.parametrize("case", ["heat3d_31_kappa", "heat2d_31_two_cols"])
def test_bf16_smoothing_matches_oracle(case):
    if case == "heat3d_31_kappa":
        # tau = 1e-3 as in the 3D workload, 400 sensors every 10th step
        spec = synth.workload("heat3d_63", n=31, nt=50, T=0.05)
        spec.kappa = synth.kappa_faces(31, 3, spec.seed + 7)
        tuning = dict(team_ctas=4, team_cols=1)
    else:
        spec = synth.small_spec(dim=2, n=31, nt=40, obs_every=4, n_obs=12, sigma=1e-2, alpha=0.05, seed=111)
        tuning = dict(team_ctas=2, team_cols=2)
    P = OProblem(spec)
    U = synth.normal_block(P.nx, 3, 112)
    out = {}
    for bf in (0, 1):
        G = lrp.lrp_setup_problem(spec, precision=lrp.LRP_MIXED, mg_bf16=bf, **tuning)
        H, st = lrp.lrp_hessian_apply(G, U)
        assert st["status"] == lrp.LRP_OK, (bf, st, lrp.lrp_last_error())
        assert lrp.lrp_problem_tuning(G)["last_kernel"] == 1
        assert st["max_rel_residual"] <= 1e-10, st
        out[bf] = (H, st)
        D, st = lrp.lrp_forward_observe(G, U)
        assert st["status"] == lrp.LRP_OK
        assert relerr(D, P.forward(U)) < TOL, (bf, st)
        G.close()
    ref = P.hessian_apply(U)
    assert relerr(out[1][0], ref) < TOL, out[1][1]
    assert relerr(out[1][0], out[0][0]) < TOL
