"""The allocation-free Hessian apply (for callers that cannot allocate
device memory while they run) gives the same result as lrp_hessian_apply,
call after call. It goes through the C ABI like every other GPU test. This
file is named to be collected last."""
import numpy as np
import pytest

import synth

lrp = pytest.importorskip("paper_1703_05638_gb300")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_05638_gb300 import build
    build.build()
    lrp.load()


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-6)])
def test_noalloc_matches_hessian_apply(precision, tol):
    spec = synth.small_spec(dim=2, n=31, nt=16, obs_every=2, n_obs=10, with_kappa=True, seed=9)
    G = lrp.lrp_setup_problem(spec, precision=precision, team_ctas=2, team_cols=2)
    X = torch.from_numpy(synth.normal_block(G.nx, 5, 4)).cuda()
    ref, _ = lrp.lrp_hessian_apply(G, X)
    ref = ref.cpu().numpy()
    scale = np.abs(ref).max()
    for _ in range(2):
        Y, st = lrp.lrp_hessian_apply_noalloc(G, X)
        err = np.abs(Y.cpu().numpy() - ref).max() / scale
        assert err < tol, (err, st)


def test_noalloc_band_kernel():
    """A 2D problem with kappa = 1 in the mixed path and one column per
    cluster runs the shared-memory band kernel; on the fixed workspace it
    gives the same result as the ordinary apply, call after call."""
    spec = synth.small_spec(dim=2, n=63, nt=12, obs_every=2, n_obs=10, seed=19)
    G = lrp.lrp_setup_problem(spec, precision=1, team_ctas=4, team_cols=1)
    X = torch.from_numpy(synth.normal_block(G.nx, 3, 7)).cuda()
    ref, _ = lrp.lrp_hessian_apply(G, X)
    assert lrp.lrp_problem_tuning(G)["last_kernel"] == 2
    ref = ref.cpu().numpy()
    scale = np.abs(ref).max()
    for _ in range(2):
        Y, st = lrp.lrp_hessian_apply_noalloc(G, X)
        assert lrp.lrp_problem_tuning(G)["last_kernel"] == 2
        err = np.abs(Y.cpu().numpy() - ref).max() / scale
        assert err < 1e-6, (err, st)


def test_noalloc_rejects_host_arrays_and_oversize():
    spec = synth.small_spec(dim=2, n=15, nt=8, obs_every=2, n_obs=4, seed=2)
    G = lrp.lrp_setup_problem(spec, precision=1)
    with pytest.raises(ValueError):
        lrp.lrp_hessian_apply_noalloc(G, np.zeros((G.nx, 1)))
    big = lrp.lrp_setup_problem(synth.workload("heat2d_127"), precision=0, team_cols=1)
    X = torch.zeros((big.nx, 64), dtype=torch.float64, device="cuda")
    with pytest.raises(lrp.LrpError) as e:
        lrp.lrp_hessian_apply_noalloc(big, X)
    assert e.value.status == lrp.LRP_EINVAL
    assert "bytes" in str(e.value)
