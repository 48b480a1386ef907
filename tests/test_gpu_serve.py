"""Posterior-query server on the GPU: every result matches the oracle's
low-rank formulas (Sec. 2, SMW form, eigenvalues rescaled per request noise
level) and is the same whether the request was served alone or batched with
others; a tight memory budget forces evictions without changing results."""
import numpy as np
import pytest

import synth
from oracle import posterior as opost
from oracle import spectrum as ospec
from oracle.problem import Problem as OProblem

lrp = pytest.importorskip("paper_1703_05638_gb300")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

KIND = None


def relerr(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_05638_gb300 import build
    build.build()
    lrp.load()
    global KIND
    KIND = lrp.LRP_Q_MEAN | lrp.LRP_Q_VARIANCE | lrp.LRP_Q_SAMPLES


def _gap_rank(lam, lo, hi):
    """A rank k in [lo, hi] at the largest relative spectral gap (so the
    rank-k projector, hence every query, is unique)."""
    gaps = lam[lo - 1:hi] / lam[lo:hi + 1]
    return int(np.argmax(gaps)) + lo


@pytest.fixture(scope="module")
def models(tmp_path_factory):
    d = tmp_path_factory.mktemp("srv")
    specs = [
        synth.small_spec(dim=2, n=31, nt=24, obs_every=3, n_obs=16, sigma=1e-2, alpha=0.05, seed=61),
        synth.small_spec(dim=3, n=7, nt=10, obs_every=2, n_obs=12, sigma=1e-2, alpha=0.05, with_kappa=True,
                         seed=62),
    ]
    out = []
    for i, spec in enumerate(specs):
        P = OProblem(spec)
        lam, V = ospec.eig_dense(P.hessian_explicit())
        k = _gap_rank(lam, 6, 20)
        out.append((spec, P, lam[:k], V[:, :k], k, str(d / f"m{i}.bin")))
    return out


def _requests(models, n, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        m = i % len(models)
        spec, P, *_ = models[m]
        u = P.prior_half(synth.normal_block(P.nx, 1, seed + 10 * i)[:, 0])
        sigma = float(10 ** rng.uniform(-2.5, -1.5))
        y = P.forward(u) + sigma * synth.normal_block(P.n_data, 1, seed + 10 * i + 1)[:, 0]
        pts = synth.query_nodes(P.nx, 1 + (37 * i) % 60, seed + 10 * i + 2)
        xi = synth.normal_block(P.nx, 1 + i % 3, seed + 10 * i + 3)
        reqs.append((m, y, sigma, pts, xi))
    return reqs


def _serve(models, reqs, **cfg):
    srv = lrp.Server(**cfg)
    ids = [srv.add_model(spec, k, precision=lrp.LRP_MIXED, block=4, eig_tol=1e-9, factors_path=path)[0]
           for spec, P, lam, V, k, path in models]
    tickets = [srv.submit(ids[m], KIND, y_obs=y, sigma=s, points=p, xi=x) for m, y, s, p, x in reqs]
    outs = [srv.wait(t, timeout=300.0) for t in tickets]
    info = srv.info()
    srv.close()
    return outs, info


def test_server_matches_oracle_and_alone(models):
    reqs = _requests(models, 10, 500)
    mixed, info = _serve(models, reqs, slots=3, max_batch=4, max_samples=4, max_points=64)
    assert info["served"] == len(reqs) and info["pending"] == 0
    assert max(o["stats"]["batch"] for o in mixed) > 1  # something really was batched
    alone, _ = _serve(models, reqs, slots=1, max_batch=1, max_samples=4, max_points=64)
    for (m, y, s, pts, xi), a, b in zip(reqs, mixed, alone):
        spec, P, lam, V, k, _ = models[m]
        m_ref = opost.mean_lowrank(P, lam, V, y, sigma=s)
        v_ref = opost.variance_lowrank(P, lam, V, pts, sigma=s)
        s_ref = opost.samples_lowrank(P, lam, V, m_ref, xi, sigma=s)
        assert relerr(a["mean"], m_ref) < 1e-6
        assert relerr(a["variance"], v_ref) < 1e-6
        assert relerr(a["samples"], s_ref) < 1e-6
        # the same request alone and in the mix
        for key in ("mean", "variance", "samples"):
            assert relerr(a[key], b[key]) < 1e-9, key
        assert a["latency_ms"] > 0


def test_server_budget_evicts_and_readmits(models):
    reqs = _requests(models, 8, 900)
    ref, _ = _serve(models, reqs, slots=2, max_batch=2, max_samples=4, max_points=64)
    # learn one model's footprint, then give room for about one at a time
    srv = lrp.Server(slots=1, max_batch=2, max_samples=4, max_points=64)
    mids = [srv.add_model(spec, k, precision=lrp.LRP_MIXED, block=4, eig_tol=1e-9, factors_path=path)[0]
            for spec, P, lam, V, k, path in models]
    for mid in mids:
        srv.wait(srv.submit(mid, lrp.LRP_Q_VARIANCE, points=[0]))
    per_model = srv.info()["device_bytes"]
    srv.close()
    outs, info = _serve(models, reqs, hbm_budget=int(0.75 * per_model), slots=1, max_batch=2, max_samples=4,
                        max_points=64)
    assert info["evictions"] >= 2 and info["admissions"] >= 3
    assert any(o["stats"]["admitted"] for o in outs[2:])
    for a, b in zip(outs, ref):
        for key in ("mean", "variance", "samples"):
            assert relerr(a[key], b[key]) < 1e-9


def test_server_rejects_what_cannot_fit_and_bad_input(models):
    spec, P, lam, V, k, path = models[0]
    srv = lrp.Server(hbm_budget=4096, slots=1, max_points=16)
    mid, _ = srv.add_model(spec, k, precision=lrp.LRP_MIXED, block=4, eig_tol=1e-9, factors_path=path)
    t = srv.submit(mid, lrp.LRP_Q_VARIANCE, points=[1, 2])
    with pytest.raises(lrp.LrpError) as e:
        srv.wait(t, timeout=120.0)
    assert e.value.status == lrp.LRP_EBUDGET
    with pytest.raises(lrp.LrpError):
        srv.submit(mid, lrp.LRP_Q_VARIANCE, points=[P.nx])  # node out of range
    with pytest.raises(lrp.LrpError):
        srv.submit(mid + 5, lrp.LRP_Q_VARIANCE, points=[0])  # unknown model
    with pytest.raises(lrp.LrpError):
        srv.submit(mid, lrp.LRP_Q_VARIANCE, points=list(range(17)))  # above max_points
    srv.close()
