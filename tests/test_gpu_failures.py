"""Failure paths of the C ABI, each made on the host (no GPU fault, trap or
hang): an iteration cap that a solve cannot meet (LRP_ENOCONV, outputs and
stats still filled), a Lanczos basis cap (LRP_ENOCONV with a usable
posterior), an injected device-allocation failure (LRP_ENOMEM, the context
stays usable), a bounded wait on a busy server (LRP_ETIMEOUT, the ticket
stays valid) and corrupt checkpoints (LRP_EINVAL)."""
import struct

import numpy as np
import pytest

import synth
from oracle.problem import Problem as OProblem

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
    yield
    lrp.lrp_debug_fail_alloc(-1)


def _spec():
    return synth.small_spec(dim=2, n=31, nt=12, obs_every=2, n_obs=10, sigma=1e-2, alpha=0.05, seed=71)


@pytest.mark.parametrize("precision", [lrp.LRP_FP64, lrp.LRP_MIXED])
def test_pcg_cap_gives_enoconv_with_outputs(precision):
    """A solve that cannot reach its tolerance within its caps (FP64: one PCG
    iteration; mixed: a tolerance below what FP64 refinement reaches, so the
    refinement cap binds) still writes finite outputs and its statistics, and
    returns LRP_ENOCONV."""
    spec = _spec()
    cap = dict(pcg_maxit=1) if precision == lrp.LRP_FP64 else dict(solve_rtol=1e-18)
    G = lrp.lrp_setup_problem(spec, precision=precision, **cap)
    X = synth.normal_block(G.nx, 3, 2)
    Y, st = lrp.lrp_hessian_apply(G, X)
    assert st["status"] == lrp.LRP_ENOCONV, st
    assert np.all(np.isfinite(Y)) and np.abs(Y).max() > 0
    assert st["n_solves"] > 0 and st["pcg_iters_max"] >= 1
    assert st["max_rel_residual"] > (1e-10 if precision == lrp.LRP_FP64 else 1e-18)
    assert "tolerance" in lrp.lrp_last_error() or lrp.lrp_last_error() != ""
    # the same problem without the cap converges
    G2 = lrp.lrp_setup_problem(spec, precision=precision)
    _, st2 = lrp.lrp_hessian_apply(G2, X)
    assert st2["status"] == lrp.LRP_OK, st2


def test_query_reports_enoconv(tmp_path):
    """A query whose solves miss their tolerance reports LRP_ENOCONV (the
    factors come from a converged run, saved and loaded into a problem with
    pcg_maxit = 1; the checkpoint hash covers the problem, not the solver
    settings)."""
    spec = _spec()
    G = lrp.lrp_setup_problem(spec, precision=lrp.LRP_FP64)
    post, st = lrp.lrp_lowrank_posterior(G, k=6, block=2, eig_tol=1e-9)
    assert st["status"] == lrp.LRP_OK
    path = str(tmp_path / "f.bin")
    lrp.lrp_posterior_save(post, path)
    y = synth.normal_block(G.n_data, 1, 3)[:, 0]
    xi = synth.normal_block(G.nx, 2, 4)
    kind = lrp.LRP_Q_MEAN | lrp.LRP_Q_VARIANCE | lrp.LRP_Q_SAMPLES
    ok = lrp.lrp_posterior_query(post, kind, y_obs=y, points=np.arange(8, dtype=np.int32), xi=xi)
    assert ok["status"] == lrp.LRP_OK
    Gc = lrp.lrp_setup_problem(spec, precision=lrp.LRP_FP64, pcg_maxit=1)
    postc = lrp.lrp_posterior_load(Gc, path)
    out = lrp.lrp_posterior_query(postc, kind, y_obs=y, points=np.arange(8, dtype=np.int32), xi=xi)
    assert out["status"] == lrp.LRP_ENOCONV
    assert np.all(np.isfinite(out["mean"])) and np.all(np.isfinite(out["samples"]))
    # the variance needs no solve: identical to the converged handle's
    np.testing.assert_array_equal(out["variance"], ok["variance"])


def test_basis_cap_gives_enoconv_with_usable_posterior():
    """max_basis below what k pairs need at eig_tol: LRP_ENOCONV, and the
    posterior holds the Ritz pairs found so far (orthonormal vectors)."""
    G = lrp.lrp_setup_problem(_spec(), precision=lrp.LRP_FP64)
    post, st = lrp.lrp_lowrank_posterior(G, k=8, block=2, eig_tol=1e-12, max_basis=8)
    assert st["status"] == lrp.LRP_ENOCONV, st
    assert st["k_converged"] < 8 and st["n_matvec"] <= 10
    lam, V = post.eigs(vectors=True)
    assert len(lam) >= 1 and np.all(np.diff(lam) <= 0)
    assert np.max(np.abs(V.T @ V - np.eye(V.shape[1]))) < 1e-10


def test_injected_allocation_failure_gives_enomem():
    """The next device allocation fails as on a full device: the call returns
    LRP_ENOMEM, and the problem and context stay usable."""
    spec = _spec()
    P = OProblem(spec)
    G = lrp.lrp_setup_problem(spec, precision=lrp.LRP_FP64)
    X = synth.normal_block(G.nx, 2, 5)
    ref = P.hessian_apply(X)
    lrp.lrp_debug_fail_alloc(0)  # host input -> the staging allocation fails
    with pytest.raises(lrp.LrpError) as e:
        lrp.lrp_hessian_apply(G, X)
    assert e.value.status == lrp.LRP_ENOMEM
    Y, st = lrp.lrp_hessian_apply(G, X)  # disarmed after one failure
    assert np.max(np.abs(Y - ref)) <= 1e-10 * np.abs(ref).max(), st
    # a failure part-way through problem setup: nothing half-built is returned
    for after in (0, 3, 6):
        lrp.lrp_debug_fail_alloc(after)
        with pytest.raises(lrp.LrpError) as e:
            lrp.lrp_setup_problem(spec, precision=lrp.LRP_FP64)
        assert e.value.status == lrp.LRP_ENOMEM
    lrp.lrp_debug_fail_alloc(-1)
    G3 = lrp.lrp_setup_problem(spec, precision=lrp.LRP_FP64)
    Y3, _ = lrp.lrp_hessian_apply(G3, X)
    assert np.max(np.abs(Y3 - ref)) <= 1e-10 * np.abs(ref).max()


def test_server_wait_times_out_and_ticket_stays_valid():
    """A bounded wait on a request queued behind others returns LRP_ETIMEOUT
    without consuming the ticket; an unbounded wait then gets the result."""
    spec = synth.small_spec(dim=2, n=63, nt=200, obs_every=1, n_obs=40, sigma=1e-2, alpha=0.05, seed=72)
    srv = lrp.Server(slots=1, max_batch=1, max_samples=8, max_points=16)
    mid, _ = srv.add_model(spec, k=4, precision=lrp.LRP_MIXED, block=4, eig_tol=1e-6)
    nd = spec.n_obs * len(spec.obs_steps)
    y = synth.normal_block(nd, 1, 6)[:, 0]
    tickets = [srv.submit(mid, lrp.LRP_Q_MEAN, y_obs=y) for _ in range(6)]
    with pytest.raises(lrp.LrpError) as e:
        srv.wait(tickets[-1], timeout=1e-4)
    assert e.value.status == lrp.LRP_ETIMEOUT
    outs = [srv.wait(t) for t in tickets]
    assert all(o["status"] == lrp.LRP_OK for o in outs)
    for o in outs[1:]:
        np.testing.assert_array_equal(o["mean"], outs[0]["mean"])
    srv.close()


def test_corrupt_checkpoints_are_rejected(tmp_path):
    spec = _spec()
    G = lrp.lrp_setup_problem(spec, precision=lrp.LRP_FP64)
    post, _ = lrp.lrp_lowrank_posterior(G, k=4, block=2, eig_tol=1e-9)
    path = tmp_path / "c.bin"
    lrp.lrp_posterior_save(post, str(path))
    raw = path.read_bytes()
    assert not (tmp_path / "c.bin.tmp").exists()
    # header: 8-byte magic, then hash, nx, k (uint64)
    bad_k = raw[:24] + struct.pack("<Q", G.nx + 1) + raw[32:]
    for i, blob in enumerate((bad_k, raw[:-8], b"LRPOST01")):
        p = tmp_path / f"bad{i}.bin"
        p.write_bytes(blob)
        with pytest.raises(lrp.LrpError) as e:
            lrp.lrp_posterior_load(G, str(p))
        assert e.value.status == lrp.LRP_EINVAL
    other = lrp.lrp_setup_problem(synth.small_spec(dim=2, n=31, nt=12, obs_every=2, n_obs=10, seed=73))
    with pytest.raises(lrp.LrpError) as e:
        lrp.lrp_posterior_load(other, str(path))
    assert e.value.status == lrp.LRP_EINVAL


def test_mixed_inner_cap_is_not_a_failure():
    """In the mixed path pcg_maxit caps each FP32 inner solve; the FP64
    refinement around it still reaches the tolerance (more refinement
    sweeps), so the apply converges and reports LRP_OK."""
    spec = _spec()
    P = OProblem(spec)
    G = lrp.lrp_setup_problem(spec, precision=lrp.LRP_MIXED, pcg_maxit=2)
    X = synth.normal_block(G.nx, 2, 8)
    Y, st = lrp.lrp_hessian_apply(G, X)
    assert st["status"] == lrp.LRP_OK and st["pcg_iters_max"] <= 2, st
    ref = P.hessian_apply(X)
    assert np.max(np.abs(Y - ref)) <= 1e-6 * np.abs(ref).max()
